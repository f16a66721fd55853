"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point include/dirac.h declares; argument validation answers with a
status before any device work.  No kernel is launched here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dg():
    from paper_1808_05506_gb300 import build
    build.build()
    import paper_1808_05506_gb300 as dg
    return dg


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"DIRAC_API\s+[\w\s\*]+?\b(dirac_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(dg):
    names = declared_symbols()
    assert "dirac_apply" in names and "dirac_create" in names
    L = ctypes.CDLL(dg.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    # the binding wraps exactly the declared entry points
    assert names == set(dg.SIGNATURES)


def test_version_and_status_strings(dg):
    assert b"sm_103a" in dg.dirac_version()
    assert dg.dirac_status_string(dg.ERR_INVALID_ARG) == b"invalid argument"
    assert dg.dirac_status_string(99) == b"unknown status"


def _create(dg, op=1, Nc=3, L=(4, 4, 4, 4), Nv=2, mass=0.12, prec=1):
    h = ctypes.c_void_p()
    st = dg.dirac_create(ctypes.byref(h), op, Nc, *L, Nv, mass, prec, None)
    return st, h


def test_create_validation(dg):
    assert _create(dg, Nc=4)[0] == dg.ERR_UNSUPPORTED
    assert _create(dg, L=(1, 4, 4, 4))[0] == dg.ERR_INVALID_ARG
    assert _create(dg, Nv=0)[0] == dg.ERR_INVALID_ARG
    assert _create(dg, op=1, mass=0.0)[0] == dg.ERR_INVALID_ARG     # Wilson takes kappa > 0
    assert b"kappa" in dg.dirac_last_error(None)
    assert _create(dg, op=7)[0] == dg.ERR_INVALID_ARG
    assert _create(dg, prec=9)[0] == dg.ERR_INVALID_ARG
    assert dg.dirac_create(None, 1, 3, 4, 4, 4, 4, 1, 0.1, 1, None) == dg.ERR_INVALID_ARG


def test_null_handle_calls(dg):
    assert dg.dirac_apply(None, None, None, 0) == dg.ERR_INVALID_ARG
    assert dg.dirac_set_preconditioner(None, 1) == dg.ERR_INVALID_ARG
    assert dg.dirac_get_preconditioner(None, None) == dg.ERR_INVALID_ARG
    assert dg.dirac_set_link_format(None, 1) == dg.ERR_INVALID_ARG
    assert dg.dirac_get_link_format(None, None) == dg.ERR_INVALID_ARG
    assert dg.dirac_set_residual_arithmetic(None, 1) == dg.ERR_INVALID_ARG
    assert dg.dirac_get_residual_arithmetic(None, None) == dg.ERR_INVALID_ARG
    assert dg.dirac_set_inner_fields(None, 1) == dg.ERR_INVALID_ARG
    assert dg.dirac_get_inner_fields(None, None) == dg.ERR_INVALID_ARG
    assert dg.dirac_set_links(None, None, 0, 0) == dg.ERR_INVALID_ARG
    assert dg.dirac_destroy(None) == dg.OK


def test_no_gpu_is_a_status_not_a_crash(dg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _create(dg)
    assert st == dg.ERR_CUDA


def test_missing_library_fails_loudly(dg, monkeypatch):
    monkeypatch.setattr(dg, "_lib", None)
    monkeypatch.setattr(dg, "LIB_PATH", os.path.join(ROOT, "nonexistent", "lib.so"))
    with pytest.raises(ImportError):
        dg.lib()


def test_flop_model_reproduces_paper_intensity_ratio(dg):
    """The per-site flop counts reproduce the paper's claim that D_B has about
    2.5x the computational intensity of D_W, almost independent of Nv (Sec. 5),
    under the paper's no-reuse byte count: every link (72 B) and every
    neighbour spinor (96 B per right-hand side) read per use, in sp."""
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    assert dg.flops_per_site_rhs("staggered") == 570
    assert dg.flops_per_site_rhs("wilson") == 1368
    assert dg.flops_per_site_rhs("brillouin") == 29208

    def intensity(op, Nv, fw=None):
        f = (fw or dg.flops_per_site_rhs(op)) * Nv
        nlink, nspin = (8, 9) if op == "wilson" else (80, 81)
        return f / (nlink * 72 + nspin * 96 * Nv)

    ratios = [intensity("brillouin", nv) / intensity("wilson", nv) for nv in (1, 4, 12, 1000)]
    assert all(2.2 < r < 2.6 for r in ratios)
    assert max(ratios) - min(ratios) < 0.15                      # almost invariant in Nv
    # the paper rounds to "a factor 2.5"
    assert abs(ratios[2] - gold["intensity_ratio_brillouin_over_wilson"]["value"]) < 0.2


def test_binding_calls_match_the_c_signatures(dg, monkeypatch):
    """Every Dirac method passes exactly the arguments its C entry point
    declares (checked against a stand-in library; no device work)."""
    import torch

    calls = []

    class FakeFn:
        def __init__(self, name):
            self.name = name

        def __call__(self, *args):
            argtypes = dg.SIGNATURES[self.name][1]
            assert len(args) == len(argtypes), (self.name, len(args), len(argtypes))
            calls.append(self.name)
            if self.name in ("dirac_solve", "dirac_solve_batched"):
                # inner_tol not given: 0, the library's choice for the inner solve that runs
                inner_tol = args[6] if self.name == "dirac_solve" else args[9]
                assert float(inner_tol) == 0.0, (self.name, inner_tol)
            return dg.OK if dg.SIGNATURES[self.name][0] is ctypes.c_int else b""

    class FakeLib:
        def __getattr__(self, name):
            assert name in dg.SIGNATURES, name
            return FakeFn(name)

    monkeypatch.setattr(dg, "_lib", FakeLib())
    monkeypatch.setattr(dg, "_is_device", lambda t: True)   # CPU tensors stand in for device ones
    monkeypatch.setattr(dg, "_stream_ptr", lambda stream=None: ctypes.c_void_p(0))
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    D = dg.Dirac.__new__(dg.Dirac)
    D.op, D.L, D.Nv, D.mass, D.prec, D.Nc = "wilson", (4, 4, 4, 4), 2, 0.12, "f32", 3
    D.device = torch.device("cpu")
    D._stream = None
    D.h = ctypes.c_void_p(1)
    D.canon_dtype = torch.complex64
    x = torch.zeros(D.canonical_shape, dtype=torch.complex64)
    V = torch.zeros((4, 4, 4, 4, 4, 3, 3), dtype=torch.complex64)
    D.set_links(V)
    D.set_mass(0.11)
    D.field_bytes()
    D.pack(x, out=torch.zeros(8, dtype=torch.uint8))
    D.unpack(torch.zeros(8, dtype=torch.uint8), out=x.clone())
    D.apply(torch.zeros(8, dtype=torch.uint8), out=torch.zeros(8, dtype=torch.uint8))
    D.apply(x, out=x.clone())
    D.apply_dagger(x, out=x.clone())
    D.apply_host(x, out=x.clone(), dagger=True, sync=False)
    D.force(x, x, out=V.clone())
    D.set_kernel_config(2, 128, 3)
    D.kernel_config()
    D.set_site_order(8)
    D.site_order()
    D.set_preconditioner(0)
    D.preconditioner()
    D.set_residual_arithmetic(0)
    D.residual_arithmetic()
    D.set_inner_fields(1)
    D.inner_fields()
    D.autotune()
    D.solve(x.to(torch.complex128), x0=x.to(torch.complex128))
    D.solve_batched([x.to(torch.complex128)] * 2, [0.12, 0.121])
    D.close()
    for name in ("dirac_set_links", "dirac_apply", "dirac_apply_dagger", "dirac_force", "dirac_solve",
                 "dirac_set_kernel_config", "dirac_get_kernel_config", "dirac_autotune", "dirac_destroy",
                 "dirac_solve_batched", "dirac_set_site_order", "dirac_get_site_order", "dirac_apply_host",
                 "dirac_set_preconditioner", "dirac_get_preconditioner", "dirac_set_residual_arithmetic",
                 "dirac_get_residual_arithmetic", "dirac_set_inner_fields", "dirac_get_inner_fields"):
        assert name in calls, name


def test_config_rule(dg):
    assert dg.config_supported("wilson", "f32", 2, 128, 3)
    assert not dg.config_supported("wilson", "f32", 4, 256, 3)
    assert not dg.config_supported("wilson", "f64", 1, 256, 3)
    assert dg.config_supported("wilson", "bf16", 4, 256, 3)
    assert dg.config_supported("staggered", "f32", 6, 32, 1)
    assert not dg.config_supported("staggered", "f32", 3, 32, 1)
    assert not dg.config_supported("brillouin", "f32", 2, 128, 1)
    assert not dg.config_supported("brillouin", "f32", 2, 128, 3)
    # x-rows per warp: Lx divides 32 and whole warps over the (x, y, z) volume
    assert dg.config_supported("wilson", "f32", 1, 192, 5, (32, 32, 32, 32))
    assert dg.config_supported("wilson", "bf16", 2, 32, 5, (8, 4, 2, 3))
    assert not dg.config_supported("wilson", "f32", 1, 64, 5, (24, 24, 24, 48))
    assert not dg.config_supported("wilson", "f32", 1, 64, 5, (4, 6, 2, 4))
    assert not dg.config_supported("wilson", "f32", 3, 64, 5, (32, 32, 32, 32))
    assert not dg.config_supported("wilson", "f64", 1, 64, 5, (32, 32, 32, 32))
    assert not dg.config_supported("wilson", "f32", 1, 256, 5, (32, 32, 32, 32))
    assert not dg.config_supported("staggered", "f32", 1, 64, 5, (32, 32, 32, 32))
    # x hops last: the same lattice rule, 32 or 64 sites per block
    assert dg.config_supported("wilson", "f32", 2, 64, 6, (32, 32, 32, 32))
    assert dg.config_supported("wilson", "f16", 1, 32, 6, (8, 4, 2, 3))
    assert not dg.config_supported("wilson", "f32", 2, 128, 6, (32, 32, 32, 32))
    assert not dg.config_supported("wilson", "f32", 3, 64, 6, (32, 32, 32, 32))
    assert not dg.config_supported("wilson", "f32", 2, 64, 6, (24, 24, 24, 48))
    assert not dg.config_supported("wilson", "f64", 1, 64, 6, (32, 32, 32, 32))
    assert not dg.config_supported("brillouin", "f32", 1, 64, 6, (32, 32, 32, 32))
    assert dg.config_supported("staggered", "f32", 6, 64, 6, (32, 32, 32, 32))
    assert not dg.config_supported("staggered", "f32", 3, 64, 6, (32, 32, 32, 32))
    assert not dg.config_supported("staggered", "f64", 2, 64, 6, (32, 32, 32, 32))
    # tensor cores: Brillouin with 16-bit storage, one launch shape
    assert dg.config_supported("brillouin", "bf16", 1, 128, 7)
    assert dg.config_supported("brillouin", "f16", 1, 128, 7)
    assert not dg.config_supported("brillouin", "f32", 1, 128, 7)
    assert not dg.config_supported("brillouin", "bf16", 2, 128, 7)
    assert not dg.config_supported("wilson", "bf16", 1, 128, 7)


def test_binding_rejects_mismatched_tensors(dg, monkeypatch):
    """The C ABI takes bare pointers, so the binding checks every tensor's type
    and size before passing it (a complex64 field handed to an FP64 handle
    would be read as twice its size); no C entry point is reached."""
    import torch

    class NoLib:
        def __getattr__(self, name):
            if name == "dirac_field_bytes":
                def fb(h, layout, out):
                    out._obj.value = 4096
                    return dg.OK
                return fb
            raise AssertionError(f"{name} must not be called")

    monkeypatch.setattr(dg, "_lib", NoLib())
    monkeypatch.setattr(dg, "_is_device", lambda t: True)
    D = dg.Dirac.__new__(dg.Dirac)
    D.op, D.L, D.Nv, D.mass, D.prec, D.Nc = "wilson", (4, 4, 4, 4), 2, 0.12, "f64", 3
    D.device = torch.device("cpu")
    D._stream = None
    D.h = ctypes.c_void_p(1)
    D.canon_dtype = torch.complex128
    good = torch.zeros(D.canonical_shape, dtype=torch.complex128)
    with pytest.raises(ValueError):
        D.pack(torch.zeros(10, dtype=torch.complex64))                      # wrong size
    with pytest.raises(TypeError):
        D.pack(torch.zeros(D.canonical_shape, dtype=torch.float64))         # not complex
    with pytest.raises(ValueError):
        D.unpack(torch.zeros(100, dtype=torch.uint8))                       # internal buffer too small
    with pytest.raises(ValueError):
        D.unpack(torch.zeros(4096, dtype=torch.uint8), out=good.to(torch.complex64))   # out of the wrong type
    with pytest.raises(ValueError):
        D.apply(good, out=torch.zeros(5, dtype=torch.complex128))
    with pytest.raises(ValueError):
        D.force(good, good[..., :1, :, :])
    with pytest.raises(ValueError):
        D.set_links(torch.zeros((4, 4, 4, 4, 4, 3), dtype=torch.complex128))
    with pytest.raises(ValueError):
        D.solve_batched([torch.zeros((4, 4, 4, 4, 2, 4), dtype=torch.complex128)], [0.12])
    monkeypatch.setattr(dg, "_is_device", lambda t: False)
    with pytest.raises(ValueError):
        D.pack(good)                                                        # host tensor


def test_binding_accepts_staggered_solve_shapes(dg, monkeypatch):
    """Staggered right-hand sides have no spin index: (Nt, Nz, Ny, Nx, Nv_i, 3)."""
    import torch
    seen = []

    class RecLib:
        def __getattr__(self, name):
            def f(*a):
                seen.append(name)
                return dg.OK
            return f

    monkeypatch.setattr(dg, "_lib", RecLib())
    monkeypatch.setattr(dg, "_is_device", lambda t: True)
    monkeypatch.setattr(dg, "_stream_ptr", lambda stream=None: ctypes.c_void_p(0))
    D = dg.Dirac.__new__(dg.Dirac)
    D.op, D.L, D.Nv, D.mass, D.prec, D.Nc = "staggered", (4, 4, 4, 4), 4, 0.1, "f32", 3
    D.device = torch.device("cpu")
    D._stream = None
    D.h = ctypes.c_void_p(1)
    D.canon_dtype = torch.complex64
    D.solve_batched([torch.zeros((4, 4, 4, 4, 3, 3), dtype=torch.complex128)], [0.1])
    assert "dirac_solve_batched" in seen
    with pytest.raises(ValueError):
        D.solve_batched([torch.zeros((4, 4, 4, 4, 3, 4, 3), dtype=torch.complex128)], [0.1])
