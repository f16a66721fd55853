"""dirac_apply_static: the canonical apply without device allocation.

It is for callers that cannot allocate device memory while they run: loops
that must not trigger the device synchronisation of cudaMalloc / cudaFree,
and hosts whose device memory is all reserved by their own allocator.  Its
work fields live in a fixed array of the library's device image, shared by
every call.  The checks: the result equals the allocating entry point's bit
for bit (same kernels, same launch shape) and the FP64 oracle's within the
FP32 bar, on two calls in a row; a lattice whose volume leaves padding in the
last block of 32 sites runs after a call that filled the shared array with
NaN, so a sweep that read padding sites would show it; a warmed call takes no
device memory; oversize fields are refused.  This file runs last so that a
failure here does not hide the results of the other GPU tests."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1808_05506_gb300 as dg
    torch.cuda.set_device(0)
    return dg


def _m0(op, mass):
    return oracle.kappa_to_m0(mass) if op == "wilson" else mass


def _max_rel_per_rhs(got, want):
    """max over right-hand sides of |got_v - want_v| / |want_v| (axis 4 is v)."""
    d = np.moveaxis(got - want, 4, 0).reshape(got.shape[4], -1)
    w = np.moveaxis(want, 4, 0).reshape(want.shape[4], -1)
    return float(np.max(np.linalg.norm(d, axis=1) / np.linalg.norm(w, axis=1)))


def _static(dg, D, y, x, dagger):
    return dg.dirac_apply_static(D.h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), int(dagger))


def _poison_shared_array(dg):
    """A call whose input is NaN everywhere leaves NaN in the first 1.2 MB of
    the shared array (its packed input and its output), which covers both work
    fields of the padded lattice below."""
    L, Nv = (8, 8, 4, 8), 3
    D = dg.Dirac("wilson", L, Nv, 0.124, "f32")
    D.set_links(torch.from_numpy(synth.gauge_links(L, 3, "unit", 0).astype(np.complex64)).cuda())
    x = torch.full(D.canonical_shape, float("nan"), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    assert _static(dg, D, y, x, 0) == dg.OK, dg.last_error(D.h)
    torch.cuda.synchronize()
    assert torch.isnan(torch.view_as_real(y)).all()
    D.close()


@pytest.mark.parametrize("L", [(8, 8, 4, 8), (6, 6, 6, 6)])
@pytest.mark.parametrize("op,mass", [("wilson", 0.124), ("staggered", 0.05), ("brillouin", 0.05)])
def test_static_apply_matches_apply_twice(dg, op, mass, L):
    Nv = 3
    ns = 1 if op == "staggered" else 4
    V = synth.round_to(synth.gauge_links(L, 3, "near_identity", 500), "f32")
    psi = synth.round_to(synth.spinor(L, Nv, ns, 3, 501), "f32")
    D = dg.Dirac(op, L, Nv, mass, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    x = torch.from_numpy(psi.astype(np.complex64)).cuda()
    if int(np.prod(L)) % 32:
        _poison_shared_array(dg)
    for dagger in (0, 1):
        ref = D.apply(x, dagger=bool(dagger))            # the allocating entry point
        torch.cuda.synchronize()
        want = oracle.apply(op, V, psi, _m0(op, mass), dagger=bool(dagger))
        for call in range(2):                             # two calls in a row share the array
            y = torch.full_like(x, float("nan"))
            st = _static(dg, D, y, x, dagger)
            assert st == dg.OK, dg.last_error(D.h)
            torch.cuda.synchronize()
            assert torch.equal(y, ref), (dagger, call)
            got = y.cpu().numpy().astype(np.complex128)
            assert _max_rel_per_rhs(got, want) <= 1e-6, (dagger, call)
    D.close()


def test_static_apply_takes_no_device_memory(dg):
    L, Nv = (8, 8, 8, 8), 4
    D = dg.Dirac("wilson", L, Nv, 0.122, "f32")
    D.set_links(torch.from_numpy(synth.gauge_links(L, 3, "near_identity", 502).astype(np.complex64)).cuda())
    x = torch.from_numpy(synth.spinor(L, Nv, 4, 3, 503).astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    for dagger in (0, 1):                                 # warm: kernels loaded, address known
        assert _static(dg, D, y, x, dagger) == dg.OK, dg.last_error(D.h)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for dagger in (0, 1, 0):
        assert _static(dg, D, y, x, dagger) == dg.OK, dg.last_error(D.h)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    D.close()


def test_static_apply_rejects_too_large(dg):
    L, Nv = (16, 16, 16, 16), 8                           # 2 x 50 MB of work fields > 64 MiB
    D = dg.Dirac("wilson", L, Nv, 0.12, "f32")
    D.set_links(torch.from_numpy(synth.gauge_links(L, 3, "unit", 0).astype(np.complex64)).cuda())
    x = D.new_canonical()
    y = D.new_canonical()
    st = _static(dg, D, y, x, 0)
    assert st == dg.ERR_INVALID_ARG
    assert "static area holds" in dg.last_error(D.h)
    D.close()
