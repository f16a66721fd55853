"""GB300 multi-right-hand-side Dirac mat-vec (arXiv:1808.05506): Python binding.

A thin ctypes layer over the C ABI of libdirac_gb300.so (include/dirac.h).
The functions dirac_* carry the same names and arguments as the C entry
points (plain integers and pointers); the Dirac class marshals torch tensors
(device memory, the current CUDA stream) onto them.  Every step of the
computation runs in the library's CUDA kernels; there is no CPU fallback, and
loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import weakref
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdirac_gb300.so")

STAGGERED, WILSON, BRILLOUIN = 0, 1, 2
OPS = {"staggered": STAGGERED, "wilson": WILSON, "brillouin": BRILLOUIN}
F64, F32, BF16, F16 = 0, 1, 2, 3
PRECS = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}
CANONICAL, INTERNAL = 0, 1

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA = 0, 1, 2, 3, 4
NOT_CONVERGED, BREAKDOWN, TIMEOUT = 5, 6, 7

_lib = None


class DiracError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libdirac_gb300.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double

# name -> (restype, argtypes); the C signatures of include/dirac.h
SIGNATURES = {
    "dirac_version": (ctypes.c_char_p, []),
    "dirac_status_string": (ctypes.c_char_p, [I]),
    "dirac_create": (I, [ctypes.POINTER(P), I, I, I, I, I, I, I, D, I, P]),
    "dirac_destroy": (I, [P]),
    "dirac_set_mass": (I, [P, D]),
    "dirac_set_stream": (I, [P, P]),
    "dirac_set_links": (I, [P, P, I, I]),
    "dirac_field_bytes": (I, [P, I, ctypes.POINTER(ctypes.c_size_t)]),
    "dirac_pack": (I, [P, P, P]),
    "dirac_unpack": (I, [P, P, P]),
    "dirac_apply": (I, [P, P, P, I]),
    "dirac_apply_dagger": (I, [P, P, P, I]),
    "dirac_set_kernel_config": (I, [P, I, I, I]),
    "dirac_get_kernel_config": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
    "dirac_set_site_order": (I, [P, I]),
    "dirac_apply_host": (I, [P, P, P, I]),
    "dirac_get_site_order": (I, [P, ctypes.POINTER(I)]),
    "dirac_set_link_format": (I, [P, I]),
    "dirac_get_link_format": (I, [P, ctypes.POINTER(I)]),
    "dirac_set_preconditioner": (I, [P, I]),
    "dirac_set_residual_arithmetic": (I, [P, I]),
    "dirac_set_inner_fields": (I, [P, I]),
    "dirac_get_inner_fields": (I, [P, ctypes.POINTER(I)]),
    "dirac_get_residual_arithmetic": (I, [P, ctypes.POINTER(I)]),
    "dirac_get_preconditioner": (I, [P, ctypes.POINTER(I)]),
    "dirac_last_error": (ctypes.c_char_p, [P]),
    "dirac_solve": (I, [P, P, P, D, I, I, D, P, P]),
    "dirac_force": (I, [P, P, P, P, I]),
    "dirac_autotune": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
    "dirac_solve_batched": (I, [P, I, P, P, P, P, D, I, I, D, P, P, P]),
    "dirac_apply_static": (I, [P, P, P, I]),
    "dirac_sync": (I, [P]),
}


class SystemStats(ctypes.Structure):
    """dirac_system_stats of include/dirac.h."""
    _fields_ = [("converged", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("residual_max", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    """dirac_solve_stats of include/dirac.h."""
    _fields_ = [("outer_iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int),
                ("sweeps", ctypes.c_int), ("fp64_sweeps", ctypes.c_int), ("even_odd", ctypes.c_int),
                ("df_residual", ctypes.c_int), ("split_fields", ctypes.c_int),
                ("residual_max", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _declare(L):
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _fwd(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    f.__doc__ = f"ctypes call of the C entry point {name} (include/dirac.h)."
    return f


for _n in SIGNATURES:
    globals()[_n] = _fwd(_n)


def last_error(h) -> str:
    s = lib().dirac_last_error(h)
    return s.decode() if s else ""


def check(status: int, h=None, what: str = "") -> None:
    if status != OK:
        raise DiracError(status, f"{what}: {last_error(h)}")


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _is_device(t) -> bool:
    return bool(t.is_cuda)


class Dirac:
    """One operator on one lattice, bound to a handle of the C library.

    op: "staggered" | "wilson" | "brillouin"; L = (Nx, Ny, Nz, Nt);
    mass: staggered m, Wilson kappa, Brillouin m0; prec: "f64" | "f32" | "bf16" | "f16".
    Canonical spinor tensors have shape (Nt, Nz, Ny, Nx, Nv, 4, 3) (staggered:
    (Nt, Nz, Ny, Nx, Nv, 3)) and dtype complex128 for f64, complex64 otherwise.
    """

    def __init__(self, op: str, L, Nv: int, mass: float, prec: str = "f32", Nc: int = 3,
                 stream=None):
        torch = _torch()
        self.op, self.L, self.Nv, self.mass, self.prec = op, tuple(int(v) for v in L), int(Nv), float(mass), prec
        self.Nc = Nc
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._stream = stream
        h = P()
        st = lib().dirac_create(ctypes.byref(h), OPS[op], Nc, *self.L, self.Nv, float(mass),
                                PRECS[prec], _stream_ptr(stream))
        check(st, None, "dirac_create")
        self.h = h
        self.canon_dtype = torch.complex128 if prec == "f64" else torch.complex64
        self.links_generation = 0   # advanced by every set_links
        self._links = None          # what set_links last loaded (set_links_if_changed)

    def close(self):
        if getattr(self, "h", None):
            lib().dirac_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes ---------------------------------------------------------------
    @property
    def spin_shape(self):
        return (self.Nv, 3) if self.op == "staggered" else (self.Nv, 4, 3)

    @property
    def canonical_shape(self):
        Nx, Ny, Nz, Nt = self.L
        return (Nt, Nz, Ny, Nx) + self.spin_shape

    def field_bytes(self, layout=INTERNAL) -> int:
        n = ctypes.c_size_t()
        check(lib().dirac_field_bytes(self.h, layout, ctypes.byref(n)), self.h, "dirac_field_bytes")
        return n.value

    def new_internal(self):
        torch = _torch()
        return torch.empty(self.field_bytes(INTERNAL), dtype=torch.uint8, device=self.device)

    def new_canonical(self):
        torch = _torch()
        return torch.empty(self.canonical_shape, dtype=self.canon_dtype, device=self.device)

    # -- argument checks: the C ABI takes bare pointers and cannot see a
    # tensor's size or type, so every tensor is checked here before its
    # pointer is passed (a wrong dtype or size would make a kernel read or
    # write past the end of the buffer)
    def _n_canonical(self) -> int:
        n = 1
        for d in self.canonical_shape:
            n *= d
        return n

    def _canon_in(self, t, what="field", device=True, dtype=None):
        """A canonical input: converted to `dtype` (default: this handle's complex dtype)."""
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_complex():
            raise TypeError(f"{what} must be a complex tensor")
        if device and not _is_device(t):
            raise ValueError(f"{what} must be a CUDA tensor")
        if t.numel() != self._n_canonical():
            raise ValueError(f"{what} has {t.numel()} entries, the canonical field {self.canonical_shape} "
                             f"has {self._n_canonical()}")
        return t.to(self.canon_dtype if dtype is None else dtype).contiguous()

    def _canon_out(self, t, what="out"):
        if t.dtype != self.canon_dtype or not _is_device(t) or not t.is_contiguous() \
                or t.numel() != self._n_canonical():
            raise ValueError(f"{what} must be a contiguous CUDA {self.canon_dtype} tensor with "
                             f"{self._n_canonical()} entries")
        return t

    def _internal(self, t, what="internal field"):
        torch = _torch()
        if t.dtype != torch.uint8 or not _is_device(t) or not t.is_contiguous() \
                or t.numel() < self.field_bytes(INTERNAL):
            raise ValueError(f"{what} must be a contiguous CUDA uint8 buffer of at least "
                             f"{self.field_bytes(INTERNAL)} bytes (new_internal)")
        return t

    def _sync_stream(self):
        check(lib().dirac_set_stream(self.h, _stream_ptr(self._stream)), self.h, "dirac_set_stream")

    # -- calls ------------------------------------------------------------------
    def set_links(self, V, remember: bool = True):
        """V: canonical links (Nt, Nz, Ny, Nx, 4, 3, 3), complex128/complex64, host or device.
        remember: record V (a weak reference and its version counter) for
        set_links_if_changed; False when V may change without its version
        counter moving (writes through V.data)."""
        torch = _torch()
        if V.dtype not in (torch.complex128, torch.complex64):
            raise TypeError("links must be complex128 or complex64")
        Nx, Ny, Nz, Nt = self.L
        if V.numel() != Nx * Ny * Nz * Nt * 4 * self.Nc * self.Nc:
            raise ValueError(f"links must have {Nx * Ny * Nz * Nt * 4 * self.Nc * self.Nc} entries "
                             "(Nt, Nz, Ny, Nx, 4, 3, 3)")
        key = self._links_key(V)
        Vc = V.contiguous()
        self._links = None
        self._load_links(Vc, F64 if Vc.dtype == torch.complex128 else F32)
        # what was loaded: a weak reference to the tensor object (a tensor
        # freed and replaced by another at the same address does not match)
        # and its version
        self._links = (key, weakref.ref(V)) if remember else None
        self.links_generation = getattr(self, "links_generation", 0) + 1

    def _load_links(self, Vc, prec):
        self._sync_stream()
        check(lib().dirac_set_links(self.h, _ptr(Vc), prec, 1 if Vc.is_cuda else 0), self.h, "dirac_set_links")

    @staticmethod
    def _links_key(V):
        return (V.data_ptr(), V._version, tuple(V.shape), tuple(V.stride()), V.dtype, str(V.device))

    def set_links_if_changed(self, V):
        """set_links(V) unless V is the tensor last loaded and unchanged since:
        the same memory, shape, dtype and version counter (which every tracked
        in-place change advances; writes through V.data are not tracked, so
        after those call set_links).  Returns True if the links were loaded."""
        rec = getattr(self, "_links", None)
        if rec is not None and rec[1]() is V and rec[0] == self._links_key(V):
            return False
        self.set_links(V)
        return True

    def set_mass(self, mass: float):
        check(lib().dirac_set_mass(self.h, float(mass)), self.h, "dirac_set_mass")
        self.mass = float(mass)

    def pack(self, canonical, out=None):
        canonical = self._canon_in(canonical, "canonical")
        out = self.new_internal() if out is None else self._internal(out, "out")
        self._sync_stream()
        check(lib().dirac_pack(self.h, _ptr(out), _ptr(canonical)), self.h, "dirac_pack")
        return out

    def unpack(self, internal, out=None):
        internal = self._internal(internal)
        out = self.new_canonical() if out is None else self._canon_out(out)
        self._sync_stream()
        check(lib().dirac_unpack(self.h, _ptr(out), _ptr(internal)), self.h, "dirac_unpack")
        return out

    def apply(self, x, out=None, dagger: bool = False, layout=None):
        """out = D x (or D^+ x).  x canonical (complex tensor) or internal (uint8 buffer)."""
        if layout is None:
            layout = INTERNAL if x.dtype == _torch().uint8 else CANONICAL
        if layout == INTERNAL:
            x = self._internal(x, "x")
            out = self.new_internal() if out is None else self._internal(out, "out")
        else:
            x = self._canon_in(x, "x")
            out = self.new_canonical() if out is None else self._canon_out(out)
        self._sync_stream()
        fn = lib().dirac_apply_dagger if dagger else lib().dirac_apply
        check(fn(self.h, _ptr(out), _ptr(x), layout),
              self.h, "dirac_apply_dagger" if dagger else "dirac_apply")
        return out

    def apply_host(self, x, out=None, dagger: bool = False, sync: bool = True):
        """out = D x (or D^+ x) for canonical fields in host memory (CPU tensors; pinned
        memory overlaps the copies with the sweep); see dirac_apply_host.  With sync the
        call returns once out is written, else after enqueuing (then call sync())."""
        torch = _torch()
        if x.device.type != "cpu" or x.dtype != self.canon_dtype or tuple(x.shape) != self.canonical_shape:
            raise ValueError(f"x must be a CPU {self.canon_dtype} tensor of shape {self.canonical_shape}")
        x = x.contiguous()
        if out is None:
            out = torch.empty(self.canonical_shape, dtype=self.canon_dtype, pin_memory=x.is_pinned())
        elif out.device.type != "cpu" or out.dtype != self.canon_dtype or not out.is_contiguous():
            raise ValueError("out must be a contiguous CPU tensor of the canonical dtype")
        self._sync_stream()
        check(lib().dirac_apply_host(self.h, _ptr(out), _ptr(x), 1 if dagger else 0), self.h, "dirac_apply_host")
        if sync:
            self.sync()
        return out

    def apply_dagger(self, x, out=None, layout=None):
        return self.apply(x, out=out, dagger=True, layout=layout)

    def solve(self, b, x0=None, tol: float = 1e-10, max_outer: int = 30, max_inner: int = 2000,
              inner_tol: float | None = None):
        """Solve D x = b (defect correction, FP64 outer residual).  b, x0: canonical
        complex128 device tensors.  Returns (x, per-rhs relative residuals, stats dict, status)."""
        import numpy as np
        torch = _torch()
        if inner_tol is None:
            inner_tol = 0.0   # the library's default for the inner solve that runs
        b = self._canon_in(b, "b", dtype=torch.complex128)
        x = torch.zeros_like(b) if x0 is None else self._canon_in(x0, "x0", dtype=torch.complex128).clone()
        res = np.zeros(self.Nv, dtype=np.float64)
        st = SolveStats()
        self._sync_stream()
        status = lib().dirac_solve(self.h, _ptr(x), _ptr(b), float(tol), int(max_outer), int(max_inner),
                                   float(inner_tol), res.ctypes.data_as(P), ctypes.byref(st))
        if status not in (OK, NOT_CONVERGED):
            check(status, self.h, "dirac_solve")
        return x, res, st.as_dict(), status

    def solve_batched(self, bs, masses, x0s=None, tol: float = 1e-10, max_outer: int = 30,
                      max_inner: int = 4000, inner_tol: float | None = None):
        """Solve the systems D(m_i) x_i = b_i sharing this handle's links; this
        handle's Nv is the number of resident right-hand-side slots.  bs: list of
        canonical complex128 device tensors (Nt,Nz,Ny,Nx,Nv_i,...).  Returns
        (xs, per-column residuals, per-system stats, totals, status)."""
        import numpy as np
        torch = _torch()
        if inner_tol is None:
            inner_tol = 0.0   # the library's default for the inner solve that runs
        nsys = len(bs)
        Nx, Ny, Nz, Nt = self.L
        for i, b in enumerate(bs):
            if not b.is_complex() or not _is_device(b) or b.dim() != 4 + len(self.spin_shape) \
                    or tuple(b.shape[:4]) != (Nt, Nz, Ny, Nx) \
                    or tuple(b.shape[5:]) != self.spin_shape[1:] or b.shape[4] < 1:
                raise ValueError(f"b[{i}] must be a complex CUDA tensor (Nt, Nz, Ny, Nx, Nv_i) + "
                                 f"{self.spin_shape[1:]}")
        bs = [b.to(torch.complex128).contiguous() for b in bs]
        if x0s is not None and [tuple(x.shape) for x in x0s] != [tuple(b.shape) for b in bs]:
            raise ValueError("x0s must have the shapes of bs")
        xs = [torch.zeros_like(b) for b in bs] if x0s is None else \
            [x.to(torch.complex128).contiguous().clone() for x in x0s]
        nv = (ctypes.c_int * nsys)(*[int(b.shape[4]) for b in bs])
        ms = (ctypes.c_double * nsys)(*[float(m) for m in masses])
        xp = (ctypes.c_void_p * nsys)(*[x.data_ptr() for x in xs])
        bp = (ctypes.c_void_p * nsys)(*[b.data_ptr() for b in bs])
        res = np.zeros(sum(nv), dtype=np.float64)
        sst = (SystemStats * nsys)()
        st = SolveStats()
        self._sync_stream()
        status = lib().dirac_solve_batched(self.h, nsys, ctypes.cast(nv, P), ctypes.cast(ms, P), ctypes.cast(xp, P),
                                           ctypes.cast(bp, P), float(tol), int(max_outer), int(max_inner),
                                           float(inner_tol), res.ctypes.data_as(P), ctypes.cast(sst, P),
                                           ctypes.byref(st))
        if status not in (OK, NOT_CONVERGED):
            check(status, self.h, "dirac_solve_batched")
        sys_stats = [{k: getattr(x, k) for k, _ in SystemStats._fields_} for x in sst]
        return xs, res, sys_stats, st.as_dict(), status

    def force(self, psi, g, out=None):
        """Link gradient of Re <g, D psi>: canonical links shape, complex128 (f64) / complex64."""
        torch = _torch()
        Nx, Ny, Nz, Nt = self.L
        psi = self._canon_in(psi, "psi")
        g = self._canon_in(g, "g")
        nl = Nx * Ny * Nz * Nt * 4 * self.Nc * self.Nc
        if out is None:
            out = torch.empty((Nt, Nz, Ny, Nx, 4, 3, 3), dtype=self.canon_dtype, device=self.device)
        elif out.dtype != self.canon_dtype or not _is_device(out) or not out.is_contiguous() or out.numel() != nl:
            raise ValueError(f"out must be a contiguous CUDA {self.canon_dtype} tensor with {nl} entries")
        self._sync_stream()
        check(lib().dirac_force(self.h, _ptr(out), _ptr(psi), _ptr(g), CANONICAL), self.h, "dirac_force")
        return out

    def set_kernel_config(self, R: int, block: int, variant: int = 0):
        """Launch shape: R right-hand sides per thread, block, variant (0 direct,
        1 groups in block, 2 Wilson t-march, 3 pipelined Wilson, 5 Wilson x-rows
        per warp); see dirac_set_kernel_config."""
        check(lib().dirac_set_kernel_config(self.h, R, block, variant), self.h, "dirac_set_kernel_config")

    def set_site_order(self, tchunk: int):
        """Site order of variants 0 and 1 (0 lexicographic, else t-chunks); see dirac_set_site_order."""
        check(lib().dirac_set_site_order(self.h, tchunk), self.h, "dirac_set_site_order")

    def site_order(self) -> int:
        t = I()
        check(lib().dirac_get_site_order(self.h, ctypes.byref(t)), self.h, "dirac_get_site_order")
        return t.value

    def set_link_format(self, fmt: int):
        """Links the apply sweeps read: 0 the plain links (Brillouin: 40 stored W),
        1 Wilson / staggered two-row links (special unitary links only),
        Brillouin all 80 W per site; see dirac_set_link_format."""
        check(lib().dirac_set_link_format(self.h, fmt), self.h, "dirac_set_link_format")

    def link_format(self) -> int:
        f = I()
        check(lib().dirac_get_link_format(self.h, ctypes.byref(f)), self.h, "dirac_get_link_format")
        return f.value

    def set_preconditioner(self, mode: int):
        """Inner solves: 1 even-odd Schur complement where it applies, 0 whole lattice;
        see dirac_set_preconditioner."""
        check(lib().dirac_set_preconditioner(self.h, mode), self.h, "dirac_set_preconditioner")

    def preconditioner(self) -> int:
        t = I()
        check(lib().dirac_get_preconditioner(self.h, ctypes.byref(t)), self.h, "dirac_get_preconditioner")
        return t.value

    def set_inner_fields(self, mode: int):
        """16-bit Wilson even-odd inner solves: 1 split fields (FP32 e, r, t; 16-bit p, s), 0 all
        16-bit; see dirac_set_inner_fields."""
        check(lib().dirac_set_inner_fields(self.h, mode), self.h, "dirac_set_inner_fields")

    def inner_fields(self) -> int:
        t = I()
        check(lib().dirac_get_inner_fields(self.h, ctypes.byref(t)), self.h, "dirac_get_inner_fields")
        return t.value

    def set_residual_arithmetic(self, mode: int):
        """Outer residual: 1 double-float sweep, 0 FP64; see dirac_set_residual_arithmetic."""
        check(lib().dirac_set_residual_arithmetic(self.h, mode), self.h, "dirac_set_residual_arithmetic")

    def residual_arithmetic(self) -> int:
        t = I()
        check(lib().dirac_get_residual_arithmetic(self.h, ctypes.byref(t)), self.h,
              "dirac_get_residual_arithmetic")
        return t.value

    def autotune(self, force: bool = False):
        """Pick the fastest (R, block, variant) for this handle; returns (R, block, variant, ms per sweep)."""
        R, B, Pp, ms = I(), I(), I(), D()
        self._sync_stream()
        check(lib().dirac_autotune(self.h, 1 if force else 0, ctypes.byref(R), ctypes.byref(B), ctypes.byref(Pp),
                                   ctypes.byref(ms)), self.h, "dirac_autotune")
        return R.value, B.value, Pp.value, ms.value

    def sync(self):
        """Wait for the handle's stream; raises DiracError(TIMEOUT) if a kernel's
        bounded wait ran out."""
        check(lib().dirac_sync(self.h), self.h, "dirac_sync")

    def kernel_config(self):
        R, B, Pp = I(), I(), I()
        check(lib().dirac_get_kernel_config(self.h, ctypes.byref(R), ctypes.byref(B), ctypes.byref(Pp)), self.h,
              "dirac_get_kernel_config")
        return R.value, B.value, Pp.value


VARIANTS = {"staggered": (0, 1, 6), "wilson": (0, 1, 2, 3, 5, 6), "brillouin": (0, 1, 7)}


def config_supported(op: str, prec: str, R: int, block: int, variant: int, L=None) -> bool:
    """The rule dirac_set_kernel_config applies (without a handle); L = (Nx, Ny, Nz, Nt)
    is needed for variants 5 and 6."""
    if block < 32 or block > 256 or block % 32:
        return False
    if variant == 4:
        return False   # not used
    if variant == 7:   # tensor cores: Brillouin, 16-bit storage
        return op == "brillouin" and prec in ("bf16", "f16") and R == 1 and block == 128
    if variant in (5, 6):
        if prec == "f64" or block > (192 if variant == 5 else 64) or L is None:
            return False
        if op == "wilson":
            if not 1 <= R <= 2:
                return False
        elif not (op == "staggered" and variant == 6 and R in (1, 2, 4, 6)):
            return False
        return 32 % L[0] == 0 and (L[0] * L[1] * L[2]) % 32 == 0
    if op == "staggered" and R not in (1, 2, 4, 6):
        return False
    if op != "staggered" and not 1 <= R <= 4:
        return False
    if variant == 0:
        return True
    if op == "wilson" and prec == "f64":
        return False
    if variant == 1:
        return block <= 64
    if variant == 2:
        return op == "wilson" and R <= 2 and block <= 128
    if variant == 3 and op == "wilson":
        k = {"f64": 12, "f32": 6, "bf16": 3, "f16": 3}[prec]
        lb = {"f64": 16, "f32": 8, "bf16": 4, "f16": 4}[prec]
        return (R * k * 16 + 9 * lb) * 3 * block <= 227 * 1024
    return False


# per-site, per-right-hand-side model flop counts at Nc = 3 (complex mult-add = 8,
# add = 2, real x complex = 2): staggered 64 Nc^2 - 2 Nc, Wilson 128 Nc^2 + 72 Nc,
# Brillouin 80 * 4 (8 Nc^2 - 2 Nc) + 8 Nc sum_dir (1 + |dir|_1) + 984
def flops_per_site_rhs(op: str, Nc: int = 3) -> int:
    if op == "staggered":
        return 64 * Nc * Nc - 2 * Nc
    if op == "wilson":
        return 128 * Nc * Nc + 72 * Nc
    if op == "brillouin":
        hops = sum(1 + k for k, n in ((1, 8), (2, 24), (3, 32), (4, 16)) for _ in range(n))
        return 80 * 4 * (8 * Nc * Nc - 2 * Nc) + 8 * Nc * hops + 984
    raise ValueError(op)


def bytes_per_site(op: str, Nv: int, prec: str, Nc: int = 3, link_format: int = 0) -> int:
    """Algorithmic HBM bytes per site of one sweep: links once, in and out once.
    link_format 1 (dirac_set_link_format): Wilson / staggered read two rows of
    each link, Brillouin all 80 W."""
    c = {"f64": 16, "f32": 8, "bf16": 4, "f16": 4}[prec]
    nlink = {"staggered": 4, "wilson": 4, "brillouin": 40}[op]
    per_link = Nc * Nc
    if link_format == 1:
        if op == "brillouin":
            nlink = 80
        else:
            per_link = (Nc - 1) * Nc
    ns = 1 if op == "staggered" else 4
    return nlink * per_link * c + 2 * ns * Nc * Nv * c
