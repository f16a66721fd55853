"""FP64 CPU oracle for the multi-RHS Dirac mat-vec (arXiv:1808.05506).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this package.  It shares
no code with the CUDA path (paper_1808_05506_gb300) and never imports it.

Two independent parts:
  * dirac_oracle.c (through ctypes): the gather form of D_S, D_W, D_B written
    term by term from the paper's equations (Sec. 3, Eq. def_wils, Eqs.
    def_bril / def_der / def_lap), the brute-force W_dir of Tab. tab:off-axis
    (average over all k! hop orderings), the explicit adjoint, and the link
    gradient of L = Re <g, D psi>.
  * dense.py: a numpy assembly of the same operators as dense matrices, built
    from hop matrices (W_dir by the recursive form of the path average), and
    the free-field momentum-space symbols in closed form.  It is what the C
    oracle is pinned against on small lattices.

Arrays use the canonical layouts of the synth module (complex128):
  V[t,z,y,x,mu,a,b], psi[t,z,y,x,v,spin,colour] (staggered: [..., v, colour]).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dirac_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_LIB32_PATH = os.path.join(_HERE, "_liboracle_f32.so")
_lib = None
_lib32 = None
_lock = threading.Lock()

OPS = {"staggered": 0, "wilson": 1, "brillouin": 2}


def build(force: bool = False, fp32: bool = False) -> str:
    """Compile dirac_oracle.c into oracle/_liboracle.so with gcc + OpenMP (and,
    with fp32, its single-precision instance _liboracle_f32.so, which only the
    CPU-baseline timing uses)."""
    path = _LIB32_PATH if fp32 else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared"] + (["-DORACLE_FP32"] if fp32 else []) + \
        ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _declare(L):
    P = ctypes.c_void_p
    L.oracle_apply.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_double,
                               P, P, P, P, P, ctypes.c_long, ctypes.c_int]
    L.oracle_brillouin_W.argtypes = [ctypes.c_int, P, P, P, ctypes.c_long, P]
    L.oracle_force.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_double,
                               P, P, P, P]
    L.oracle_row_terms.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_double, P,
                                   ctypes.c_long, P, P]
    L.oracle_gamma.argtypes = [ctypes.c_int, P]
    L.oracle_set_threads.argtypes = [ctypes.c_int]
    L.oracle_set_threads.restype = ctypes.c_int
    return L


def lib(fp32: bool = False):
    global _lib, _lib32
    with _lock:
        if fp32:
            if _lib32 is None:
                _lib32 = _declare(ctypes.CDLL(build(fp32=True)))
            return _lib32
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


def set_threads(n: int, fp32: bool = False) -> int:
    """OpenMP threads of the oracle's loops (n < 1: one per processor); returns
    the number its next parallel loop uses."""
    return int(lib(fp32).oracle_set_threads(int(n)))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dims(V):
    """canonical V[t,z,y,x,mu,a,b] -> (L = (Nx,Ny,Nz,Nt), Nc)"""
    Nt, Nz, Ny, Nx = V.shape[:4]
    return (Nx, Ny, Nz, Nt), V.shape[-1]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def gamma(mu: int) -> np.ndarray:
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().oracle_gamma(mu, _ptr(out))
    return out


def apply(op: str, V, psi, mass: float, sites=None, dagger: bool = False, W81=None,
          fp32: bool = False) -> np.ndarray:
    """D psi (or D^dagger psi) in FP64.

    mass: staggered m, Wilson / Brillouin bare mass m0 (not kappa).
    sites: None (whole lattice; result has psi's shape) or an int array of
    lexicographic site indices s = x + Nx (y + Ny (z + Nz t)); then the result
    is [len(sites), Nv, (4,) Nc].
    W81: optional precomputed brillouin_W(V) (all sites) to avoid rebuilding
    W per row.
    fp32: the single-precision instance (complex64 in and out), for timing only.
    """
    cast = (lambda a: np.ascontiguousarray(a, dtype=np.complex64)) if fp32 else _c128
    V = cast(V)
    psi = cast(psi)
    L, Nc = _dims(V)
    Ns = 1 if op == "staggered" else 4
    vol = int(np.prod(L))
    Nv = psi.shape[4]
    blk = psi.shape[4:]
    Larr = np.array(L, dtype=np.int32)
    odt = np.complex64 if fp32 else np.complex128
    if sites is None:
        out = np.zeros((vol,) + blk, dtype=odt)
        sp, ns = None, vol
    else:
        sp = np.ascontiguousarray(sites, dtype=np.int64)
        ns = len(sp)
        out = np.zeros((ns,) + blk, dtype=odt)
    if W81 is not None:
        W81 = cast(W81)
    rc = lib(fp32).oracle_apply(OPS[op], Nc, _ptr(Larr), Nv, float(mass), _ptr(V), _ptr(W81),
                            _ptr(psi), _ptr(out), _ptr(sp), ns, 1 if dagger else 0)
    if rc:
        raise RuntimeError("oracle_apply failed")
    assert out.shape[1:] == blk and (Ns == 4) == (len(blk) == 3)
    if sites is None:
        return out.reshape(psi.shape)
    return out


def brillouin_W(V, sites=None) -> np.ndarray:
    """W_dir(x) for all 81 dir (dir = sum_mu (d_mu+1) 3^mu), brute force over k! paths.

    Returns [t,z,y,x,81,Nc,Nc] (sites None) or [len(sites),81,Nc,Nc]."""
    V = _c128(V)
    L, Nc = _dims(V)
    Larr = np.array(L, dtype=np.int32)
    if sites is None:
        out = np.zeros(V.shape[:4] + (81, Nc, Nc), dtype=np.complex128)
        sp, ns = None, int(np.prod(L))
    else:
        sp = np.ascontiguousarray(sites, dtype=np.int64)
        ns = len(sp)
        out = np.zeros((ns, 81, Nc, Nc), dtype=np.complex128)
    lib().oracle_brillouin_W(Nc, _ptr(Larr), _ptr(V), _ptr(sp), ns, _ptr(out))
    return out


def force(op: str, V, psi, g, mass: float) -> np.ndarray:
    """dL/dV for L = Re <g, D psi>, as dL/dRe V + i dL/dIm V; shape of V."""
    V = _c128(V)
    psi = _c128(psi)
    g = _c128(g)
    L, Nc = _dims(V)
    Larr = np.array(L, dtype=np.int32)
    F = np.zeros_like(V)
    rc = lib().oracle_force(OPS[op], Nc, _ptr(Larr), psi.shape[4], float(mass), _ptr(V),
                            _ptr(psi), _ptr(g), _ptr(F))
    if rc:
        raise RuntimeError("oracle_force: unsupported operator")
    return F


def row_offsets(op: str, V, site: int = 0, mass: float = 0.0):
    """The (offset, spin) list of the terms of one row of D (for the count pins)."""
    V = _c128(V)
    L, Nc = _dims(V)
    Larr = np.array(L, dtype=np.int32)
    nmax = lib().oracle_max_terms()
    offs = np.zeros((nmax, 4), dtype=np.int32)
    spins = np.zeros(nmax, dtype=np.int32)
    n = lib().oracle_row_terms(OPS[op], Nc, _ptr(Larr), float(mass), _ptr(V), int(site),
                               _ptr(offs), _ptr(spins))
    return offs[:n].copy(), spins[:n].copy()


def kappa_to_m0(kappa: float) -> float:
    """Wilson hopping parameter -> bare mass, m0 = 1/(2 kappa) - 4."""
    return 1.0 / (2.0 * kappa) - 4.0


def site_index(L, x, y, z, t):
    Nx, Ny, Nz, Nt = L
    return x + Nx * (y + Ny * (z + Nz * t))
