"""Seeded synthetic inputs for the multi-RHS Dirac mat-vec.

This module only draws random numbers: gauge links, spinor sources,
cotangents and gauge transformations.  It holds none of the Dirac-operator
arithmetic, so both the FP64 CPU oracle (test infrastructure) and the CUDA
path may be fed from it.

Canonical host layouts (C order, complex):
  links   V[t, z, y, x, mu, a, b]        mu = 0..3 <-> x, y, z, t; V_mu(x) is the
                                          parallel transporter from x+mu to x
  Wilson / Brillouin spinors psi[t, z, y, x, v, spin, colour]
  staggered spinors          psi[t, z, y, x, v, colour]

Conventions:
  * "complex Gaussian N(0,1)": real and imaginary parts iid N(0, 1/2), so
    E|z|^2 = 1.
  * Haar SU(N): QR of a complex Gaussian matrix with the phase fix
    Q' = Q diag(R_ii/|R_ii|) (Mezzadri, Notices AMS 54 (2007) 592), which is
    Haar on U(N); dividing by the principal N-th root of det Q' lands in
    SU(N).
  * near-identity SU(N): U = exp(i eps H) with H = (A + A^dag)/2 minus its
    trace part, A complex Gaussian; the exponential is taken through the
    eigendecomposition of H.
Every field draws from its own stream keyed by (seed, stream id), so a
field does not depend on which other fields were generated before it.
"""
from __future__ import annotations

import numpy as np

# stream ids: one per kind of field, so that (seed, kind) picks the stream
STREAM_LINKS = 1
STREAM_SOURCE = 2
STREAM_COTANGENT = 3
STREAM_GAUGE = 4
STREAM_MISC = 5


def rng(seed: int, stream: int) -> np.random.Generator:
    """A numpy Generator keyed by (seed, stream)."""
    return np.random.default_rng([int(seed), int(stream)])


def complex_gaussian(shape, seed: int, stream: int = STREAM_SOURCE,
                     dtype=np.complex128) -> np.ndarray:
    """iid complex Gaussian entries with E|z|^2 = 1."""
    g = rng(seed, stream)
    n = int(np.prod(shape))
    re = g.standard_normal(n, dtype=np.float64)
    im = g.standard_normal(n, dtype=np.float64)
    z = np.empty(n, dtype=np.complex128)
    z.real = re * np.sqrt(0.5)
    z.imag = im * np.sqrt(0.5)
    return z.reshape(shape).astype(dtype, copy=False)


def haar_sun(n: int, Nc: int, seed: int, stream: int = STREAM_LINKS,
             chunk: int = 1 << 20) -> np.ndarray:
    """n Haar-random SU(Nc) matrices, shape (n, Nc, Nc), complex128."""
    g = rng(seed, stream)
    out = np.empty((n, Nc, Nc), dtype=np.complex128)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        m = hi - lo
        z = (g.standard_normal((m, Nc, Nc)) + 1j * g.standard_normal((m, Nc, Nc))) * np.sqrt(0.5)
        q, r = np.linalg.qr(z)
        d = np.diagonal(r, axis1=1, axis2=2)
        ph = d / np.abs(d)
        q = q * ph[:, None, :]
        det = np.linalg.det(q)
        root = np.exp(1j * np.angle(det) / Nc)
        out[lo:hi] = q / root[:, None, None]
    return out


def near_identity_sun(n: int, Nc: int, eps: float, seed: int,
                      stream: int = STREAM_LINKS, chunk: int = 1 << 20) -> np.ndarray:
    """n matrices exp(i eps H), H traceless Hermitian Gaussian; shape (n, Nc, Nc)."""
    g = rng(seed, stream)
    out = np.empty((n, Nc, Nc), dtype=np.complex128)
    eye = np.eye(Nc)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        m = hi - lo
        a = (g.standard_normal((m, Nc, Nc)) + 1j * g.standard_normal((m, Nc, Nc))) * np.sqrt(0.5)
        h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
        tr = np.trace(h, axis1=1, axis2=2).real / Nc
        h = h - tr[:, None, None] * eye
        w, q = np.linalg.eigh(h)
        ph = np.exp(1j * eps * w)
        out[lo:hi] = (q * ph[:, None, :]) @ np.conj(np.swapaxes(q, 1, 2))
    return out


def lattice_shape(L):
    """(Nx, Ny, Nz, Nt) -> canonical site shape (Nt, Nz, Ny, Nx)."""
    Nx, Ny, Nz, Nt = (int(v) for v in L)
    return (Nt, Nz, Ny, Nx)


def gauge_links(L, Nc: int, kind: str, seed: int, eps: float = 0.3) -> np.ndarray:
    """Links V[t,z,y,x,mu,a,b] (complex128).

    kind: "haar" (Haar SU(Nc)), "near_identity" (exp(i eps H)), "unit" (V = 1).
    """
    sh = lattice_shape(L)
    nlink = int(np.prod(sh)) * 4
    if kind == "haar":
        m = haar_sun(nlink, Nc, seed)
    elif kind == "near_identity":
        m = near_identity_sun(nlink, Nc, eps, seed)
    elif kind == "unit":
        m = np.broadcast_to(np.eye(Nc, dtype=np.complex128), (nlink, Nc, Nc)).copy()
    else:
        raise ValueError(f"unknown link kind {kind!r}")
    return m.reshape(sh + (4, Nc, Nc))


def gauge_transform(L, Nc: int, seed: int) -> np.ndarray:
    """Haar-random g(x), shape (t, z, y, x, a, b)."""
    sh = lattice_shape(L)
    return haar_sun(int(np.prod(sh)), Nc, seed, stream=STREAM_GAUGE).reshape(sh + (Nc, Nc))


def spinor(L, Nv: int, Ns: int, Nc: int, seed: int, stream: int = STREAM_SOURCE,
           dtype=np.complex128) -> np.ndarray:
    """Gaussian source; Ns = 4 (Wilson, Brillouin) or 1 (staggered, squeezed)."""
    sh = lattice_shape(L)
    if Ns == 1:
        return complex_gaussian(sh + (Nv, Nc), seed, stream, dtype)
    return complex_gaussian(sh + (Nv, Ns, Nc), seed, stream, dtype)


def round_to(x: np.ndarray, prec: str) -> np.ndarray:
    """Round complex128 data to a storage precision and return it as complex128.

    prec: "f64", "f32", "bf16", "f16".  bf16 uses round-to-nearest-even on
    the float32 bit pattern; f16 uses numpy's IEEE half.
    """
    if prec == "f64":
        return np.asarray(x, dtype=np.complex128)
    if prec == "f32":
        return np.asarray(x, dtype=np.complex64).astype(np.complex128)
    r = np.ascontiguousarray(np.asarray(x).real, dtype=np.float64)
    i = np.ascontiguousarray(np.asarray(x).imag, dtype=np.float64)
    if prec == "f16":
        return r.astype(np.float16).astype(np.float64) + 1j * i.astype(np.float16).astype(np.float64)
    if prec == "bf16":
        return _bf16(r) + 1j * _bf16(i)
    raise ValueError(prec)


def _bf16(a: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
