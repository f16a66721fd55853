"""The even-odd (Schur-complement) decomposition the GPU inner solver relies
on, checked on the oracle's dense matrices.

Sec. 4 names the even-odd decomposition as the next tuning step; the split
follows from the stencils: with every extent even, the Wilson and staggered
hopping terms link only sites of opposite parity, so D restricted to one
parity is a times the identity (a = 4 + m0, or m), and D e = r is solved
exactly by the Schur complement of the odd sites, S = a - H_oe H_eo / a, and
the even reconstruction e_e = (r_e - H_eo e_o) / a.  S inherits gamma5
hermiticity (Wilson: CGLS with S^+ = gamma5 S gamma5) and, for staggered, is
hermitian and definite with the sign of m (CG).  The Brillouin operator's
2- and 4-hop terms link equal parities: it has no such split.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import dense

NS = {"staggered": 1, "wilson": 4, "brillouin": 4}


def _parity_of_rows(L, ns, nc=3):
    Nx, Ny, Nz, Nt = L
    t, z, y, x = np.meshgrid(np.arange(Nt), np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    par = ((x + y + z + t) % 2).ravel()                 # site order s = x + Nx (y + ...)
    return np.repeat(par, ns * nc)                      # rows ordered (site, spin, colour)


def _blocks(op, L, mass, seed):
    V = synth.gauge_links(L, 3, "near_identity", seed)
    D = dense.dense(op, V, mass)
    par = _parity_of_rows(L, NS[op])
    e, o = np.flatnonzero(par == 0), np.flatnonzero(par == 1)
    return D, e, o


@pytest.mark.parametrize("op,mass", [("wilson", oracle.kappa_to_m0(0.122)), ("staggered", 0.07),
                                     ("staggered", -0.07)])
def test_schur_complement_solves_the_whole_system(op, mass):
    L = (4, 2, 4, 2)
    D, e, o = _blocks(op, L, mass, 600)
    a = 4.0 + mass if op == "wilson" else mass
    # the hopping term links opposite parities only
    assert np.array_equal(D[np.ix_(e, e)], a * np.eye(len(e)))
    assert np.array_equal(D[np.ix_(o, o)], a * np.eye(len(o)))
    H_eo, H_oe = D[np.ix_(e, o)], D[np.ix_(o, e)]
    rng = np.random.default_rng(601)
    r = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
    S = a * np.eye(len(o)) - H_oe @ H_eo / a
    x = np.zeros_like(r)
    x[o] = np.linalg.solve(S, r[o] - H_oe @ r[e] / a)
    x[e] = (r[e] - H_eo @ x[o]) / a
    assert np.linalg.norm(D @ x - r) / np.linalg.norm(r) < 1e-12
    assert np.linalg.norm(x - np.linalg.solve(D, r)) / np.linalg.norm(x) < 1e-10
    # the residual of D e = r after the reconstruction is the Schur residual on
    # the odd sites and zero on the even ones, for any odd e_o
    y = np.zeros_like(r)
    y[o] = rng.standard_normal(len(o)) + 1j * rng.standard_normal(len(o))
    y[e] = (r[e] - H_eo @ y[o]) / a
    res = r - D @ y
    assert np.abs(res[e]).max() < 1e-12 * np.abs(r).max()
    assert np.allclose(res[o], (r[o] - H_oe @ r[e] / a) - S @ y[o], atol=1e-12)
    if op == "staggered":
        # S = m + H_eo^+ H_eo / m: hermitian, definite with the sign of m
        assert np.allclose(S, S.conj().T, atol=1e-13)
        ev = np.linalg.eigvalsh(S)
        assert np.all(np.sign(ev) == np.sign(mass)) and np.abs(ev).min() >= abs(mass) - 1e-12
    else:
        # gamma5-hermitian: S^+ = gamma5 S gamma5 on the odd sites
        g5 = np.kron(np.ones(len(o) // 12), np.repeat(np.diag(dense.gamma5()).real, 3))
        assert np.allclose(S.conj().T, g5[:, None] * S * g5[None, :], atol=1e-13)


def test_brillouin_links_equal_parities():
    L = (4, 2, 4, 2)
    D, e, o = _blocks("brillouin", L, 0.05, 602)
    Dee = D[np.ix_(e, e)]
    off = Dee - np.diag(np.diag(Dee))
    assert np.abs(off).max() > 1e-3   # the 2- and 4-hop terms: no even-odd split


def test_odd_extent_breaks_the_split():
    # periodic wrap-around of an odd extent links equal parities
    L = (3, 2, 2, 2)
    D, e, o = _blocks("wilson", L, 0.1, 603)
    Dee = D[np.ix_(e, e)]
    assert np.abs(Dee - np.diag(np.diag(Dee))).max() > 1e-3
