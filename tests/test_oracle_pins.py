"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the C oracle (gather form written term by term from the
paper's equations) to something other than itself: the independent dense
assembly (oracle/dense.py, hop matrices and the recursive path average),
closed-form free-field symbols, exact symmetries, printed counts and
coefficients (tests/golden/paper_constants.json), and finite differences.
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle
import synth
from oracle import dense

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
NS = {"staggered": 1, "wilson": 4, "brillouin": 4}


def _psi(L, op, Nv, seed):
    return synth.spinor(L, Nv, NS[op], 3, seed)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


# ---- gamma algebra (reading: Euclidean chiral basis) ------------------------

def test_gamma_algebra():
    g = [oracle.gamma(mu) for mu in range(4)]
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            assert np.allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2 * (mu == nu) * np.eye(4))
        assert np.allclose(g[mu], dense.gammas()[mu])
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


# ---- P1: gather oracle == dense brute force ---------------------------------

@pytest.mark.parametrize("op", ["staggered", "wilson", "brillouin"])
@pytest.mark.parametrize("L", [(2, 2, 2, 2), (2, 2, 2, 4), (3, 2, 2, 4), (4, 4, 2, 2)])
def test_dense_brute_force(op, L):
    V = synth.gauge_links(L, 3, "haar", 101)
    psi = _psi(L, op, 2, 102)
    m = 0.173
    D = dense.dense(op, V, m)
    assert _rel(oracle.apply(op, V, psi, m), dense.dense_apply(D, psi)) < 1e-14
    assert _rel(oracle.apply(op, V, psi, m, dagger=True), dense.dense_apply(D.conj().T, psi)) < 1e-14


@pytest.mark.parametrize("op", ["staggered", "wilson"])
def test_dense_brute_force_4444(op):
    L = (4, 4, 4, 4)
    V = synth.gauge_links(L, 3, "near_identity", 103)
    psi = _psi(L, op, 1, 104)
    D = dense.dense(op, V, -0.21)
    assert _rel(oracle.apply(op, V, psi, -0.21), dense.dense_apply(D, psi)) < 1e-14


def test_sampled_sites_match_full():
    L = (3, 4, 2, 4)
    V = synth.gauge_links(L, 3, "haar", 105)
    for op in ["staggered", "wilson", "brillouin"]:
        psi = _psi(L, op, 3, 106)
        full = oracle.apply(op, V, psi, 0.3).reshape((-1,) + psi.shape[4:])
        fulld = oracle.apply(op, V, psi, 0.3, dagger=True).reshape((-1,) + psi.shape[4:])
        sites = np.array([0, 5, 17, 95, 63])
        assert np.array_equal(oracle.apply(op, V, psi, 0.3, sites=sites), full[sites])
        assert np.allclose(oracle.apply(op, V, psi, 0.3, sites=sites, dagger=True), fulld[sites],
                           rtol=0, atol=1e-13)


# ---- P2: free field, closed forms --------------------------------------------

@pytest.mark.parametrize("op", ["wilson", "brillouin"])
def test_free_field_plane_waves(op):
    L = (4, 4, 2, 6)
    V = synth.gauge_links(L, 3, "unit", 0)
    chi = synth.complex_gaussian((2, 4, 3), 107)
    m = 0.05
    for p in dense.momenta(L):
        psi = dense.plane_wave(L, p, 2, 4, 3, chi)
        out = oracle.apply(op, V, psi, m)
        want = dense.plane_wave(L, p, 2, 4, 3, np.einsum("st,vta->vsa", dense.free_symbol(op, p, m), chi))
        assert np.abs(out - want).max() < 1e-13


def test_free_field_staggered_square():
    L = (4, 2, 4, 6)
    V = synth.gauge_links(L, 3, "unit", 0)
    chi = synth.complex_gaussian((1, 3), 108)
    for p in dense.momenta(L):
        psi = dense.plane_wave(L, p, 1, 1, 3, chi)
        dd = oracle.apply("staggered", V, oracle.apply("staggered", V, psi, 0.0), 0.0)
        assert np.abs(-dd - np.sum(np.sin(p) ** 2) * psi).max() < 1e-13


def _match(a, b):
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


@pytest.mark.parametrize("op", ["wilson", "brillouin"])
def test_free_spectrum_dense(op):
    """Eigenvalues of the position-space D (V=1) = union over p of those of D(p), x Nc."""
    L = (4, 2, 2, 4)
    V = synth.gauge_links(L, 3, "unit", 0)
    m = 0.1
    ev = np.linalg.eigvals(dense.dense(op, V, m))
    want = np.concatenate([np.repeat(np.linalg.eigvals(dense.free_symbol(op, p, m)), 3)
                           for p in dense.momenta(L)])
    assert _match(ev, want) < 1e-10
    # closed-form eigenvalues m + R(p) +- i sqrt(sum_mu s_mu^2), each 2 Nc times
    for p in dense.momenta(L)[:9]:
        S = dense.free_symbol(op, p, m)
        re = S[0, 0].real
        im = np.sqrt(sum(abs(np.trace(S @ dense.gammas()[mu]) / 4) ** 2 for mu in range(4)))
        assert _match(np.linalg.eigvals(S), np.array([re + 1j * im] * 2 + [re - 1j * im] * 2)) < 1e-12


def test_free_spectrum_staggered():
    L = (4, 4, 2, 2)
    V = synth.gauge_links(L, 3, "unit", 0)
    m = 0.2
    ev = np.linalg.eigvals(dense.dense("staggered", V, m))
    mod = np.sort(np.abs(ev - m) ** 2)
    want = np.sort(np.repeat([np.sum(np.sin(p) ** 2) for p in dense.momenta(L)], 3))
    assert np.abs(mod - want).max() < 1e-10
    assert np.abs(ev.real - m).max() < 1e-10


# ---- P3: symmetries ----------------------------------------------------------

@pytest.mark.parametrize("op", ["wilson", "brillouin"])
def test_gamma5_hermiticity(op):
    L = (3, 2, 4, 2)
    V = synth.gauge_links(L, 3, "haar", 109)
    psi = _psi(L, op, 2, 110)
    g5 = np.array([1, 1, -1, -1])[:, None]
    lhs = oracle.apply(op, V, psi, 0.37, dagger=True)
    rhs = g5 * oracle.apply(op, V, g5 * psi, 0.37)
    assert _rel(lhs, rhs) < 1e-14


def test_staggered_antihermitian_and_epsilon():
    L = (4, 2, 2, 4)
    V = synth.gauge_links(L, 3, "haar", 111)
    psi = _psi(L, "staggered", 2, 112)
    d = oracle.apply("staggered", V, psi, 0.0)
    assert _rel(oracle.apply("staggered", V, psi, 0.0, dagger=True), -d) < 1e-14
    Nx, Ny, Nz, Nt = L
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (Nt, Nz, Ny, Nx)], indexing="ij")
    eps = ((-1.0) ** (x + y + z + t))[..., None, None]
    assert _rel(eps * oracle.apply("staggered", V, eps * psi, 0.0), -d) < 1e-14


@pytest.mark.parametrize("op", ["staggered", "wilson", "brillouin"])
def test_adjoint_inner_product(op):
    L = (3, 2, 2, 3)
    V = synth.gauge_links(L, 3, "haar", 113)
    psi = _psi(L, op, 2, 114)
    phi = _psi(L, op, 2, 115)
    a = np.vdot(phi, oracle.apply(op, V, psi, 0.11))
    b = np.vdot(oracle.apply(op, V, phi, 0.11, dagger=True), psi)
    assert abs(a - b) < 1e-12 * abs(a)


# ---- P4: gauge covariance ----------------------------------------------------

def _gauge_rotate(V, g):
    Vg = np.empty_like(V)
    for mu in range(4):
        gp = np.roll(g, -1, axis=3 - mu)          # g(x + mu)
        Vg[..., mu, :, :] = g @ V[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    return Vg


@pytest.mark.parametrize("op", ["staggered", "wilson", "brillouin"])
def test_gauge_covariance(op):
    L = (2, 3, 2, 4)
    V = synth.gauge_links(L, 3, "near_identity", 116)
    g = synth.gauge_transform(L, 3, 117)
    psi = _psi(L, op, 2, 118)
    Vg = _gauge_rotate(V, g)
    if op == "staggered":
        gpsi = np.einsum("tzyxab,tzyxvb->tzyxva", g, psi)
        lhs = oracle.apply(op, Vg, gpsi, 0.3)
        rhs = np.einsum("tzyxab,tzyxvb->tzyxva", g, oracle.apply(op, V, psi, 0.3))
    else:
        gpsi = np.einsum("tzyxab,tzyxvsb->tzyxvsa", g, psi)
        lhs = oracle.apply(op, Vg, gpsi, 0.3)
        rhs = np.einsum("tzyxab,tzyxvsb->tzyxvsa", g, oracle.apply(op, V, psi, 0.3))
    assert _rel(lhs, rhs) < 1e-13


# ---- P5: W identities --------------------------------------------------------

def _dirs():
    return [(i % 3 - 1, (i // 3) % 3 - 1, (i // 9) % 3 - 1, (i // 27) % 3 - 1) for i in range(81)]


def _shift_sites(L, d):
    Nx, Ny, Nz, Nt = L
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (Nt, Nz, Ny, Nx)], indexing="ij")
    return (((x + d[0]) % Nx) + Nx * (((y + d[1]) % Ny) + Ny * (((z + d[2]) % Nz) + Nz * ((t + d[3]) % Nt)))).ravel()


def test_W_unit_and_pure_gauge():
    L = (2, 3, 2, 3)
    Vu = synth.gauge_links(L, 3, "unit", 0)
    W = oracle.brillouin_W(Vu)
    assert np.abs(W - np.eye(3)).max() < 1e-15
    g = synth.gauge_transform(L, 3, 119)
    Vg = _gauge_rotate(Vu, g)                     # pure gauge V_mu(x) = g(x) g(x+mu)^+
    W = oracle.brillouin_W(Vg).reshape(-1, 81, 3, 3)
    gf = g.reshape(-1, 3, 3)
    for i, d in enumerate(_dirs()):
        want = gf @ np.conj(np.swapaxes(gf[_shift_sites(L, d)], -1, -2))
        assert np.abs(W[:, i] - want).max() < 1e-13


def test_W_reflection_and_unitarity():
    L = (3, 2, 3, 2)
    V = synth.gauge_links(L, 3, "haar", 120)
    W = oracle.brillouin_W(V).reshape(-1, 81, 3, 3)
    nonunitary = 0
    reps = 0
    for i, d in enumerate(_dirs()):
        md = tuple(-c for c in d)
        j = _dirs().index(md)
        # W_{-dir}(x) = W_dir(x - dir)^dagger
        back = _shift_sites(L, md)
        assert np.abs(W[:, j] - np.conj(np.swapaxes(W[back, i], -1, -2))).max() < 1e-14
        k = sum(abs(c) for c in d)
        first = next((c for c in d if c != 0), 0)
        if first > 0:                                 # one representative of each +-dir pair
            reps += 1
            u = np.abs(W[:, i] @ np.conj(np.swapaxes(W[:, i], -1, -2)) - np.eye(3)).max()
            if k == 1:
                assert u < 1e-13
            elif u > 1e-3:
                nonunitary += 1
    assert reps == GOLD["stored_directions"]["value"]
    assert nonunitary == GOLD["non_special_unitary_directions"]["value"]


def test_W_bruteforce_equals_recursion():
    L = (2, 2, 3, 2)
    V = synth.gauge_links(L, 3, "haar", 121)
    Wb = oracle.brillouin_W(V)
    Wr = dense.W_from_hops(dense.hop_matrices_W(V), V)
    assert np.abs(Wb - Wr).max() < 1e-13


def test_W_sampled_sites():
    L = (3, 3, 2, 2)
    V = synth.gauge_links(L, 3, "haar", 122)
    full = oracle.brillouin_W(V).reshape(-1, 81, 3, 3)
    s = np.array([4, 0, 35, 17])
    assert np.array_equal(oracle.brillouin_W(V, sites=s), full[s])


# ---- P6: counts and normalisations -------------------------------------------

def test_table_counts_and_coefficients():
    tab = GOLD["off_axis_table"]
    by_k = {k: 0 for k in range(5)}
    for d in _dirs():
        by_k[sum(abs(c) for c in d)] += 1
    assert [by_k[k] for k in tab["hops"]] == tab["terms"]
    import math
    assert [math.factorial(k) for k in tab["hops"]] == tab["paths"]
    rho = np.array(GOLD["rho"]["values_times_432"]) / 432.0
    lam = np.array(GOLD["lambda"]["values_times_64"]) / 64.0
    assert np.allclose(rho, dense.RHO[1:]) and np.allclose(lam, dense.LAMBDA)
    # free-field grad^iso(p) -> i p: sum over dir with dir_mu != 0 of rho_k dir_mu^2 = 1
    s = sum(rho[sum(abs(c) for c in d) - 1] for d in _dirs() if d[0] != 0)
    assert abs(s - 1.0) < 1e-15
    # lap^bri annihilates constants: lambda_0 + sum_dir lambda_k = 0
    assert abs(lam[0] + sum(lam[sum(abs(c) for c in d)] for d in _dirs() if any(d))) < 1e-15


def test_row_term_counts():
    L = (3, 3, 3, 3)
    V = synth.gauge_links(L, 3, "haar", 123)
    offs, spins = oracle.row_offsets("brillouin", V, site=13)
    for mu in range(4):
        sel = {tuple(o) for o, s in zip(offs, spins) if s == mu}
        assert len(sel) == GOLD["derivative_points"]["value"]
        assert all(o[mu] != 0 for o in sel)
    lap = {tuple(o) for o, s in zip(offs, spins) if s < 0}
    assert len(lap) == GOLD["laplacian_points"]["value"]
    offs, spins = oracle.row_offsets("wilson", V, site=13)
    assert len({tuple(o) for o, s in zip(offs, spins) if s < 0}) == GOLD["wilson_laplacian_points"]["value"]


# ---- P7 / P8: continuum limit and doublers -----------------------------------

def _symbol_from_oracle(op, L, p, m):
    V = synth.gauge_links(L, 3, "unit", 0)
    S = np.zeros((4, 4), dtype=complex)
    for s in range(4):
        chi = np.zeros((1, 4, 3), dtype=complex)
        chi[0, s, 0] = 1
        out = oracle.apply(op, V, dense.plane_wave(L, p, 1, 4, 3, chi), m)
        S[:, s] = out[0, 0, 0, 0, 0, :, 0]
    return S


def test_continuum_limit_brillouin():
    g = dense.gammas()
    errs = []
    for n in (32, 64):
        L = (n, 2, 2, 2)
        p = np.array([2 * np.pi / n, 0, 0, 0])
        S = _symbol_from_oracle("brillouin", L, p, 0.0)
        nab = np.trace(g[0] @ S) / 4
        lap = -2 * (np.trace(S) / 4).real
        errs.append((abs(nab - 1j * p[0]), abs(lap + p[0] ** 2)))
    assert errs[1][0] < 2e-4 and errs[1][1] < 1e-5
    assert 6 < errs[0][0] / errs[1][0] < 10        # O(p^3)
    assert 12 < errs[0][1] / errs[1][1] < 20       # O(p^4)


def test_doublers():
    L = (2, 2, 2, 2)
    m = 0.05
    import itertools
    for bits in itertools.product((0, 1), repeat=4):
        if not any(bits):
            continue
        p = np.pi * np.array(bits, dtype=float)
        Sb = _symbol_from_oracle("brillouin", L, p, m)
        Sw = _symbol_from_oracle("wilson", L, p, m)
        assert np.abs(Sb - (m + 2) * np.eye(4)).max() < 1e-13
        assert np.abs(Sw - (m + 2 * sum(bits)) * np.eye(4)).max() < 1e-13


# ---- P9: translation covariance, kappa convention ----------------------------

@pytest.mark.parametrize("op", ["staggered", "wilson", "brillouin"])
def test_translation_covariance(op):
    L = (2, 4, 2, 4)      # shift by 2 sites keeps the staggered phases
    V = synth.gauge_links(L, 3, "haar", 124)
    psi = _psi(L, op, 1, 125)
    sh = dict(shift=(2, 2), axis=(2, 3))   # y and t by two sites
    out = oracle.apply(op, np.roll(V, **sh), np.roll(psi, **sh), 0.2)
    assert _rel(out, np.roll(oracle.apply(op, V, psi, 0.2), **sh)) < 1e-14


def test_kappa_convention():
    assert oracle.kappa_to_m0(0.125) == 0.0
    L = (2, 2, 3, 2)
    V = synth.gauge_links(L, 3, "haar", 126)
    psi = _psi(L, "wilson", 1, 127)
    k = 0.121
    D = oracle.apply("wilson", V, psi, oracle.kappa_to_m0(k))
    H = (oracle.apply("wilson", V, psi, -4.0) - 0.0 * psi)   # D at m0=-4 is -1/2 * hopping
    assert _rel(2 * k * D, psi + 2 * k * H) < 1e-14          # 2 kappa D_W = 1 - kappa * (hopping)


# ---- P11: link force ---------------------------------------------------------

def _loss(op, V, psi, g, m):
    return np.vdot(g, oracle.apply(op, V, psi, m)).real


@pytest.mark.parametrize("op", ["staggered", "wilson"])
def test_force_finite_differences(op):
    L = (2, 3, 2, 2)
    V = synth.gauge_links(L, 3, "haar", 128)
    psi = _psi(L, op, 2, 129)
    g = _psi(L, op, 2, 130)
    m = 0.15
    F = oracle.force(op, V, psi, g, m)
    rng = synth.rng(131, synth.STREAM_MISC)
    eps = 1e-6
    for _ in range(16):
        idx = tuple(int(rng.integers(0, n)) for n in V.shape[:5])
        dV = synth.complex_gaussian((3, 3), int(rng.integers(1 << 30)))
        Vp = V.copy()
        Vm = V.copy()
        Vp[idx] += eps * dV
        Vm[idx] -= eps * dV
        fd = (_loss(op, Vp, psi, g, m) - _loss(op, Vm, psi, g, m)) / (2 * eps)
        an = np.vdot(F[idx], dV).real
        assert abs(fd - an) < 1e-8 * max(1.0, abs(an))


@pytest.mark.parametrize("L", [(2, 3, 2, 3), (3, 3, 3, 3)])
def test_brillouin_force_finite_differences(L):
    """The Brillouin link gradient through the path products of W (Tab.
    tab:off-axis): L is a polynomial of degree 4 in V, so the central
    difference with eps = 1e-5 is exact to ~1e-10; extent 2 makes a path use
    the same link twice."""
    V = synth.gauge_links(L, 3, "haar", 140)
    psi = _psi(L, "brillouin", 2, 141)
    g = _psi(L, "brillouin", 2, 142)
    m = 0.07
    F = oracle.force("brillouin", V, psi, g, m)
    rng = synth.rng(143, synth.STREAM_MISC)
    eps = 1e-5
    for _ in range(10):
        idx = tuple(int(rng.integers(0, n)) for n in V.shape[:5])
        dV = synth.complex_gaussian((3, 3), int(rng.integers(1 << 30)))
        Vp = V.copy()
        Vm = V.copy()
        Vp[idx] += eps * dV
        Vm[idx] -= eps * dV
        fd = (_loss("brillouin", Vp, psi, g, m) - _loss("brillouin", Vm, psi, g, m)) / (2 * eps)
        an = np.vdot(F[idx], dV).real
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (idx, fd, an)


def test_brillouin_force_unit_links_closed_form():
    """At V = 1 every path product is 1, so the gradient of W_d(y),
    G_d(y) = sum_{v,s} g_v(y)_s (M_d psi_v(y+d))_s^+ with the paper's spin
    matrix M_d = rho_k (d . gamma) - lambda_k / 2 (Sec. 5, coefficients after
    def_lap), reaches each link of each of the k! orderings with weight 1/k!.
    A hop along mu that follows the subset S of the other hops of d sits at
    y + sum(S) and occurs in |S|! (k-1-|S|)! orderings; a -mu hop acts through
    V_mu at one site further back and receives the adjoint."""
    from itertools import combinations, product
    from math import factorial
    L = (2, 2, 3, 2)
    V = synth.gauge_links(L, 3, "unit", 0)
    psi = _psi(L, "brillouin", 1, 144)
    g = _psi(L, "brillouin", 1, 145)
    F = oracle.force("brillouin", V, psi, g, 0.0)
    rho = [0.0] + [r / 432.0 for r in GOLD["rho"]["values_times_432"]]
    lam = [x / 64.0 for x in GOLD["lambda"]["values_times_64"]]
    Nx, Ny, Nz, Nt = L
    vol = Nx * Ny * Nz * Nt
    G = dense.gammas()
    ps = psi.reshape(vol, 1, 4, 3)
    gs = g.reshape(vol, 1, 4, 3)

    def site(x):
        return x[0] + Nx * (x[1] + Ny * (x[2] + Nz * x[3]))

    want = np.zeros((vol, 4, 3, 3), dtype=complex)
    for y in range(vol):
        xy = [y % Nx, (y // Nx) % Ny, (y // (Nx * Ny)) % Nz, y // (Nx * Ny * Nz)]
        for d in product((-1, 0, 1), repeat=4):
            k = sum(abs(c) for c in d)
            if k == 0:
                continue
            M = rho[k] * sum(d[m] * G[m] for m in range(4)) - 0.5 * lam[k] * np.eye(4)
            chi = np.einsum("st,vtb->vsb", M, ps[site([(xy[m] + d[m]) % L[m] for m in range(4)])])
            Gd = np.einsum("vsa,vsb->ab", gs[y], chi.conj())
            for mu in range(4):
                if d[mu] == 0:
                    continue
                others = [m for m in range(4) if d[m] != 0 and m != mu]
                for r in range(len(others) + 1):
                    for sub in combinations(others, r):
                        w = factorial(r) * factorial(k - 1 - r) / factorial(k)
                        z = list(xy)
                        for m in sub:
                            z[m] = (z[m] + d[m]) % L[m]
                        if d[mu] > 0:
                            want[site(z), mu] += w * Gd
                        else:
                            z[mu] = (z[mu] - 1) % L[mu]
                            want[site(z), mu] += w * Gd.conj().T
    assert np.abs(F.reshape(vol, 4, 3, 3) - want).max() < 1e-12


def test_force_closed_forms():
    """Closed forms of the link gradient, derived from Sec. 3 / def_wils:
    staggered F_mu(x) = 1/2 eta_mu(x) sum_v [g_v(x) psi_v(x+mu)^+ - psi_v(x) g_v(x+mu)^+]
    Wilson    F_mu(x) = -1/2 sum_v,s [(1-g_mu) g_v(x)] psi_v(x+mu)^+ - 1/2 sum_v,s psi_v(x) [(1+g_mu) g_v(x+mu)]^+"""
    L = (2, 2, 3, 2)
    V = synth.gauge_links(L, 3, "haar", 132)
    Nx, Ny, Nz, Nt = L
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (Nt, Nz, Ny, Nx)], indexing="ij")
    coords = [x, y, z, t]
    psi = _psi(L, "staggered", 2, 133)
    g = _psi(L, "staggered", 2, 134)
    F = oracle.force("staggered", V, psi, g, 0.0)
    for mu in range(4):
        eta = (-1.0) ** sum(coords[:mu]) if mu else np.ones_like(x, dtype=float)
        pp = np.roll(psi, -1, axis=3 - mu)
        gp = np.roll(g, -1, axis=3 - mu)
        want = 0.5 * eta[..., None, None] * (np.einsum("...va,...vb->...ab", g, pp.conj())
                                             - np.einsum("...va,...vb->...ab", psi, gp.conj()))
        assert np.abs(F[..., mu, :, :] - want).max() < 1e-13
    psi = _psi(L, "wilson", 2, 135)
    g = _psi(L, "wilson", 2, 136)
    F = oracle.force("wilson", V, psi, g, 0.3)
    G = dense.gammas()
    for mu in range(4):
        pp = np.roll(psi, -1, axis=3 - mu)
        gp = np.roll(g, -1, axis=3 - mu)
        hm = g - np.einsum("st,...vta->...vsa", G[mu], g)
        hp = gp + np.einsum("st,...vta->...vsa", G[mu], gp)
        want = -0.5 * np.einsum("...vsa,...vsb->...ab", hm, pp.conj()) \
               - 0.5 * np.einsum("...vsa,...vsb->...ab", psi, hp.conj())
        assert np.abs(F[..., mu, :, :] - want).max() < 1e-13
