"""The decomposition the tensor-core Brillouin sweep (launch variant 7) computes,
restated in numpy and checked against the oracle on the CPU (no GPU).

Sec. 5, Eqs. def_bril, def_der, def_lap at c_SW = 0: the colour and spin
factors of each term commute, so with the five coefficient classes
C_0(d) = -lambda_k / 2 and C_{1+mu}(d) = rho_k d_mu (k = |d|_1),
    T_j = sum_{d != 0} C_j(d) W_d(x) psi(x + d),
    D_B psi = (m0 + 15/8) psi + T_0 + sum_mu gamma_mu T_{1+mu},
and D_B^+ negates the rho classes.  The sweep applies gamma_mu through fixed
couplings (spin s takes T_1, T_2 from spin 3 - s and T_3, T_4 from spin s ^ 2
with factors -i/+i, -1/+1, -i/+i, +1), and forms each complex product from
real ones with the B pairs (Y_re, -Y_im) and (Y_im, Y_re).  These tests pin
all three against the oracle's own D_B, D_B^+ and gamma matrices."""
import itertools

import numpy as np

import oracle
import synth

RHO = [0.0, 64.0 / 432.0, 16.0 / 432.0, 4.0 / 432.0, 1.0 / 432.0]
LAM = [-240.0 / 64.0, 8.0 / 64.0, 4.0 / 64.0, 2.0 / 64.0, 1.0 / 64.0]


def couplings(sp):
    """(partner spin, factor) of gamma_1 .. gamma_4 for output spin sp, as the
    sweep's epilogue applies them."""
    s1 = -1.0 if sp < 2 else 1.0
    s2 = -1.0 if sp in (0, 3) else 1.0
    return [(3 - sp, s1 * 1j), (3 - sp, s2), (sp ^ 2, s2 * 1j), (sp ^ 2, 1.0)]


def decomposed_apply(V, psi, m0, dagger=False):
    W = oracle.brillouin_W(V)                       # [t, z, y, x, 81, 3, 3]
    T = np.zeros((5,) + psi.shape, dtype=np.complex128)
    for d in itertools.product((-1, 0, 1), repeat=4):     # d = (dx, dy, dz, dt)
        k = sum(1 for e in d if e)
        if k == 0:
            continue
        code = sum((e + 1) * 3 ** mu for mu, e in enumerate(d))
        shifted = np.roll(psi, shift=(-d[3], -d[2], -d[1], -d[0]), axis=(0, 1, 2, 3))
        wpsi = np.einsum("tzyxab,tzyxvsb->tzyxvsa", W[..., code, :, :], shifted)
        sg = -1.0 if dagger else 1.0
        T[0] += (-0.5 * LAM[k]) * wpsi
        for mu in range(4):
            if d[mu]:
                T[1 + mu] += sg * RHO[k] * d[mu] * wpsi
    out = (m0 + 15.0 / 8.0) * psi + T[0]
    for sp in range(4):
        for mu, (src, f) in enumerate(couplings(sp)):
            out[..., sp, :] += f * T[1 + mu][..., src, :]
    return out


def test_couplings_are_the_oracle_gamma_matrices():
    for mu in range(4):
        g = oracle.gamma(mu)
        for sp in range(4):
            src, f = couplings(sp)[mu]
            row = np.zeros(4, dtype=np.complex128)
            row[src] = f
            assert np.array_equal(g[sp], row), (mu, sp, g[sp])


def test_decomposition_equals_the_oracle():
    for L, Nv, seed in (((3, 4, 2, 3), 2, 700), ((4, 3, 3, 2), 3, 710)):
        V = synth.gauge_links(L, 3, "haar", seed)
        psi = synth.spinor(L, Nv, 4, 3, seed + 1)
        for dagger in (False, True):
            want = oracle.apply("brillouin", V, psi, 0.07, dagger=dagger)
            got = decomposed_apply(V, psi, 0.07, dagger=dagger)
            err = np.max(np.abs(got - want)) / np.max(np.abs(want))
            assert err < 1e-12, (L, dagger, err)


def test_real_form_of_the_products():
    """The B columns for (re) and (im): pairs (Y_re, -Y_im) and (Y_im, Y_re)
    against the A pairs (X_re, X_im) give Re(X Y) and Im(X Y)."""
    rng = np.random.default_rng(720)
    X = rng.normal(size=(64, 40)) + 1j * rng.normal(size=(64, 40))
    Y = rng.normal(size=(40, 30)) + 1j * rng.normal(size=(40, 30))
    A = np.stack([X.real, X.imag], axis=2).reshape(64, 80)
    B = np.zeros((80, 60))
    B[0::2, 0::2], B[1::2, 0::2] = Y.real, -Y.imag
    B[0::2, 1::2], B[1::2, 1::2] = Y.imag, Y.real
    D = A @ B
    assert np.allclose(D[:, 0::2] + 1j * D[:, 1::2], X @ Y, rtol=0, atol=1e-12)
