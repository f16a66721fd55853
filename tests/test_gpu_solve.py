"""GPU defect-correction solves (dirac_solve) checked by the FP64 oracle.

Several x are correct only up to the tolerance, so what is compared is what
is unique: the true FP64 relative residual |b - D x| / |b| re-evaluated by
the oracle must be <= 1e-10 for every right-hand side, and on small lattices
x must agree with the dense LU solution within cond(D) * 1e-10.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS = {"staggered": 1, "wilson": 4, "brillouin": 4}


@pytest.fixture(scope="module")
def dg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1808_05506_gb300 as dg
    torch.cuda.set_device(0)
    return dg


def m0_of(op, mass):
    return oracle.kappa_to_m0(mass) if op == "wilson" else mass


def oracle_residual(op, V, x, b, m0):
    r = b - oracle.apply(op, V, x, m0)
    ax = tuple(i for i in range(r.ndim) if i != 4)
    return np.sqrt(np.sum(np.abs(r) ** 2, axis=ax) / np.sum(np.abs(b) ** 2, axis=ax))


def links_for(prec, V):
    # the handle keeps the links it was given in FP64 for the outer residual;
    # FP32 input is the common case for mixed-precision handles
    return synth.round_to(V, "f32") if prec != "f64" else V


@pytest.mark.parametrize("op,mass", [("wilson", 0.12), ("staggered", 0.1), ("brillouin", 0.05)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_solve_small_vs_dense_lu(dg, op, mass, prec):
    L, Nv = (4, 4, 2, 4), 3
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", 300))
    b = synth.spinor(L, Nv, NS[op], 3, 301)
    D = dg.Dirac(op, L, Nv, mass, prec)
    D.set_links(torch.from_numpy(V.astype(np.complex64 if prec != "f64" else np.complex128)).cuda())
    x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=40, max_inner=3000)
    D.close()
    assert status == dg.OK, (res, st)
    x = x.cpu().numpy()
    m0 = m0_of(op, mass)
    true_res = oracle_residual(op, V, x, b, m0)
    assert true_res.max() <= 1e-10, true_res
    assert np.allclose(true_res, res, rtol=1e-3, atol=1e-13)     # the library's own FP64 residual
    Dm = dense.dense(op, V, m0)
    vol = int(np.prod(L))
    bm = b.reshape(vol, Nv, -1).transpose(1, 0, 2).reshape(Nv, -1)   # [v, (site, spin, colour)]
    xg = x.reshape(vol, Nv, -1).transpose(1, 0, 2).reshape(Nv, -1)
    xl = np.linalg.solve(Dm, bm.T).T
    cond = np.linalg.cond(Dm)
    assert np.linalg.norm(xg - xl) / np.linalg.norm(xl) <= cond * 1e-10


def test_solve_resume_and_zero_rhs(dg):
    """x0 = the solution: no refinement step is taken; a zero right-hand side
    converges at once; the result does not depend on the other columns."""
    L, Nv = (4, 2, 4, 4), 2
    V = links_for("f32", synth.gauge_links(L, 3, "near_identity", 310))
    b = synth.spinor(L, Nv, 4, 3, 311)
    b[..., 1, :, :] = 0
    D = dg.Dirac("wilson", L, Nv, 0.124, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    bt = torch.from_numpy(b).cuda()
    x, res, st, status = D.solve(bt, tol=1e-10)
    assert status == dg.OK and res.max() <= 1e-10
    assert np.abs(x.cpu().numpy()[..., 1, :, :]).max() == 0.0
    x2, res2, st2, status2 = D.solve(bt, x0=x, tol=1e-10)
    assert status2 == dg.OK and st2["outer_iterations"] == 0
    D.close()


def test_solve_not_converged_status(dg):
    L, Nv = (4, 4, 4, 4), 1
    V = links_for("f32", synth.gauge_links(L, 3, "near_identity", 320))
    b = synth.spinor(L, Nv, 4, 3, 321)
    D = dg.Dirac("wilson", L, Nv, 0.124, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=1, max_inner=3)
    assert status == dg.NOT_CONVERGED and res.max() > 1e-10
    assert st["outer_iterations"] == 1 and st["inner_iterations"] == 3
    with pytest.raises(dg.DiracError):
        D.solve(torch.from_numpy(b).cuda(), tol=-1.0)
    D.close()
