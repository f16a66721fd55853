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


@pytest.mark.parametrize("op,mass", [("wilson", 0.122), ("staggered", 0.08), ("staggered", -0.08)])
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_solve_even_odd_vs_whole_lattice(dg, op, mass, prec):
    """The even-odd inner solve (Schur complement of the odd sites: CGLS for
    Wilson, CG for staggered, including a negative staggered mass, where the
    Schur complement is negative definite) and the whole-lattice one both
    reach the oracle-checked FP64 residual 1e-10 and agree on x within the
    tolerance; with FP32 / FP64 inner arithmetic the even-odd one needs fewer
    sweeps."""
    L, Nv = (4, 4, 4, 8), 4
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", 330))
    b = synth.spinor(L, Nv, NS[op], 3, 331)
    D = dg.Dirac(op, L, Nv, mass, prec)
    D.set_links(torch.from_numpy(V.astype(np.complex64 if prec != "f64" else np.complex128)).cuda())
    assert D.preconditioner() == 1   # the default
    out = {}
    for precond in (1, 0):
        D.set_preconditioner(precond)
        x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=40, max_inner=3000)
        assert status == dg.OK, (precond, res, st)
        assert st["even_odd"] == precond
        x = x.cpu().numpy()
        true_res = oracle_residual(op, V, x, b, m0_of(op, mass))
        assert true_res.max() <= 1e-10, (precond, true_res)
        out[precond] = (x, st)
    D.close()
    x1, x0 = out[1][0], out[0][0]
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < 1e-7
    if prec in ("f32", "f64"):
        assert out[1][1]["sweeps"] < out[0][1]["sweeps"], (out[1][1], out[0][1])


@pytest.mark.parametrize("op,mass", [("wilson", 0.123), ("staggered", 0.06), ("brillouin", 0.07)])
def test_solve_residual_arithmetic(dg, op, mass):
    """The outer residual in double-float arithmetic (default of non-FP64
    handles) and in FP64 both certify the oracle-checked 1e-10, and the
    library's residuals match the oracle's at that level (so the
    double-float residual resolves far below 1e-10); a right-hand side
    outside FP32's exponent range falls back to FP64."""
    L, Nv = (4, 4, 2, 6), 2
    V = links_for("bf16", synth.gauge_links(L, 3, "near_identity", 340))
    b = synth.spinor(L, Nv, NS[op], 3, 341)
    D = dg.Dirac(op, L, Nv, mass, "bf16")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    assert D.residual_arithmetic() == 1   # the default of 16-bit handles
    m0 = m0_of(op, mass)
    for mode in (1, 0):
        D.set_residual_arithmetic(mode)
        x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=60, max_inner=3000)
        assert status == dg.OK, (mode, res, st)
        assert st["df_residual"] == mode
        true_res = oracle_residual(op, V, x.cpu().numpy(), b, m0)
        assert true_res.max() <= 1e-10, (mode, true_res)
        assert np.allclose(true_res, res, rtol=1e-3, atol=1e-14), (mode, true_res, res)
    D.set_residual_arithmetic(1)
    tiny = b * 1e-20   # mean square 1e-40: outside the double-float range
    x, res, st, status = D.solve(torch.from_numpy(tiny).cuda(), tol=1e-10, max_outer=60, max_inner=3000)
    assert status == dg.OK and st["df_residual"] == 0, st
    assert oracle_residual(op, V, x.cpu().numpy(), tiny, m0).max() <= 1e-10
    D.close()


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_solve_split_inner_fields(dg, prec):
    """Split inner fields for 16-bit Wilson handles (FP32 solution, residual,
    operator products and links; 16-bit search directions): single and
    batched solves certified by the oracle, and fewer refinement steps than
    with every inner field in 16 bits (the inner solve reaches FP32-level
    reductions)."""
    L, Nv = (4, 4, 4, 8), 4
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", 350))
    b = synth.spinor(L, Nv, 4, 3, 351)
    D = dg.Dirac("wilson", L, Nv, 0.1235, prec)
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    assert D.inner_fields() == 1   # the default
    m0 = oracle.kappa_to_m0(0.1235)
    outer = {}
    for mode in (1, 0):
        D.set_inner_fields(mode)
        x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=60, max_inner=3000)
        assert status == dg.OK, (mode, res, st)
        assert st["split_fields"] == mode and st["even_odd"] == 1
        true_res = oracle_residual("wilson", V, x.cpu().numpy(), b, m0)
        assert true_res.max() <= 1e-10, (mode, true_res)
        outer[mode] = st["outer_iterations"]
    D.close()
    assert outer[1] < outer[0], outer
    nv_list, kap = [1, 3, 2, 4, 1], [0.120, 0.1225, 0.124, 0.121, 0.1232]
    V, bs, xs, res, sys_stats, tot, status = _batched_case(dg, "wilson", (4, 4, 2, 4), nv_list, kap, prec, 4, 360,
                                                          inner_fields=1)
    assert status == dg.OK and tot["split_fields"] == 1, (sys_stats, tot)
    for bi, xi, k in zip(bs, xs, kap):
        assert oracle_residual("wilson", V, xi, bi, oracle.kappa_to_m0(k)).max() <= 1e-10


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_brillouin_split_inner_fields(dg, prec):
    """Split inner fields for 16-bit Brillouin handles (whole-lattice inner
    CGLS: FP32 W, solution, residual and products; 16-bit search
    directions): single and batched solves certified by the oracle, fewer
    refinement steps than with every inner field in 16 bits, and a new gauge
    field reaches the FP32 W copy of a handle whose solver graph is cached."""
    L, Nv = (4, 4, 2, 6), 3
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", 380))
    b = synth.spinor(L, Nv, 4, 3, 381)
    D = dg.Dirac("brillouin", L, Nv, 0.06, prec)
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    outer = {}
    for mode in (1, 0):
        D.set_inner_fields(mode)
        x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=60, max_inner=3000)
        assert status == dg.OK, (mode, res, st)
        assert st["split_fields"] == mode and st["even_odd"] == 0
        assert oracle_residual("brillouin", V, x.cpu().numpy(), b, 0.06).max() <= 1e-10, mode
        outer[mode] = st["outer_iterations"]
    assert outer[1] < outer[0], outer
    D.set_inner_fields(1)
    V2 = links_for(prec, synth.gauge_links(L, 3, "near_identity", 382))
    D.set_links(torch.from_numpy(V2.astype(np.complex64)).cuda())
    x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=60, max_inner=3000)
    assert status == dg.OK and st["split_fields"] == 1, (res, st)
    assert oracle_residual("brillouin", V2, x.cpu().numpy(), b, 0.06).max() <= 1e-10
    D.close()
    masses = [0.05, 0.1, 0.2, 0.07]
    V, bs, xs, res, sys_stats, tot, status = _batched_case(dg, "brillouin", (4, 4, 2, 4), [1, 3, 2, 2], masses, prec,
                                                          4, 383, inner_fields=1)
    assert status == dg.OK and tot["split_fields"] == 1, (sys_stats, tot)
    for bi, xi, m in zip(bs, xs, masses):
        assert oracle_residual("brillouin", V, xi, bi, m).max() <= 1e-10


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_solve_tensor_core_config(dg, prec):
    """Solves of a 16-bit Brillouin handle configured for the tensor-core
    sweep (launch variant 7): with split inner fields and with every inner
    field in 16 bits (whose whole-lattice inner sweeps are the tensor-core
    sweep, captured in the solver graph), then after new links (the
    site-major W copy the sweep reads is rebuilt in place), and a batched
    solve (per-column diagonal); all certified by the oracle."""
    L, Nv = (4, 4, 2, 6), 3
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", 390))
    b = synth.spinor(L, Nv, 4, 3, 391)
    D = dg.Dirac("brillouin", L, Nv, 0.06, prec)
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    D.set_kernel_config(1, 128, 7)
    assert D.link_format() == 1
    for mode in (1, 0):
        D.set_inner_fields(mode)
        x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=80, max_inner=3000)
        assert status == dg.OK, (mode, res, st)
        assert oracle_residual("brillouin", V, x.cpu().numpy(), b, 0.06).max() <= 1e-10, mode
    V2 = links_for(prec, synth.gauge_links(L, 3, "near_identity", 392))
    D.set_links(torch.from_numpy(V2.astype(np.complex64)).cuda())
    x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=80, max_inner=3000)
    assert status == dg.OK, (res, st)
    assert oracle_residual("brillouin", V2, x.cpu().numpy(), b, 0.06).max() <= 1e-10
    D.sync()
    D.close()
    masses = [0.05, 0.1, 0.2]
    V, bs, xs, res, sys_stats, tot, status = _batched_case(dg, "brillouin", (4, 4, 2, 4), [1, 3, 2], masses, prec,
                                                          4, 393, inner_fields=0, cfg=(1, 128, 7))
    assert status == dg.OK, (sys_stats, tot)
    for bi, xi, m in zip(bs, xs, masses):
        assert oracle_residual("brillouin", V, xi, bi, m).max() <= 1e-10


@pytest.mark.parametrize("op,masses", [("wilson", [0.120, 0.1225, 0.124]), ("brillouin", [0.05, 0.1, 0.2])])
@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_solve_link_format_1(dg, op, masses, prec):
    """Single and batched solves with link format 1 (Wilson two-row links in
    the whole-lattice inner sweeps, Brillouin 80 stored W), the per-column
    diagonal of the batched sweep included, certified by the oracle."""
    L = (4, 4, 2, 4)
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", 390))
    b = synth.spinor(L, 3, 4, 3, 391)
    D = dg.Dirac(op, L, 3, masses[0], prec)
    D.set_preconditioner(0)          # whole-lattice inner solves: the sweeps that read format 1
    D.set_kernel_config(2, 64, 1)
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    D.set_link_format(1)
    m0 = oracle.kappa_to_m0 if op == "wilson" else (lambda m: m)
    x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=60, max_inner=3000)
    assert status == dg.OK, (res, st)
    assert oracle_residual(op, V, x.cpu().numpy(), b, m0(masses[0])).max() <= 1e-10
    bs = [synth.spinor(L, nv, 4, 3, 392 + i) for i, nv in enumerate([2, 1, 3])]
    xs, res, sys_stats, tot, status = D.solve_batched([torch.from_numpy(bi).cuda() for bi in bs], masses,
                                                      tol=1e-10, max_outer=60, max_inner=3000)
    assert status == dg.OK, (sys_stats, tot)
    assert D.link_format() == 1
    for bi, xi, m in zip(bs, xs, masses):
        assert oracle_residual(op, V, xi.cpu().numpy(), bi, m0(m)).max() <= 1e-10
    D.close()


def test_solve_after_set_mass_and_set_links(dg):
    """A second solve on the same handle after dirac_set_mass, and after
    dirac_set_links with new links, solves the current operator: the captured
    inner-iteration graphs and the FP32 link copy of the split inner solve
    follow the change (Brillouin: whole-lattice inner solve; BF16 Wilson:
    even-odd with split fields)."""
    L, Nv = (4, 4, 2, 4), 2
    V = links_for("f32", synth.gauge_links(L, 3, "near_identity", 370))
    b = synth.spinor(L, Nv, 4, 3, 371)
    D = dg.Dirac("brillouin", L, Nv, 0.05, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    for m in (0.05, 0.2):
        D.set_mass(m)
        x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=40, max_inner=3000)
        assert status == dg.OK, (m, res, st)
        assert oracle_residual("brillouin", V, x.cpu().numpy(), b, m).max() <= 1e-10
    D.close()
    V2 = links_for("f32", synth.gauge_links(L, 3, "near_identity", 372))
    D = dg.Dirac("wilson", L, Nv, 0.122, "bf16")
    for VV in (V, V2):
        D.set_links(torch.from_numpy(VV.astype(np.complex64)).cuda())
        x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=40, max_inner=3000)
        assert status == dg.OK and st["split_fields"] == 1, (res, st)
        assert oracle_residual("wilson", VV, x.cpu().numpy(), b, oracle.kappa_to_m0(0.122)).max() <= 1e-10
    D.close()


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


def _batched_case(dg, op, L, nv_list, masses, prec, window, seed, tol=1e-10, precond=1, inner_fields=1, cfg=None):
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", seed))
    bs = [synth.spinor(L, nv, NS[op], 3, seed + 1 + i) for i, nv in enumerate(nv_list)]
    D = dg.Dirac(op, L, window, masses[0], prec)
    D.set_preconditioner(precond)
    D.set_inner_fields(inner_fields)
    D.set_links(torch.from_numpy(V.astype(np.complex64 if prec != "f64" else np.complex128)).cuda())
    if cfg:
        D.set_kernel_config(*cfg)
    xs, res, sys_stats, tot, status = D.solve_batched([torch.from_numpy(b).cuda() for b in bs], masses, tol=tol,
                                                      max_outer=40, max_inner=4000)
    D.close()
    return V, bs, [x.cpu().numpy() for x in xs], res, sys_stats, tot, status


@pytest.mark.parametrize("op,masses", [("wilson", [0.120, 0.1225, 0.124, 0.121, 0.1232]),
                                       ("staggered", [0.05, 0.11, 0.2, 0.08, 0.3]),
                                       ("brillouin", [0.05, 0.1, 0.2, 0.07, 0.3])])
@pytest.mark.parametrize("prec", ["bf16", "f32"])
@pytest.mark.parametrize("precond", [1, 0])
def test_solve_batched_queue(dg, op, masses, prec, precond):
    """Five systems with uneven Nv and masses through a window of 4 slots
    (columns are admitted and retired while others are still iterating);
    every column's true FP64 residual, re-evaluated by the oracle, is <= 1e-10.
    Both inner solvers: even-odd (Wilson, staggered) and whole lattice."""
    L = (4, 4, 2, 4)
    nv_list = [1, 3, 2, 4, 1]
    V, bs, xs, res, sys_stats, tot, status = _batched_case(dg, op, L, nv_list, masses, prec, 4, 400,
                                                          precond=precond)
    assert status == dg.OK, (sys_stats, tot)
    assert tot["even_odd"] == (1 if precond and op != "brillouin" else 0)
    k = 0
    for i, (b, x, m) in enumerate(zip(bs, xs, masses)):
        true_res = oracle_residual(op, V, x, b, m0_of(op, m))
        assert true_res.max() <= 1e-10, (i, true_res)
        assert np.allclose(true_res, res[k:k + nv_list[i]], rtol=1e-3, atol=1e-13)
        assert sys_stats[i]["converged"] == 1
        k += nv_list[i]


@pytest.mark.parametrize("op,mass", [("wilson", 0.121), ("staggered", 0.1), ("brillouin", 0.08)])
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_solve_ragged_volume(dg, op, mass, prec):
    """A volume that is not a multiple of 32 (3 x 4 x 2 x 5 = 120 sites): the
    last block of the internal layout has 8 padding sites, which the solver's
    vector kernels must see as zeros.  Single and batched solves."""
    L = (3, 4, 2, 5)
    V = links_for(prec, synth.gauge_links(L, 3, "near_identity", 410))
    b = synth.spinor(L, 3, NS[op], 3, 411)
    D = dg.Dirac(op, L, 3, mass, prec)
    D.set_links(torch.from_numpy(V.astype(np.complex64 if prec != "f64" else np.complex128)).cuda())
    x, res, st, status = D.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_outer=40, max_inner=3000)
    D.close()
    assert status == dg.OK, (res, st)
    assert st["even_odd"] == 0   # odd extents: the whole-lattice inner solve
    true_res = oracle_residual(op, V, x.cpu().numpy(), b, m0_of(op, mass))
    assert true_res.max() <= 1e-10, true_res
    V, bs, xs, res, sys_stats, tot, status = _batched_case(dg, op, L, [2, 1, 3], [mass, mass * 1.01, mass * 0.99],
                                                          prec, 4, 412)
    assert status == dg.OK, (sys_stats, tot)
    assert tot["even_odd"] == 0
    for b, x, m in zip(bs, xs, [mass, mass * 1.01, mass * 0.99]):
        assert oracle_residual(op, V, x, b, m0_of(op, m)).max() <= 1e-10


def test_solve_batched_matches_single(dg):
    """A batch of one system equals dirac_solve on it (same iterates up to the
    tolerance)."""
    L = (4, 4, 4, 2)
    V = links_for("f32", synth.gauge_links(L, 3, "near_identity", 410))
    b = synth.spinor(L, 3, 4, 3, 411)
    D = dg.Dirac("wilson", L, 3, 0.122, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    x1, r1, st1, s1 = D.solve(torch.from_numpy(b).cuda())
    xs, rb, sys_stats, tot, sb = D.solve_batched([torch.from_numpy(b).cuda()], [0.122])
    D.close()
    assert s1 == dg.OK and sb == dg.OK
    x1 = x1.cpu().numpy()
    xb = xs[0].cpu().numpy()
    assert np.linalg.norm(x1 - xb) / np.linalg.norm(x1) < 1e-8


def test_solve_batched_c5_shape_reduced(dg):
    """The batched configuration's shape at a reduced volume: 48 Wilson
    systems, Nv drawn uniformly from 1..24, kappa uniform in [0.120, 0.124],
    BF16 storage, FP64 refinement to 1e-10, on 8^3 x 16 with 96 resident
    slots.  The residuals of two sampled columns per system are re-evaluated
    by the oracle."""
    L = (8, 8, 8, 16)
    rng = synth.rng(1005, synth.STREAM_MISC)
    nv_list = [int(v) for v in rng.integers(1, 25, 48)]
    kappas = [float(k) for k in rng.uniform(0.120, 0.124, 48)]
    V, bs, xs, res, sys_stats, tot, status = _batched_case(dg, "wilson", L, nv_list, kappas, "bf16", 96, 1005)
    assert status == dg.OK, tot
    assert res.max() <= 1e-10
    for i in range(0, 48, 6):
        cols = sorted({0, nv_list[i] - 1})
        r = oracle_residual("wilson", V, xs[i][..., cols, :, :], bs[i][..., cols, :, :], oracle.kappa_to_m0(kappas[i]))
        assert r.max() <= 1e-10, (i, r)


def test_solve_batched_c5_one_wave(dg):
    """The batched configuration at its full size -- 32^3 x 64, BF16 storage
    with the library's defaults (even-odd inner solves, split inner fields),
    64 resident slots, one shared gauge field -- for one wave of its systems:
    the first systems of the 48-system draw, up to 96 columns (the waves the
    benchmark feeds), with complex Gaussian sources drawn on the device.
    Every column's FP64 residual from the library is <= 1e-10, and two
    columns per system are re-evaluated by the oracle."""
    L = (32, 32, 32, 64)
    Nx, Ny, Nz, Nt = L
    rng = synth.rng(1005, synth.STREAM_MISC)
    nv_list = [int(v) for v in rng.integers(1, 25, 48)]
    kappas = [float(k) for k in rng.uniform(0.120, 0.124, 48)]
    wave, cols = [], 0
    for i in range(48):
        if cols + nv_list[i] > 96:
            break
        wave.append(i)
        cols += nv_list[i]
    V = synth.round_to(synth.gauge_links(L, 3, "near_identity", 1005), "f32")
    D = dg.Dirac("wilson", L, 64, kappas[0], "bf16")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    bs = []
    for j in wave:
        g = torch.Generator(device="cuda")
        g.manual_seed(2005 + j)
        z = torch.randn((Nt, Nz, Ny, Nx, nv_list[j], 4, 3, 2), dtype=torch.float64, device="cuda", generator=g)
        bs.append(torch.view_as_complex(z.mul_(0.5 ** 0.5)))
    xs, res, sys_stats, tot, status = D.solve_batched(bs, [kappas[j] for j in wave], tol=1e-10, max_outer=60,
                                                      max_inner=8000)
    D.close()
    assert status == dg.OK, tot
    assert len(res) == cols and res.max() <= 1e-10
    assert tot["even_odd"] == 1 and tot["split_fields"] == 1
    for j, b, x in zip(wave, bs, xs):
        cj = sorted({0, nv_list[j] - 1})
        r = oracle_residual("wilson", V, x[..., cj, :, :].cpu().numpy(), b[..., cj, :, :].cpu().numpy(),
                            oracle.kappa_to_m0(kappas[j]))
        assert r.max() <= 1e-10, (j, r)
    del bs, xs
    torch.cuda.empty_cache()


@pytest.mark.skipif(not __import__("os").environ.get("DIRAC_FULL_BATCHED"),
                    reason="full-size batched configuration (several GPU-minutes): set DIRAC_FULL_BATCHED=1")
def test_solve_batched_c5_full(dg):
    """48 Wilson systems on 32^3 x 64, Nv ~ U{1..24}, kappa ~ U[0.120, 0.124],
    BF16 storage, FP32 arithmetic, FP64 refinement to 1e-10, shared links.
    The canonical FP64 b and x of all 48 systems (about 600 columns of 403 MB)
    do not fit one GPU at once, so the systems go through dirac_solve_batched
    in waves that fill the handle's slots; every column's FP64 residual comes
    from the library, and two sampled columns per system are re-evaluated by
    the oracle."""
    import time
    L = (32, 32, 32, 64)
    rng = synth.rng(1005, synth.STREAM_MISC)
    nv_list = [int(v) for v in rng.integers(1, 25, 48)]
    kappas = [float(k) for k in rng.uniform(0.120, 0.124, 48)]
    V = synth.round_to(synth.gauge_links(L, 3, "near_identity", 1005), "f32")
    # 64 resident slots (solver: 3 FP64 + 5 BF16 fields of 64 columns, ~110 GB)
    # and waves of at most 96 columns (their FP64 b and x, ~77 GB)
    D = dg.Dirac("wilson", L, 64, kappas[0], "bf16")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    D.autotune()
    t0 = time.perf_counter()
    i, total_cols, worst = 0, 0, 0.0
    while i < 48:
        wave = []
        cols = 0
        while i < 48 and cols + nv_list[i] <= 96:
            wave.append(i)
            cols += nv_list[i]
            i += 1
        bs = [torch.from_numpy(synth.spinor(L, nv_list[j], 4, 3, 2005 + j)).cuda() for j in wave]
        xs, res, sys_stats, tot, status = D.solve_batched(bs, [kappas[j] for j in wave], tol=1e-10,
                                                          max_outer=60, max_inner=8000)
        assert status == dg.OK, (wave, tot)
        worst = max(worst, float(res.max()))
        for j, b, x in zip(wave, bs, xs):
            cols_j = sorted({0, nv_list[j] - 1})
            xc = x[..., cols_j, :, :].cpu().numpy()
            bc = b[..., cols_j, :, :].cpu().numpy()
            r = oracle_residual("wilson", V, xc, bc, oracle.kappa_to_m0(kappas[j]))
            assert r.max() <= 1e-10, (j, r)
        total_cols += cols
        del bs, xs
        torch.cuda.empty_cache()
    D.close()
    print(f"batched full: {total_cols} columns, worst residual {worst:.3e}, {time.perf_counter() - t0:.1f} s")
