"""Backward pass of out = D(V) psi: dL/dpsi = D^+ g and the link force,
checked against the FP64 oracle's gradient (term by term; for Brillouin
through the path products of W), against FP64 central finite differences of
the GPU forward pass (L = Re <g, D psi> is linear in V for staggered and
Wilson, so the difference quotient is exact up to rounding; a polynomial of
degree 4 for Brillouin), and by torch.autograd.gradcheck."""
import numpy as np
import pytest

import oracle
import synth

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


@pytest.mark.parametrize("op,mass", [("wilson", 0.125), ("staggered", 0.03)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_force_vs_oracle_16x4(dg, op, mass, prec, tol):
    """16^4, Nv = 8 (the differentiable configuration)."""
    L, Nv = (16, 16, 16, 16), 8
    rin = "f64" if prec == "f64" else "f32"
    V = synth.round_to(synth.gauge_links(L, 3, "near_identity", 1004), rin)
    psi = synth.round_to(synth.spinor(L, Nv, NS[op], 3, 2004), rin)
    g = synth.round_to(synth.spinor(L, Nv, NS[op], 3, 3004), rin)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    D = dg.Dirac(op, L, Nv, mass, prec)
    D.set_links(torch.from_numpy(V).to(cdt).cuda())
    F = D.force(torch.from_numpy(psi).to(cdt).cuda(), torch.from_numpy(g).to(cdt).cuda()).cpu().numpy()
    D.close()
    want = oracle.force(op, V, psi, g, m0_of(op, mass))
    err = np.linalg.norm(F - want) / np.linalg.norm(want)
    assert err <= tol, err


@pytest.mark.parametrize("op,mass", [("wilson", 0.121), ("staggered", 0.2)])
def test_force_finite_differences(dg, op, mass):
    """FP64 central differences, eps = 1e-6, on 64 random link directions."""
    L, Nv = (16, 16, 16, 16), 8
    V = synth.gauge_links(L, 3, "near_identity", 1004)
    psi = synth.spinor(L, Nv, NS[op], 3, 2004)
    g = synth.spinor(L, Nv, NS[op], 3, 3004)
    D = dg.Dirac(op, L, Nv, mass, "f64")
    Vt = torch.from_numpy(V).cuda()
    pt = torch.from_numpy(psi).cuda()
    gt = torch.from_numpy(g).cuda()
    D.set_links(Vt)
    F = D.force(pt, gt).cpu().numpy()
    rng = synth.rng(1005, synth.STREAM_MISC)
    eps = 1e-6

    def loss(Vx):
        D.set_links(Vx)
        return torch.vdot(gt.reshape(-1), D.apply(pt).reshape(-1)).real.item()

    for _ in range(64):
        idx = tuple(int(rng.integers(0, n)) for n in V.shape[:5])
        dV = synth.complex_gaussian((3, 3), int(rng.integers(1 << 30)))
        Vp = Vt.clone()
        Vm = Vt.clone()
        Vp[idx] += eps * torch.from_numpy(dV).cuda()
        Vm[idx] -= eps * torch.from_numpy(dV).cuda()
        fd = (loss(Vp) - loss(Vm)) / (2 * eps)
        an = np.vdot(F[idx], dV).real
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-6, (fd, an)
    D.close()


@pytest.mark.parametrize("op,mass", [("wilson", 0.13), ("staggered", 0.1)])
def test_autograd_function(dg, op, mass):
    from paper_1808_05506_gb300.autograd import dirac_apply
    L, Nv = (4, 2, 2, 4), 2
    V = torch.from_numpy(synth.gauge_links(L, 3, "haar", 1006)).cuda().requires_grad_(True)
    psi = torch.from_numpy(synth.spinor(L, Nv, NS[op], 3, 2006)).cuda().requires_grad_(True)
    D = dg.Dirac(op, L, Nv, mass, "f64")
    # gradcheck: Jacobian of the differentiable apply by finite differences vs our backward
    assert torch.autograd.gradcheck(lambda p, v: dirac_apply(D, p, v, reuse_links=False), (psi, V), eps=1e-6, atol=1e-7,
                                    rtol=1e-6, fast_mode=True)
    g = torch.from_numpy(synth.spinor(L, Nv, NS[op], 3, 3006)).cuda()
    out = dirac_apply(D, psi, V)
    loss = torch.vdot(g.reshape(-1), out.reshape(-1)).real
    loss.backward()
    Vn, pn, gn = V.detach().cpu().numpy(), psi.detach().cpu().numpy(), g.cpu().numpy()
    m0 = m0_of(op, mass)
    want_psi = oracle.apply(op, Vn, gn, m0, dagger=True)
    want_V = oracle.force(op, Vn, pn, gn, m0)
    assert np.linalg.norm(psi.grad.cpu().numpy() - want_psi) / np.linalg.norm(want_psi) < 1e-13
    assert np.linalg.norm(V.grad.cpu().numpy() - want_V) / np.linalg.norm(want_V) < 1e-13
    D.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
@pytest.mark.parametrize("L", [(4, 4, 2, 6), (6, 6, 4, 4), (2, 3, 2, 4)])
def test_brillouin_force_vs_oracle(dg, prec, tol, L):
    """The Brillouin link gradient through the rebuilt transporters against the
    oracle's path enumeration; extent 2 makes paths reuse links.  Every step
    of the GPU gradient runs in FP64 (the FP32 inputs are exact there), so
    the FP32 result differs from the oracle's by its final rounding."""
    Nv = 3
    rin = "f64" if prec == "f64" else "f32"
    V = synth.round_to(synth.gauge_links(L, 3, "haar", 1010), rin)
    psi = synth.round_to(synth.spinor(L, Nv, 4, 3, 2010), rin)
    g = synth.round_to(synth.spinor(L, Nv, 4, 3, 3010), rin)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    D = dg.Dirac("brillouin", L, Nv, 0.05, prec)
    D.set_links(torch.from_numpy(V).to(cdt).cuda())
    F = D.force(torch.from_numpy(psi).to(cdt).cuda(), torch.from_numpy(g).to(cdt).cuda()).cpu().numpy()
    D.close()
    want = oracle.force("brillouin", V, psi, g, 0.05)
    err = np.linalg.norm(F - want) / np.linalg.norm(want)
    assert err <= tol, err


def test_brillouin_force_finite_differences(dg):
    """FP64 central differences of the GPU forward pass (W rebuilt by
    dirac_set_links each time), eps = 1e-5, 24 random link directions, 8^4,
    near-identity links."""
    L, Nv = (8, 8, 8, 8), 4
    V = synth.gauge_links(L, 3, "near_identity", 1011)
    psi = synth.spinor(L, Nv, 4, 3, 2011)
    g = synth.spinor(L, Nv, 4, 3, 3011)
    D = dg.Dirac("brillouin", L, Nv, 0.05, "f64")
    Vt = torch.from_numpy(V).cuda()
    pt = torch.from_numpy(psi).cuda()
    gt = torch.from_numpy(g).cuda()
    D.set_links(Vt)
    F = D.force(pt, gt).cpu().numpy()
    rng = synth.rng(1012, synth.STREAM_MISC)
    eps = 1e-5

    def loss(Vx):
        D.set_links(Vx)
        return torch.vdot(gt.reshape(-1), D.apply(pt).reshape(-1)).real.item()

    for _ in range(24):
        idx = tuple(int(rng.integers(0, n)) for n in V.shape[:5])
        dV = synth.complex_gaussian((3, 3), int(rng.integers(1 << 30)))
        Vp = Vt.clone()
        Vm = Vt.clone()
        Vp[idx] += eps * torch.from_numpy(dV).cuda()
        Vm[idx] -= eps * torch.from_numpy(dV).cuda()
        fd = (loss(Vp) - loss(Vm)) / (2 * eps)
        an = np.vdot(F[idx], dV).real
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-6, (fd, an)
    D.close()


def test_brillouin_autograd_function(dg):
    from paper_1808_05506_gb300.autograd import dirac_apply
    L, Nv = (2, 2, 2, 4), 1
    V = torch.from_numpy(synth.gauge_links(L, 3, "haar", 1013)).cuda().requires_grad_(True)
    psi = torch.from_numpy(synth.spinor(L, Nv, 4, 3, 2013)).cuda().requires_grad_(True)
    D = dg.Dirac("brillouin", L, Nv, 0.1, "f64")
    assert torch.autograd.gradcheck(lambda p, v: dirac_apply(D, p, v, reuse_links=False), (psi, V), eps=1e-6, atol=1e-7,
                                    rtol=1e-6, fast_mode=True)
    g = torch.from_numpy(synth.spinor(L, Nv, 4, 3, 3013)).cuda()
    out = dirac_apply(D, psi, V)
    torch.vdot(g.reshape(-1), out.reshape(-1)).real.backward()
    Vn, pn, gn = V.detach().cpu().numpy(), psi.detach().cpu().numpy(), g.cpu().numpy()
    want_V = oracle.force("brillouin", Vn, pn, gn, 0.1)
    assert np.linalg.norm(V.grad.cpu().numpy() - want_V) / np.linalg.norm(want_V) < 1e-12
    D.close()
