"""GPU parity of the Dirac sweeps against the FP64 oracle, through the C ABI.

Bar: relative L2 error per right-hand side, the maximum over the
right-hand sides, <= 1e-6 in FP32 and <= 1e-13 in FP64, the oracle run on the same rounded
inputs the GPU saw.  BF16/FP16 storage has no apply parity target; the sweep
is checked against its own rounding bound (a few units of the storage
precision's epsilon).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "bf16": 3e-2, "f16": 4e-3}
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


def inputs(op, L, Nv, prec, seed, kind="haar"):
    V = synth.gauge_links(L, 3, kind, seed)
    psi = synth.spinor(L, Nv, NS[op], 3, seed + 1)
    rin = "f64" if prec == "f64" else "f32"
    V = synth.round_to(V, rin)
    psi = synth.round_to(psi, rin)
    return V, psi


def rel_l2(got, want, rhs_axis=4):
    """max over right-hand sides v of |got_v - want_v|_2 / |want_v|_2 (the
    parity metric per right-hand side; rhs_axis is v's axis: 4 for canonical
    fields (Nt, Nz, Ny, Nx, Nv, ...), 1 for sampled sites (n, Nv, ...))."""
    n = got.shape[rhs_axis]
    d = np.moveaxis(got - want, rhs_axis, 0).reshape(n, -1)
    w = np.moveaxis(want, rhs_axis, 0).reshape(n, -1)
    return float(np.max(np.linalg.norm(d, axis=1) / np.linalg.norm(w, axis=1)))


def run(dg, op, L, Nv, mass, prec, V, psi, dagger=False, cfg=None, internal=False):
    D = dg.Dirac(op, L, Nv, mass, prec)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    D.set_links(torch.from_numpy(V.astype(np.complex128 if prec == "f64" else np.complex64)).cuda())
    if cfg:
        D.set_kernel_config(*cfg)
    x = torch.from_numpy(psi).to(cdt).cuda()
    if internal:
        xi = D.pack(x)
        yi = D.new_internal()
        yi.fill_(0xFF)                      # NaN pattern: every element must be overwritten
        D.apply(xi, out=yi, dagger=dagger)
        D.sync()                                # kernel-side timeouts surface here
        y = D.unpack(yi)
    else:
        y = D.apply(x, dagger=dagger)
    D.sync()
    D.close()
    return y.cpu().numpy().astype(np.complex128)


def rounded_for_oracle(V, psi, prec):
    if prec in ("bf16", "f16"):
        return synth.round_to(V, prec), synth.round_to(psi, prec)
    return V, psi


@pytest.mark.parametrize("op,mass", [("wilson", 0.1237), ("staggered", 0.031), ("brillouin", 0.05)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dagger", [False, True])
def test_parity_ragged(dg, op, mass, prec, dagger):
    """Several blocks plus a ragged tail (vol = 720 is not a multiple of any
    block size) and an Nv that leaves a partial right-hand-side group."""
    L, Nv = (6, 4, 6, 5), 5
    V, psi = inputs(op, L, Nv, prec, 200)
    got = run(dg, op, L, Nv, mass, prec, V, psi, dagger=dagger)
    want = oracle.apply(op, V, psi, m0_of(op, mass), dagger=dagger)
    assert rel_l2(got, want) <= TOL[prec]


@pytest.mark.parametrize("op,mass", [("wilson", 0.125), ("staggered", 0.0), ("brillouin", 0.3)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_parity_every_config(dg, op, mass, prec):
    L, Nv = (4, 6, 2, 4), 7
    V, psi = inputs(op, L, Nv, prec, 210)
    want = oracle.apply(op, V, psi, m0_of(op, mass))
    Rs = (1, 2, 4, 6) if op == "staggered" else (1, 2, 3, 4)
    for R in Rs:
        for block in (32, 64, 128, 256):
            for variant in dg.VARIANTS[op]:
                if not dg.config_supported(op, prec, R, block, variant, L):
                    continue
                got = run(dg, op, L, Nv, mass, prec, V, psi, cfg=(R, block, variant), internal=True)
                assert rel_l2(got, want) <= TOL[prec], (R, block, variant)


@pytest.mark.parametrize("op,mass", [("wilson", 0.11), ("staggered", 0.2), ("brillouin", -0.1)])
@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_low_precision_storage(dg, op, mass, prec):
    L, Nv = (4, 4, 4, 4), 4
    V, psi = inputs(op, L, Nv, prec, 220, kind="near_identity")
    got = run(dg, op, L, Nv, mass, prec, V, psi)
    Vr, pr = rounded_for_oracle(V, psi, prec)
    if op == "brillouin":
        # W is built in FP64 from the FP32 links and rounded once to the storage type
        pr = synth.round_to(psi, prec)
        want = oracle.apply(op, V, pr, m0_of(op, mass))
    else:
        want = oracle.apply(op, Vr, pr, m0_of(op, mass))
    assert rel_l2(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_wilson_xrow_shapes(dg, prec):
    """The warp-per-x-rows variant (x hops by lane exchange, t hops carried):
    rows of 32, 16, 8 and 4 sites (one to eight rows per warp), t-extents
    that leave a partial t-chunk, and Nv that leaves a partial group."""
    for L, Nv in (((32, 2, 2, 3), 3), ((16, 2, 3, 5), 5), ((8, 4, 2, 10), 4), ((4, 4, 2, 3), 2)):
        V, psi = inputs("wilson", L, Nv, "f32", 270)
        Vr, pr = rounded_for_oracle(V, psi, prec)
        for dagger in (False, True):
            want = oracle.apply("wilson", Vr, pr, oracle.kappa_to_m0(0.121), dagger=dagger)
            for R in (1, 2):
                for block in (32, 96, 192):
                    assert dg.config_supported("wilson", prec, R, block, 5, L)
                    got = run(dg, "wilson", L, Nv, 0.121, prec, V, psi, dagger=dagger, cfg=(R, block, 5),
                              internal=True)
                    assert rel_l2(got, want) <= TOL[prec], (L, Nv, R, block, dagger)


@pytest.mark.parametrize("op,mass", [("wilson", 0.121), ("staggered", 0.07)])
@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_xlast_shapes(dg, op, mass, prec):
    """Variant 6 (x hops last, by lane exchange of the site's own spinor):
    rows of 32, 16, 8 and 4 sites (one to eight rows per warp, rows of one
    warp in different planes when Lx Ly is not a multiple of 32), Nv that
    leaves a partial group, both link formats, D and D^+."""
    Rs = (1, 2) if op == "wilson" else (1, 2, 4)
    for L, Nv in (((32, 2, 2, 3), 3), ((16, 2, 3, 5), 5), ((8, 2, 2, 10), 4), ((4, 4, 2, 3), 2)):
        V, psi = inputs(op, L, Nv, "f32", 275)
        Vr, pr = rounded_for_oracle(V, psi, prec)
        D = dg.Dirac(op, L, Nv, mass, prec)
        D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
        xi = D.pack(torch.from_numpy(psi.astype(np.complex64)).cuda())
        for dag in (False, True):
            want = oracle.apply(op, Vr, pr, m0_of(op, mass), dagger=dag)
            for fmt in (0, 1):
                D.set_link_format(fmt)
                for R in Rs:
                    for block in (32, 64):
                        assert dg.config_supported(op, prec, R, block, 6, L)
                        for tc in (0, 2):
                            D.set_kernel_config(R, block, 6)
                            D.set_site_order(tc)
                            yi = D.new_internal()
                            yi.fill_(0xFF)
                            D.apply(xi, out=yi, dagger=dag)
                            got = D.unpack(yi).cpu().numpy().astype(np.complex128)
                            assert rel_l2(got, want) <= TOL[prec], (L, Nv, fmt, R, block, tc, dag)
        D.close()


@pytest.mark.parametrize("op,mass", [("wilson", 0.124), ("staggered", 0.05), ("brillouin", 0.2)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_apply_host_matches_device_apply(dg, op, mass, prec):
    """dirac_apply_host (host fields, slabs of t-slices streamed through the
    device) gives the device apply bit for bit: one slice per slab (Nt = 2, 5),
    two slices per slab with a one-slice last slab (Nt = 17), three with a
    one-slice last slab (Nt = 34); pinned and pageable host memory, D and D^+."""
    for L in ((4, 4, 2, 2), (4, 2, 4, 5), (2, 2, 4, 17), (2, 2, 2, 34)):
        Nv = 3
        V, psi = inputs(op, L, Nv, prec, 290)
        D = dg.Dirac(op, L, Nv, mass, prec)
        D.set_links(torch.from_numpy(V.astype(np.complex128 if prec == "f64" else np.complex64)).cuda())
        D.set_kernel_config(2, 64, 0 if prec == "f64" else 1)
        x = torch.from_numpy(psi.astype(np.complex128 if prec == "f64" else np.complex64))
        for dagger in (False, True):
            ref = D.apply(x.cuda(), dagger=dagger).cpu()
            for pinned in (True, False):
                xin = x.pin_memory() if pinned else x.clone()
                got = D.apply_host(xin, dagger=dagger)
                assert torch.equal(got, ref), (L, dagger, pinned)
            want = oracle.apply(op, V, psi, m0_of(op, mass), dagger=dagger)
            assert rel_l2(got.numpy().astype(np.complex128), want) <= TOL[prec]
        D.close()


@pytest.mark.parametrize("variant", [0, 2, 5, 6, 3])
def test_apply_host_launch_variants(dg, variant):
    """The slab sweeps of the t-march (2), x-row (5) and x-last (6) Wilson
    variants, and a configuration that cannot sweep a slab (3: replaced by
    variant 1)."""
    L, Nv = (8, 4, 2, 10), 5
    V, psi = inputs("wilson", L, Nv, "f32", 291)
    D = dg.Dirac("wilson", L, Nv, 0.122, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    D.set_kernel_config(2, 64, variant)
    x = torch.from_numpy(psi.astype(np.complex64)).pin_memory()
    want = oracle.apply("wilson", V, psi, oracle.kappa_to_m0(0.122))
    got = D.apply_host(x)
    assert rel_l2(got.numpy().astype(np.complex128), want) <= TOL["f32"]
    # repeated calls reuse the staging buffers and streams
    got2 = D.apply_host(x, out=torch.empty_like(x).pin_memory())
    assert torch.equal(got, got2)
    D.close()


def test_apply_host_rejects_device_memory(dg):
    L, Nv = (4, 4, 4, 4), 2
    D = dg.Dirac("wilson", L, Nv, 0.12, "f32")
    x = torch.zeros(D.canonical_shape, dtype=torch.complex64)
    with pytest.raises(dg.DiracError):
        D.apply_host(x)                                   # no links yet
    V, _ = inputs("wilson", L, Nv, "f32", 292)
    D.set_links(torch.from_numpy(V.astype(np.complex64)))
    xd = x.cuda()
    st = dg.dirac_apply_host(D.h, dg._ptr(xd), dg._ptr(xd), 0)
    assert st == dg.ERR_INVALID_ARG
    st = dg.dirac_apply_host(D.h, dg._ptr(x), dg._ptr(x), 0)   # out overlaps in
    assert st == dg.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        D.apply_host(xd)
    D.close()


def test_autotune(dg, tmp_path, monkeypatch):
    """The tuner keeps a supported configuration that reproduces the sweep and
    writes / reuses its cache file."""
    monkeypatch.setenv("DIRAC_TUNE_CACHE", str(tmp_path / "tune.txt"))
    L, Nv = (8, 8, 4, 8), 6
    V, psi = inputs("wilson", L, Nv, "f32", 250)
    D = dg.Dirac("wilson", L, Nv, 0.12, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    R, B, variant, ms = D.autotune(force=True)
    assert (R, B, variant) == D.kernel_config() and ms > 0
    assert "R%d B%d P%d T%d" % (R, B, variant, D.site_order()) in (tmp_path / "tune.txt").read_text()
    x = torch.from_numpy(psi.astype(np.complex64)).cuda()
    got = D.apply(x).cpu().numpy().astype(np.complex128)
    want = oracle.apply("wilson", V, psi, oracle.kappa_to_m0(0.12))
    assert rel_l2(got, want) <= TOL["f32"]
    D2 = dg.Dirac("wilson", L, Nv, 0.12, "f32")
    D2.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    assert D2.autotune()[:3] == (R, B, variant)           # from the cache
    assert D2.site_order() == D.site_order()
    D.close()
    D2.close()


@pytest.mark.parametrize("op,mass", [("wilson", 0.125), ("staggered", 0.02), ("brillouin", 0.1)])
def test_site_order_bit_identical(dg, op, mass):
    """The site order only permutes independent per-site work: every order
    gives the lexicographic result bit for bit (Nt = 5 leaves a partial
    t-chunk for tchunk = 2 and 3)."""
    L, Nv = (6, 4, 6, 5), 5
    V, psi = inputs(op, L, Nv, "f32", 280)
    D = dg.Dirac(op, L, Nv, mass, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    xi = D.pack(torch.from_numpy(psi.astype(np.complex64)).cuda())
    for variant in (0, 1):
        D.set_kernel_config(2, 64, variant)
        D.set_site_order(0)
        # zeroed outputs: the padding sites of the last block of 32 are never written
        ref = D.apply(xi, out=D.new_internal().zero_(), dagger=True).clone()
        for tc in (1, 2, 3, 5):
            D.set_site_order(tc)
            assert D.kernel_config() == (2, 64, variant) and D.site_order() == tc
            got = D.apply(xi, out=D.new_internal().zero_(), dagger=True)
            assert torch.equal(got, ref), (variant, tc)
    with pytest.raises(dg.DiracError):
        D.set_site_order(6)
    with pytest.raises(dg.DiracError):
        D.set_site_order(-1)
    D.close()


@pytest.mark.parametrize("op,mass", [("wilson", 0.13), ("staggered", 0.1), ("brillouin", 0.05)])
def test_tiny_and_odd_lattices(dg, op, mass):
    """Extent 2 (x+mu = x-mu, both hops land on the same site), odd extents,
    a single right-hand side."""
    for L, Nv in (((2, 2, 2, 2), 1), ((3, 5, 2, 3), 2), ((2, 3, 7, 2), 3)):
        V, psi = inputs(op, L, Nv, "f64", 230)
        got = run(dg, op, L, Nv, mass, "f64", V, psi, internal=True)
        want = oracle.apply(op, V, psi, m0_of(op, mass))
        assert rel_l2(got, want) <= TOL["f64"], L


def test_staggered_config_c1_full(dg):
    """Staggered, 8^4 periodic, Nv = 4, FP32, Haar links, m = 0: the whole lattice."""
    L, Nv = (8, 8, 8, 8), 4
    V, psi = inputs("staggered", L, Nv, "f32", 1001)
    got = run(dg, "staggered", L, Nv, 0.0, "f32", V, psi)
    assert rel_l2(got, oracle.apply("staggered", V, psi, 0.0)) <= TOL["f32"]


def _sampled(L, n, seed):
    vol = int(np.prod(L))
    rng = synth.rng(seed, synth.STREAM_MISC)
    Nx, Ny, Nz, Nt = L
    corners = [0, vol - 1, Nx - 1, Nx * Ny * Nz * (Nt - 1)]
    return np.unique(np.concatenate([corners, rng.integers(0, vol, n)]))


def test_wilson_full_size_sampled(dg):
    """Wilson 32^4, Nv = 12, FP32, kappa = 0.125, U = exp(0.3 i H): the
    workload the benchmark times, in every launch configuration the tuner can
    pick (so also the one the benchmark runs), D and D^+, checked on sampled
    sites including the lattice corners."""
    L, Nv = (32, 32, 32, 32), 12
    V = synth.round_to(synth.gauge_links(L, 3, "near_identity", 1002), "f32")
    psi = synth.round_to(synth.spinor(L, Nv, 4, 3, 2002), "f32")
    sites = _sampled(L, 256, 7)
    want = {dag: oracle.apply("wilson", V, psi, 0.0, sites=sites, dagger=dag) for dag in (False, True)}
    D = dg.Dirac("wilson", L, Nv, 0.125, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    xi = D.pack(torch.from_numpy(psi.astype(np.complex64)).cuda())
    yi = D.new_internal()
    st = torch.from_numpy(sites).cuda()
    for R in (1, 2, 3, 4):
        for block in (32, 64, 128, 256):
            for variant in dg.VARIANTS["wilson"]:
                if not dg.config_supported("wilson", "f32", R, block, variant, L):
                    continue
                D.set_kernel_config(R, block, variant)
                for dag in (False, True):
                    yi.fill_(0xFF)
                    D.apply(xi, out=yi, dagger=dag)
                    D.sync()                           # bounded waits of the staged variant report here
                    y = D.unpack(yi).reshape(-1, Nv, 4, 3)
                    assert bool(torch.isfinite(torch.view_as_real(y)).all())
                    got = y[st].cpu().numpy().astype(np.complex128)
                    assert rel_l2(got, want[dag], rhs_axis=1) <= TOL["f32"], (R, block, variant, dag)
    D.close()


def test_brillouin_full_size_sampled(dg):
    """Brillouin 24^3 x 48, Nv = 12, FP32 storage, m0 = 0.05, near-identity links."""
    L, Nv = (24, 24, 24, 48), 12
    V = synth.round_to(synth.gauge_links(L, 3, "near_identity", 1003), "f32")
    psi = synth.round_to(synth.spinor(L, Nv, 4, 3, 2003), "f32")
    got = run(dg, "brillouin", L, Nv, 0.05, "f32", V, psi).reshape(-1, Nv, 4, 3)
    sites = _sampled(L, 48, 8)
    want = oracle.apply("brillouin", V, psi, 0.05, sites=sites)
    assert rel_l2(got[sites], want, rhs_axis=1) <= TOL["f32"]


@pytest.mark.parametrize("op,mass", [("wilson", 0.1237), ("staggered", 0.031)])
@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_two_row_links(dg, op, mass, prec):
    """Link format 1 for Wilson and staggered (gauge compression: the first
    two rows of each Haar link stored, the third rebuilt as the conjugate
    cross product): parity with the oracle on a ragged volume in every launch
    shape that reads it, D and D^+; links that are not special unitary are
    refused and format 0 stays."""
    L, Nv = (6, 4, 6, 5), 5
    V, psi = inputs(op, L, Nv, "f32", 300)
    Vr, pr = rounded_for_oracle(V, psi, prec)
    D = dg.Dirac(op, L, Nv, mass, prec)
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    D.set_link_format(1)
    assert D.link_format() == 1
    xi = D.pack(torch.from_numpy(psi.astype(np.complex64)).cuda())
    Rs = (1, 2, 4, 6) if op == "staggered" else (1, 2, 3, 4)
    for dag in (False, True):
        want = oracle.apply(op, Vr, pr, m0_of(op, mass), dagger=dag)
        for R in Rs:
            for block in (32, 64):
                if not dg.config_supported(op, prec, R, block, 1, L):
                    continue
                D.set_kernel_config(R, block, 1)
                yi = D.new_internal()
                yi.fill_(0xFF)
                D.apply(xi, out=yi, dagger=dag)
                got = D.unpack(yi).cpu().numpy().astype(np.complex128)
                assert rel_l2(got, want) <= TOL[prec], (R, block, dag)
    # Gaussian matrices are not special unitary: refused, format 0 stays
    G = synth.complex_gaussian(synth.lattice_shape(L) + (4, 3, 3), 301)
    D.set_link_format(0)
    D.set_links(torch.from_numpy(G.astype(np.complex64)).cuda())
    with pytest.raises(dg.DiracError) as e:
        D.set_link_format(1)
    assert e.value.status == dg.ERR_INVALID_ARG and "special unitary" in str(e.value)
    assert D.link_format() == 0
    # recorded before the links: built at set_links; links that fail the check switch back to 0
    D2 = dg.Dirac(op, L, Nv, mass, prec)
    D2.set_link_format(1)
    D2.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    assert D2.link_format() == 1
    D2.set_links(torch.from_numpy(G.astype(np.complex64)).cuda())
    assert D2.link_format() == 0
    D.close()
    D2.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_brillouin_80_stored_links(dg, prec):
    """Brillouin link format 1 (all 80 W stored per site, W_{-d}(x) copied
    from W_d(x - d)^+ without rounding): bit for bit the 40-link sweep in
    variants 0 and 1, D and D^+, and parity with the oracle."""
    L, Nv = (4, 6, 2, 5), 3
    V, psi = inputs("brillouin", L, Nv, prec, 310, kind="near_identity")
    cdt = np.complex128 if prec == "f64" else np.complex64
    D = dg.Dirac("brillouin", L, Nv, 0.07, prec)
    D.set_links(torch.from_numpy(V.astype(cdt)).cuda())
    xi = D.pack(torch.from_numpy(psi.astype(cdt)).cuda())
    for variant in (0, 1):
        D.set_kernel_config(2, 64, variant)
        for dag in (False, True):
            D.set_link_format(0)
            ref = D.apply(xi, out=D.new_internal().zero_(), dagger=dag).clone()
            D.set_link_format(1)
            got = D.apply(xi, out=D.new_internal().zero_(), dagger=dag)
            assert torch.equal(got, ref), (variant, dag)
    if prec != "bf16":
        y = D.unpack(got).cpu().numpy().astype(np.complex128)
        want = oracle.apply("brillouin", V, psi, 0.07, dagger=True)
        assert rel_l2(y, want) <= TOL[prec]
    D.close()


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_brillouin_tensor_cores(dg, prec):
    """Variant 7, the Brillouin sweep on the tensor cores (tcgen05.mma, 16-bit
    operands, FP32 accumulation): parity with the oracle at the storage
    rounding bound, D and D^+, ragged volumes, partial and full blocks of 16
    right-hand sides, one and two blocks, x-rows of length 2 to 4 (the ring of
    A slots wraps around), canonical and internal fields, and the
    host-buffer apply (t-slabs)."""
    for L, Nv in (((4, 6, 2, 5), 5), ((4, 4, 4, 4), 12), ((3, 4, 2, 4), 20), ((2, 3, 4, 3), 7), ((4, 4, 2, 4), 16),
                  ((3, 2, 2, 3), 32)):
        V, psi = inputs("brillouin", L, Nv, prec, 320, kind="near_identity")
        pr = synth.round_to(psi, prec)     # W is built in FP64 from the FP32 links, rounded once
        D = dg.Dirac("brillouin", L, Nv, 0.07, prec)
        D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
        D.set_kernel_config(1, 128, 7)
        assert D.link_format() == 1
        x = torch.from_numpy(psi.astype(np.complex64)).cuda()
        for dag in (False, True):
            want = oracle.apply("brillouin", V, pr, 0.07, dagger=dag)
            got = D.apply(x, dagger=dag).cpu().numpy().astype(np.complex128)
            assert rel_l2(got, want) <= TOL[prec], (L, Nv, dag)
            xi = D.pack(x)
            yi = D.new_internal()
            yi.fill_(0xFF)
            D.apply(xi, out=yi, dagger=dag)
            D.sync()
            got = D.unpack(yi).cpu().numpy().astype(np.complex128)
            assert rel_l2(got, want) <= TOL[prec], (L, Nv, dag, "internal")
        hx = torch.from_numpy(psi.astype(np.complex64)).pin_memory()
        got = D.apply_host(hx).numpy().astype(np.complex128)
        assert rel_l2(got, oracle.apply("brillouin", V, pr, 0.07)) <= TOL[prec]
        D.close()


def test_autotune_link_format(dg, tmp_path, monkeypatch):
    """The tuner times both link formats and records the winner; the tuned
    handle reproduces the sweep, and a second handle takes the format from the
    cache."""
    monkeypatch.setenv("DIRAC_TUNE_CACHE", str(tmp_path / "tune.txt"))
    L, Nv = (8, 8, 4, 8), 4
    V, psi = inputs("wilson", L, Nv, "f32", 311)
    D = dg.Dirac("wilson", L, Nv, 0.12, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    D.autotune(force=True)
    f = D.link_format()
    assert f in (0, 1)
    assert " F%d " % f in (tmp_path / "tune.txt").read_text()
    got = D.apply(torch.from_numpy(psi.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    assert rel_l2(got, oracle.apply("wilson", V, psi, oracle.kappa_to_m0(0.12))) <= TOL["f32"]
    D2 = dg.Dirac("wilson", L, Nv, 0.12, "f32")
    D2.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    D2.autotune()
    assert D2.link_format() == f and D2.kernel_config() == D.kernel_config()
    D.close()
    D2.close()


def test_error_paths(dg):
    D = dg.Dirac("wilson", (4, 4, 4, 4), 2, 0.12, "f32")
    x = D.new_canonical()
    with pytest.raises(dg.DiracError) as e:          # links not loaded yet
        D.apply(x)
    assert e.value.status == dg.ERR_INVALID_ARG
    V = synth.gauge_links((4, 4, 4, 4), 3, "haar", 240)
    D.set_links(torch.from_numpy(V))                 # host links are copied
    with pytest.raises(dg.DiracError):               # aliasing
        D.apply(x, out=x)
    xh = torch.zeros_like(x, device="cpu")
    with pytest.raises(ValueError):                  # host tensor: stopped by the binding
        D.apply(xh, out=torch.zeros_like(xh))
    # the C entry point rejects host pointers by itself
    assert dg.dirac_apply(D.h, dg._ptr(torch.zeros_like(xh)), dg._ptr(xh), dg.CANONICAL) == dg.ERR_INVALID_ARG
    with pytest.raises(dg.DiracError) as e:
        D.set_kernel_config(5, 128)
    assert e.value.status == dg.ERR_UNSUPPORTED
    with pytest.raises(dg.DiracError) as e:
        D.set_kernel_config(4, 256, 3)               # 3 stages x 256 threads x 4 rhs: > 227 KB
    with pytest.raises(dg.DiracError):
        D.set_kernel_config(2, 128, 1)               # variant 1 takes 32 or 64 sites per block
    assert e.value.status == dg.ERR_UNSUPPORTED
    D.close()
