// Host emulation of the sweep bodies of the library (compiled for the CPU by
// tests/test_host_emulation.py; no GPU involved).  The per-site bodies are
// host-device functions, so they can run on the host over small lattices and
// be compared with one another:
//   1. even-odd half sweeps (dirac_eo.cuh) against the whole-lattice sweeps
//      restricted to one parity, FP32 and FP64, Wilson and staggered, both
//      adjoints, every site order of the half lattice (bit for bit), and
//      the half-lattice site order is a bijection;
//   2. the mixed-type sweeps of the split inner solve against the FP32
//      sweep applied to the 16-bit values (bit for bit);
//   3. the element mapping of the split CGLS step (16-bit element <-> two
//      FP32 elements of the same site);
//   4. double-float sweeps (dirac_df.cuh) against FP64 sweeps, all three
//      operators (relative difference below 1e-14).
// Exit status 0 when every check holds.
#include "dirac_df.cuh"
#include "dirac_eo.cuh"

#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

using namespace dirac;

namespace dirac {
// the launchers are not used on the host
cudaError_t launch_eo_wilson(int, bool, const EoArgs&, int, int, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_eo_staggered(int, bool, const EoArgs&, int, int, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_brillouin_tc(int, bool, const ApplyArgs&, cudaStream_t) { return cudaErrorInvalidValue; }
}  // namespace dirac

static int g_fail = 0;
static void expect(bool ok, const char* what)
{
    if (!ok) {
        printf("FAIL: %s\n", what);
        ++g_fail;
    }
}

static int parity(const Geom& g, long s)
{
    long r = s;
    int sum = 0;
    for (int mu = 0; mu < 4; ++mu) {
        sum += (int)(r % g.L[mu]);
        r /= g.L[mu];
    }
    return sum & 1;
}

// ---- 1. even-odd sweeps vs whole-lattice sweeps
template <typename T, int NSC, int R>
static double eo_vs_whole(int op, const int* L, int Nv, bool dag, int tc, unsigned seed)
{
    using A = typename Store<T>::A;
    const Geom g = make_geom(L[0], L[1], L[2], L[3]);
    const long vol = g.vol, vh = vol / 2;
    std::mt19937 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<cx<A>> links(4 * nblk_of(vol) * 9 * 32);
    for (auto& c : links) c = cx<A>{(A)(0.3 * nd(rng)), (A)(0.3 * nd(rng))};
    const size_t nf = (size_t)Nv * nblk_of(vol) * NSC * 32, nh = (size_t)Nv * nblk_of(vh) * NSC * 32;
    std::vector<cx<A>> psi(nf), full(nf), pe(nh), po(nh), oe(nh), oo(nh);
    for (auto& c : psi) c = cx<A>{(A)nd(rng), (A)nd(rng)};
    const double a = 4.3;
    ApplyArgs w{};
    w.g = g;
    w.Nv = Nv;
    w.in = psi.data();
    w.out = full.data();
    w.links = links.data();
    w.diag = a;
    w.diagf = (float)a;
    w.nsites = vol;
    w.nt = L[3];
    for (long s = 0; s < vol; ++s)
        for (int gi = 0; gi < Nv / R; ++gi) {
            if (op == OP_WILSON) {
                if (dag) wilson_site<T, R, true, 0>(w, s, gi);
                else wilson_site<T, R, false, 0>(w, s, gi);
            } else {
                if (dag) staggered_site<T, R, true, 0>(w, s, gi);
                else staggered_site<T, R, false, 0>(w, s, gi);
            }
        }
    for (int v = 0; v < Nv; ++v)
        for (long s = 0; s < vol; ++s) {
            cx<A> b[NSC];
            load_spinor<T, NSC>(psi.data(), vol, v, s, b);
            store_spinor<T, NSC>(parity(g, s) ? po.data() : pe.data(), vh, v, s >> 1, b);
        }
    std::vector<A> coef(2 * Nv);
    for (int v = 0; v < Nv; ++v) {
        coef[v] = (A)a;
        coef[Nv + v] = (A)1;
    }
    for (int par = 0; par < 2; ++par) {
        const EoArgs e = make_eo_args(g, Nv, par, par ? pe.data() : po.data(), par ? po.data() : pe.data(),
                                      par ? oo.data() : oe.data(), links.data(), coef.data(), tc);
        std::vector<int> seen(vh, 0);
        for (long p = 0; p < vh; ++p) {
            const long h = site_of(e.gh, p, e.tc, g.L[3], e.fdc, e.fdt);
            if (h < 0 || h >= vh) return 1e30;
            seen[h]++;
            const long s = eo_site(e, h);
            if (parity(g, s) != par || (s >> 1) != h) return 1e30;
        }
        for (long h = 0; h < vh; ++h)
            if (seen[h] != 1) return 1e30;
        for (long h = 0; h < vh; ++h)
            for (int gi = 0; gi < Nv / R; ++gi) {
                A q[R];
                if (op == OP_WILSON) {
                    if (dag) wilson_eo_site<T, T, T, T, R, true>(e, h, gi, q);
                    else wilson_eo_site<T, T, T, T, R, false>(e, h, gi, q);
                } else {
                    if (dag) staggered_eo_site<T, T, T, T, R, true>(e, h, gi, q);
                    else staggered_eo_site<T, T, T, T, R, false>(e, h, gi, q);
                }
            }
    }
    double d = 0.0;
    for (int v = 0; v < Nv; ++v)
        for (long s = 0; s < vol; ++s) {
            cx<A> x[NSC], y[NSC];
            load_spinor<T, NSC>(full.data(), vol, v, s, x);
            load_spinor<T, NSC>(parity(g, s) ? oo.data() : oe.data(), vh, v, s >> 1, y);
            for (int k = 0; k < NSC; ++k)
                d = std::fmax(d, std::fabs((double)x[k].re - (double)y[k].re) + std::fabs((double)x[k].im - (double)y[k].im));
        }
    return d;
}

// ---- 2. split-field sweeps vs the FP32 sweep on the 16-bit values
template <typename H>
static double split_vs_uniform(unsigned seed, double* norm_err)
{
    *norm_err = 0.0;
    const Geom g = make_geom(4, 4, 2, 6);
    const long vh = g.vol / 2;
    const int Nv = 4;
    constexpr int R = 2;
    std::mt19937 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    std::vector<cx<float>> links(4 * nblk_of(g.vol) * 9 * 32);
    for (auto& c : links) c = {0.3f * nd(rng), 0.3f * nd(rng)};
    const size_t n32 = (size_t)Nv * nblk_of(vh) * 12 * 32;
    std::vector<cx<float>> p32(n32), r32(n32), out32(n32), ref32(n32), tmp(n32);
    std::vector<uint32_t> p16(n32), o16(n32);
    for (int v = 0; v < Nv; ++v)
        for (long h = 0; h < vh; ++h) {
            cx<float> c[12], back[12];
            for (int k = 0; k < 12; ++k) c[k] = {nd(rng), nd(rng)};
            store_spinor<H, 12>(p16.data(), vh, v, h, c);
            load_spinor<H, 12>(p16.data(), vh, v, h, back);
            store_spinor<float, 12>(p32.data(), vh, v, h, back);
            for (int k = 0; k < 12; ++k) c[k] = {nd(rng), nd(rng)};
            store_spinor<float, 12>(r32.data(), vh, v, h, c);
        }
    std::vector<float> coef(2 * Nv);
    for (int v = 0; v < Nv; ++v) {
        coef[v] = 4.1f + 0.01f * (float)v;
        coef[Nv + v] = -1.f / coef[v];
    }
    double worst = 0.0;
    for (int kind = 0; kind < 4; ++kind) {
        EoArgs m = make_eo_args(g, Nv, kind % 2, nullptr, nullptr, nullptr, links.data(), coef.data(), 4);
        EoArgs u = m;
        const bool dag = kind >= 2;
        switch (kind) {
        case EO_SPLIT_HP: m.in = p16.data(); m.out = out32.data(); u.in = p32.data(); break;
        case EO_SPLIT_SP: m.in = r32.data(); m.in2 = p16.data(); m.out = out32.data(); u.in = r32.data(); u.in2 = p32.data(); break;
        case EO_SPLIT_HR: m.in = r32.data(); m.out = o16.data(); u.in = r32.data(); break;
        default: m.in = p16.data(); m.in2 = r32.data(); m.out = o16.data(); u.in = p32.data(); u.in2 = r32.data(); break;
        }
        u.out = ref32.data();
        // the fused norm of the stored output (the sweep only tests npart for null)
        std::vector<double> flag(1);
        m.npart = flag.data();
        for (long h = 0; h < vh; ++h)
            for (int gi = 0; gi < Nv / R; ++gi) {
                float q[R], qu[R];
                switch (kind) {
                case EO_SPLIT_HP: wilson_eo_site<float, H, float, float, R, false>(m, h, gi, q); break;
                case EO_SPLIT_SP: wilson_eo_site<float, float, H, float, R, false>(m, h, gi, q); break;
                case EO_SPLIT_HR: wilson_eo_site<float, float, float, H, R, true>(m, h, gi, q); break;
                default: wilson_eo_site<float, H, float, H, R, true>(m, h, gi, q); break;
                }
                if (dag) wilson_eo_site<float, float, float, float, R, true>(u, h, gi, qu);
                else wilson_eo_site<float, float, float, float, R, false>(u, h, gi, qu);
                for (int r = 0; r < R; ++r) {
                    cx<float> o[12];
                    if (kind < 2) load_spinor<float, 12>(out32.data(), vh, gi * R + r, h, o);
                    else load_spinor<H, 12>(o16.data(), vh, gi * R + r, h, o);
                    double n2 = 0.0;
                    for (int k = 0; k < 12; ++k) n2 += (double)o[k].re * o[k].re + (double)o[k].im * o[k].im;
                    *norm_err = std::fmax(*norm_err, std::fabs(q[r] - n2) / std::fmax(n2, 1e-30));
                }
            }
        for (int v = 0; v < Nv; ++v)
            for (long h = 0; h < vh; ++h) {
                cx<float> x[12], y[12];
                if (kind < 2) load_spinor<float, 12>(out32.data(), vh, v, h, x);
                else load_spinor<H, 12>(o16.data(), vh, v, h, x);
                load_spinor<float, 12>(ref32.data(), vh, v, h, y);
                if (kind >= 2) {   // the 16-bit output is the FP32 result rounded once
                    store_spinor<H, 12>(tmp.data(), vh, v, h, y);
                    load_spinor<H, 12>(tmp.data(), vh, v, h, y);
                }
                for (int k = 0; k < 12; ++k)
                    worst = std::fmax(worst, std::fabs((double)x[k].re - y[k].re) + std::fabs((double)x[k].im - y[k].im));
            }
    }
    return worst;
}

// ---- 3. the split CGLS step's element mapping
static long split_step_mapping()
{
    const long vh = 96 + 17;   // a ragged last block
    const int Nv = 3;
    const size_t m16 = nblk_of(vh) * 3 * 32;   // 16-byte elements per column of the 16-bit field
    long bad = 0;
    for (int v = 0; v < Nv; ++v)
        for (size_t i = 0; i < m16; ++i) {
            const size_t blk = i / 96, k = (i / 32) % 3, lane = i % 32;
            const size_t j0 = 2 * (v * m16) + (blk * 6 + 2 * k) * 32 + lane;
            const long h = (long)(blk * 32 + lane);
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * (int)k + q;
                if (blk_index(vh, 3, v, (int)k, h) != v * m16 + i) ++bad;
                if (blk_index(vh, 6, v, c / 2, h) != j0 + (size_t)(q / 2) * 32) ++bad;
            }
        }
    return bad;
}

// ---- 4. double-float sweeps vs FP64 sweeps
template <int NSC>
static double df_vs_f64(int op, const int* L, int Nv, double diag, unsigned seed)
{
    const Geom g = make_geom(L[0], L[1], L[2], L[3]);
    const long vol = g.vol;
    std::mt19937 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    const int nmat = op == OP_BRILLOUIN ? 40 : 4;
    const size_t nl = (size_t)nmat * nblk_of(vol) * 9 * 32, nf = (size_t)Nv * nblk_of(vol) * NSC * 32;
    std::vector<cx<double>> l64(nl), in64(nf), out64(nf);
    std::vector<float4> ldf(nl), indf(nf), outdf(nf);
    for (auto& c : l64) c = {0.4 * nd(rng), 0.4 * nd(rng)};
    for (auto& c : in64) c = {nd(rng), nd(rng)};
    auto conv = [](const std::vector<cx<double>>& a, std::vector<float4>& b) {
        for (size_t i = 0; i < a.size(); ++i) {
            const dfl r(a[i].re), m(a[i].im);
            b[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
        }
    };
    conv(l64, ldf);
    conv(in64, indf);
    ApplyArgs a{};
    a.g = g;
    a.Nv = Nv;
    a.diag = diag;
    a.diagf = (float)diag;
    a.nt = L[3];
    a.nsites = vol;
    ApplyArgs b = a;
    a.in = in64.data();
    a.out = out64.data();
    a.links = l64.data();
    b.in = indf.data();
    b.out = outdf.data();
    b.links = ldf.data();
    BriDir dirs[80];
    int reps[40];
    brillouin_tables(dirs, reps);
    for (long s = 0; s < vol; ++s)
        for (int v = 0; v < Nv; ++v) {
            if (op == OP_WILSON) {
                wilson_site<double, 1, false, 0>(a, s, v);
                wilson_site<f64df, 1, false, 0>(b, s, v);
            } else if (op == OP_STAGGERED) {
                staggered_site<double, 1, false, 0>(a, s, v);
                staggered_site<f64df, 1, false, 0>(b, s, v);
            } else {
                brillouin_site<double, 1, false>(a, s, v, dirs);
                brillouin_site<f64df, 1, false>(b, s, v, dirs);
            }
        }
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < nf; ++i) {
        const double re = (double)outdf[i].x + (double)outdf[i].y, im = (double)outdf[i].z + (double)outdf[i].w;
        num += (re - out64[i].re) * (re - out64[i].re) + (im - out64[i].im) * (im - out64[i].im);
        den += out64[i].re * out64[i].re + out64[i].im * out64[i].im;
    }
    return std::sqrt(num / den);
}

int main()
{
    const int shapes[][4] = {{4, 4, 4, 4}, {2, 2, 2, 2}, {6, 4, 2, 10}, {4, 2, 6, 12}, {8, 4, 4, 6}};
    for (const auto& L : shapes)
        for (int dag = 0; dag < 2; ++dag)
            for (int tc : {0, 4, 8}) {
                char what[128];
                snprintf(what, sizeof(what), "even-odd = whole lattice, %dx%dx%dx%d dag %d order %d", L[0], L[1], L[2],
                         L[3], dag, tc);
                expect(eo_vs_whole<float, 12, 2>(OP_WILSON, L, 4, dag, tc, 1) == 0.0, what);
                expect(eo_vs_whole<float, 12, 1>(OP_WILSON, L, 3, dag, tc, 2) == 0.0, what);
                expect(eo_vs_whole<float, 3, 4>(OP_STAGGERED, L, 8, dag, tc, 3) == 0.0, what);
                expect(eo_vs_whole<double, 12, 1>(OP_WILSON, L, 2, dag, tc, 4) == 0.0, what);
                expect(eo_vs_whole<double, 3, 2>(OP_STAGGERED, L, 2, dag, tc, 5) == 0.0, what);
            }
    double ne16 = 0.0, neh = 0.0;
    expect(split_vs_uniform<__nv_bfloat16>(6, &ne16) == 0.0, "split sweeps (BF16) = FP32 sweep on the BF16 values");
    expect(split_vs_uniform<__half>(7, &neh) == 0.0, "split sweeps (FP16) = FP32 sweep on the FP16 values");
    printf("fused output norms vs FP64 norms of the stored values: %.2e %.2e\n", ne16, neh);
    expect(ne16 < 1e-6 && neh < 1e-6, "fused |out|^2 per site = the norm of the stored output (FP32 sum of 24 squares)");
    expect(split_step_mapping() == 0, "split CGLS step element mapping");
    const int L1[4] = {4, 4, 4, 4}, L2[4] = {3, 4, 5, 2}, L3[4] = {4, 2, 4, 6}, L4[4] = {4, 4, 2, 4};
    const double dw = df_vs_f64<12>(OP_WILSON, L1, 2, 4.1, 8), dw2 = df_vs_f64<12>(OP_WILSON, L2, 3, 4.17, 9);
    const double ds = df_vs_f64<3>(OP_STAGGERED, L3, 2, 0.05, 10), db = df_vs_f64<12>(OP_BRILLOUIN, L4, 1, 1.925, 11);
    printf("double-float vs FP64: wilson %.2e %.2e staggered %.2e brillouin %.2e\n", dw, dw2, ds, db);
    expect(dw < 1e-14 && dw2 < 1e-14 && ds < 1e-14 && db < 1e-14, "double-float sweeps = FP64 sweeps to 1e-14");
    printf("%s (%d failures)\n", g_fail ? "FAILED" : "all checks hold", g_fail);
    return g_fail ? 1 : 0;
}
