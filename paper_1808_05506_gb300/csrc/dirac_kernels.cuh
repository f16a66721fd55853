// Per-site bodies of the three Dirac operators.  One call computes every
// component of the output spinor at one site for R right-hand sides, keeps
// the sums in registers and writes each output element once.
//
//   Wilson (Sec. 4, Eq. def_wils at c_SW = 0, lattice spacing 1):
//     D_W psi(x) = (4 + m0) psi(x)
//                  - 1/2 sum_mu [(1 - gamma_mu) V_mu(x) psi(x+mu)
//                               + (1 + gamma_mu) V_mu(x-mu)^+ psi(x-mu)]
//     (the 2-point derivative and the 9-point Laplacian combined; the spin
//     projectors 1 -+ gamma_mu have rank 2, so only a half spinor is
//     transported).  D_W^+ = gamma5 D_W gamma5 swaps the two projectors.
//   staggered (Sec. 3, plus a mass term):
//     D_S psi(x) = m psi(x) + 1/2 sum_mu eta_mu(x) [V_mu(x) psi(x+mu) - V_mu(x-mu)^+ psi(x-mu)]
//     D_S^+ = m - (hopping part).
//   Brillouin (Sec. 5, Eqs. def_bril, def_der, def_lap at c_SW = 0):
//     D_B psi(x) = (m0 + 15/8) psi(x)
//                  + sum_{dir != 0} W_dir(x) [rho_k (dir . gamma) - lambda_k / 2] psi(x+dir)
//     with k = |dir|_1; the 80 off-centre directions use 40 stored links and
//     W_{-dir}(x) = W_dir(x-dir)^+ (Tab. tab:off-axis caption).
//     D_B^+ = gamma5 D_B gamma5 flips the sign of the rho part.
//
// Chiral basis: gamma_mu = [[0, B_mu], [B_mu^+, 0]] with B_k = -i sigma_k,
// B_4 = 1; gamma5 = diag(1, 1, -1, -1).
#pragma once

#include <type_traits>

#include "dirac_common.cuh"

namespace dirac {

struct ApplyArgs {
    Geom g;
    int Nv;
    const void* in;       // internal spinor layout
    void* out;            // internal spinor layout
    const void* links;    // internal link layout (V_mu or the 40 stored W)
    double diag;          // (4 + m0) Wilson, m staggered, (m0 + 15/8) Brillouin
    const double* diag_v; // per-right-hand-side diagonal (device, Nv entries) or null: diag for all
    float diagf;          // the same in FP32, for the FP32-arithmetic sweeps (no FP64
    const float* diag_vf; // conversion inside them)
    int* err;             // device error word (kernels with bounded waits record DIRAC_TIMEOUT) or null
    int tc;               // site order of the grid (site_of): 0 lexicographic, else t-chunk
    // the sweep covers the slab of nt t-slices starting at slice t0 (sites
    // t0 Lx Ly Lz .. + nsites); the whole lattice: t0 = 0, nt = Nt
    int t0, nt;
    long nsites;
    FDiv fdc, fdt;        // division by Lz tc and by tc (site_of)
};

// site of the p-th work item of a sweep over the slab of a
template <typename Args> HD long slab_site(const Args& a, long p)
{
    return (long)a.t0 * a.g.stride[3] + site_of(a.g, p, a.tc, a.nt, a.fdc, a.fdt);
}

template <typename A> DEV_INLINE A diag_of(const ApplyArgs& a, int v)
{
    if constexpr (sizeof(A) == 4) return a.diag_vf ? a.diag_vf[v] : (a.diag_v ? (A)a.diag_v[v] : a.diagf);
    else return a.diag_v ? a.diag_v[v] : a.diag;
}

// ---------------------------------------------------------------- Wilson
// h = u + S B_MU d  (u: spins 0,1; d: spins 2,3), per colour
template <int MU, int S, typename A>
HD void wilson_project(const cx<A>* p, cx<A>* h)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<A> u0 = p[c], u1 = p[3 + c], d0 = p[6 + c], d1 = p[9 + c];
        cx<A> b0, b1;  // (B d)_0, (B d)_1
        if constexpr (MU == 0) { b0 = times_mi(d1); b1 = times_mi(d0); }
        else if constexpr (MU == 1) { b0 = -d1; b1 = d0; }
        else if constexpr (MU == 2) { b0 = times_mi(d0); b1 = times_i(d1); }
        else { b0 = d0; b1 = d1; }
        if constexpr (S > 0) { h[c] = u0 + b0; h[3 + c] = u1 + b1; }
        else { h[c] = u0 - b0; h[3 + c] = u1 - b1; }
    }
}

// acc(upper) += w, acc(lower) += S B_MU^+ w
template <int MU, int S, typename A>
HD void wilson_reconstruct(const cx<A>* w, cx<A>* acc)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<A> w0 = w[c], w1 = w[3 + c];
        acc[c] = acc[c] + w0;
        acc[3 + c] = acc[3 + c] + w1;
        cx<A> l0, l1;  // (B^+ w)_0, (B^+ w)_1
        if constexpr (MU == 0) { l0 = times_i(w1); l1 = times_i(w0); }
        else if constexpr (MU == 1) { l0 = w1; l1 = -w0; }
        else if constexpr (MU == 2) { l0 = times_i(w0); l1 = times_mi(w1); }
        else { l0 = w0; l1 = w1; }
        if constexpr (S > 0) { acc[6 + c] = acc[6 + c] + l0; acc[9 + c] = acc[9 + c] + l1; }
        else { acc[6 + c] = acc[6 + c] - l0; acc[9 + c] = acc[9 + c] - l1; }
    }
}

// one hop: acc_r += (1 + S gamma_MU) U psi_r(nbr),  U = V_MU(lsite) or its adjoint (BACK);
// NA: the loads bypass L1 (data this SM will not read again soon)
// FULL: every group holds R right-hand sides (Nv % R == 0), no clamping
// LF: link format (0 nine entries per link, 1 two rows, reconstructed)
template <typename T, int R, int MU, int S, bool BACK, bool NA = false, bool FULL = false, int LF = 0>
DEV_INLINE void wilson_hop(const ApplyArgs& a, long nbr, long lsite, int v0,
                           cx<typename Store<T>::A> (&acc)[R][12])
{
    using A = typename Store<T>::A;
    cx<A> U[9];
    load_link_f<T, NA, LF>(a.links, a.g.vol, MU, lsite, U);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        // a partial last group recomputes the last right-hand side instead of
        // branching, so that the loads of all R right-hand sides can be issued
        // together; only the stores are guarded
        const int v = FULL ? v0 + r : min(v0 + r, a.Nv - 1);
        cx<A> p[12], h[6], w[6];
        load_spinor_p<T, 12, NA>(a.in, a.g.vol, v, nbr, p);
        wilson_project<MU, S>(p, h);
        if constexpr (BACK) { mat_dag_vec(U, h, w); mat_dag_vec(U, h + 3, w + 3); }
        else { mat_vec(U, h, w); mat_vec(U, h + 3, w + 3); }
        wilson_reconstruct<MU, S>(w, acc[r]);
    }
}

// MODE 0: general.  MODE 1: whole groups (Nv % R == 0) and one diagonal for
// all right-hand sides; MODE 2: whole groups and a per-column diagonal.
// Modes 1 and 2 need no clamping and no branch on the diagonal.
template <typename A> DEV_INLINE A diag_mode(const ApplyArgs& a, int v, int mode)
{
    if (mode == 1) return sizeof(A) == 4 ? (A)a.diagf : (A)a.diag;
    if (mode == 2) {
        if constexpr (sizeof(A) == 4) return a.diag_vf[v];
        else return a.diag_v[v];
    }
    return diag_of<A>(a, v);
}

template <typename T, int R, bool DAG, int MODE = 0, int LF = 0>
DEV_INLINE void wilson_site(const ApplyArgs& a, long s, int group)
{
    constexpr bool FULL = MODE != 0;
    using A = typename Store<T>::A;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s, fwd, bwd, x);
    const int v0 = group * R;
    cx<A> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[r][i] = cx<A>{A(0), A(0)};
    // forward hop carries (1 - gamma), backward (1 + gamma); the adjoint swaps them
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    wilson_hop<T, R, 0, SF, false, false, FULL, LF>(a, s + fwd[0], s, v0, acc);
    wilson_hop<T, R, 0, SB, true, false, FULL, LF>(a, s + bwd[0], s + bwd[0], v0, acc);
    wilson_hop<T, R, 1, SF, false, false, FULL, LF>(a, s + fwd[1], s, v0, acc);
    wilson_hop<T, R, 1, SB, true, false, FULL, LF>(a, s + bwd[1], s + bwd[1], v0, acc);
    wilson_hop<T, R, 2, SF, false, false, FULL, LF>(a, s + fwd[2], s, v0, acc);
    wilson_hop<T, R, 2, SB, true, false, FULL, LF>(a, s + bwd[2], s + bwd[2], v0, acc);
    wilson_hop<T, R, 3, SF, false, false, FULL, LF>(a, s + fwd[3], s, v0, acc);
    wilson_hop<T, R, 3, SB, true, false, FULL, LF>(a, s + bwd[3], s + bwd[3], v0, acc);
    const A mh = (A)(-0.5);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = FULL ? v0 + r : min(v0 + r, a.Nv - 1);
        const A dg = diag_mode<A>(a, v, MODE);
        cx<A> p[12];
        load_spinor<T, 12>(a.in, a.g.vol, v, s, p);
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            cx<A> o;
            o.re = fma(mh, acc[r][i].re, dg * p[i].re);
            o.im = fma(mh, acc[r][i].im, dg * p[i].im);
            p[i] = o;
        }
        if (FULL || v0 + r < a.Nv) store_spinor<T, 12>(a.out, a.g.vol, v0 + r, s, p);
    }
}

// ---------------------------------------------------------------- Wilson, x hops last
// wilson_site with the 32 lanes of a warp on whole x-rows (Lx divides 32 and
// every warp starts at a multiple of 32 sites of its plane): the y, z and t
// hops load their spinors as usual; then, per right-hand side, the site's own
// spinor -- loaded once -- serves the diagonal term and both x hops.  Lane x
// forms (1 + SF gamma_1) psi(x), the forward projection, and sends it to
// lane x - 1; it forms U_x(x)^+ (1 + SB gamma_1) psi(x) with its own link, the
// backward hop of site x + 1, and sends it to lane x + 1.  Two of the nine
// spinor loads per site and one of the eight link loads disappear.  Every
// lane of the warp must call this with the same group.
// lane: the thread's lane in its warp; the warp's 32 consecutive work items
// start at a multiple of 32, so lane = x mod Lx and the row occupies the lanes
// lane - x .. lane - x + Lx - 1
template <typename T, int R, bool DAG, int MODE = 0, int LF = 0>
DEV_INLINE void wilson_site_xlast(const ApplyArgs& a, long s, int lane, int group)
{
    constexpr bool FULL = MODE != 0;
    using A = typename Store<T>::A;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s, fwd, bwd, x);
    const int Lx = a.g.L[0];
    const int lane_f = lane - x[0] + (x[0] + 1 == Lx ? 0 : x[0] + 1);   // site x + 1
    const int lane_b = lane - x[0] + (x[0] == 0 ? Lx - 1 : x[0] - 1);   // site x - 1
    const int v0 = group * R;
    cx<A> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[r][i] = cx<A>{A(0), A(0)};
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    wilson_hop<T, R, 1, SF, false, false, FULL, LF>(a, s + fwd[1], s, v0, acc);
    wilson_hop<T, R, 1, SB, true, false, FULL, LF>(a, s + bwd[1], s + bwd[1], v0, acc);
    wilson_hop<T, R, 2, SF, false, false, FULL, LF>(a, s + fwd[2], s, v0, acc);
    wilson_hop<T, R, 2, SB, true, false, FULL, LF>(a, s + bwd[2], s + bwd[2], v0, acc);
    wilson_hop<T, R, 3, SF, false, false, FULL, LF>(a, s + fwd[3], s, v0, acc);
    wilson_hop<T, R, 3, SB, true, false, FULL, LF>(a, s + bwd[3], s + bwd[3], v0, acc);
    cx<A> U[9];
    load_link_f<T, false, LF>(a.links, a.g.vol, 0, s, U);
    const A mh = (A)(-0.5);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = FULL ? v0 + r : min(v0 + r, a.Nv - 1);
        cx<A> pc[12], h[6], w[6], q[6];
        load_spinor<T, 12>(a.in, a.g.vol, v, s, pc);
        wilson_project<0, SF>(pc, h);
#pragma unroll
        for (int i = 0; i < 6; ++i) q[i] = shfl_cx(h[i], lane_f);
        mat_vec(U, q, w);
        mat_vec(U, q + 3, w + 3);
        wilson_reconstruct<0, SF>(w, acc[r]);
        wilson_project<0, SB>(pc, h);
        mat_dag_vec(U, h, w);
        mat_dag_vec(U, h + 3, w + 3);
#pragma unroll
        for (int i = 0; i < 6; ++i) q[i] = shfl_cx(w[i], lane_b);
        wilson_reconstruct<0, SB>(q, acc[r]);
        const A dg = diag_mode<A>(a, v, MODE);
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            cx<A> o;
            o.re = fma(mh, acc[r][i].re, dg * pc[i].re);
            o.im = fma(mh, acc[r][i].im, dg * pc[i].im);
            pc[i] = o;
        }
        if (FULL || v0 + r < a.Nv) store_spinor<T, 12>(a.out, a.g.vol, v0 + r, s, pc);
    }
}

// ---------------------------------------------------------------- Wilson, t-march
// One thread owns the site column (x, y, z) for the slices t0 <= t < t1 and
// one group of R right-hand sides.  Along t each spinor and each t-link is
// read once: psi(t + 1), loaded for the forward t hop of slice t, is the
// diagonal term of slice t + 1, and U_t(t), loaded for that hop, also forms
// the backward t hop of slice t + 1, U_t(t)^+ (1 + S gamma_4) psi(t), which
// is carried to the next step as a half spinor.  Only the x, y and z hops go
// to memory at every step.
template <typename T, int R, bool DAG>
DEV_INLINE void wilson_column(const ApplyArgs& a, long s3, int group, int t0, int t1)
{
    using A = typename Store<T>::A;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const long vol3 = a.g.stride[3];
    const int Lt = a.g.L[3];
    const int v0 = group * R;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s3, fwd, bwd, x);   // x, y, z offsets do not depend on t
    cx<A> pc[R][12];   // psi(t)
    cx<A> hb[R][6];    // U_t(t - 1)^+ (1 + SB gamma_4) psi(t - 1)
    {
        const long sp = s3 + vol3 * (t0 == 0 ? Lt - 1 : t0 - 1);
        cx<A> U[9];
        load_link<T>(a.links, a.g.vol, 3, sp, U);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = min(v0 + r, a.Nv - 1);
            cx<A> p[12], h[6];
            load_spinor<T, 12>(a.in, a.g.vol, v, sp, p);
            wilson_project<3, SB>(p, h);
            mat_dag_vec(U, h, hb[r]);
            mat_dag_vec(U, h + 3, hb[r] + 3);
            load_spinor<T, 12>(a.in, a.g.vol, v, s3 + vol3 * t0, pc[r]);
        }
    }
    const A mh = (A)(-0.5);
#pragma unroll 1
    for (int t = t0; t < t1; ++t) {
        const long s = s3 + vol3 * t;
        const long sn = s3 + vol3 * (t + 1 == Lt ? 0 : t + 1);
        cx<A> acc[R][12];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[r][i] = cx<A>{A(0), A(0)};
        wilson_hop<T, R, 0, SF, false>(a, s + fwd[0], s, v0, acc);
        wilson_hop<T, R, 0, SB, true>(a, s + bwd[0], s + bwd[0], v0, acc);
        wilson_hop<T, R, 1, SF, false>(a, s + fwd[1], s, v0, acc);
        wilson_hop<T, R, 1, SB, true>(a, s + bwd[1], s + bwd[1], v0, acc);
        wilson_hop<T, R, 2, SF, false>(a, s + fwd[2], s, v0, acc);
        wilson_hop<T, R, 2, SB, true>(a, s + bwd[2], s + bwd[2], v0, acc);
        cx<A> U[9];
        load_link<T>(a.links, a.g.vol, 3, s, U);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = min(v0 + r, a.Nv - 1);
            cx<A> pn[12], h[6], w[6];
            load_spinor<T, 12>(a.in, a.g.vol, v, sn, pn);
            // forward t hop of slice t, then the carried backward hop
            wilson_project<3, SF>(pn, h);
            mat_vec(U, h, w);
            mat_vec(U, h + 3, w + 3);
            wilson_reconstruct<3, SF>(w, acc[r]);
            wilson_reconstruct<3, SB>(hb[r], acc[r]);
            // backward t hop of slice t + 1
            wilson_project<3, SB>(pc[r], h);
            mat_dag_vec(U, h, hb[r]);
            mat_dag_vec(U, h + 3, hb[r] + 3);
            const A dg = diag_of<A>(a, v);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                cx<A> o;
                o.re = fma(mh, acc[r][i].re, dg * pc[r][i].re);
                o.im = fma(mh, acc[r][i].im, dg * pc[r][i].im);
                acc[r][i] = o;
                pc[r][i] = pn[i];
            }
            if (v0 + r < a.Nv) store_spinor<T, 12>(a.out, a.g.vol, v0 + r, s, acc[r]);
        }
    }
}

// ---------------------------------------------------------------- Wilson, x-rows in a warp
// wilson_column with the 32 lanes of a warp on 32 consecutive sites of the
// (x, y, z) volume, i.e. on whole x-rows (Lx divides 32).  The x hops need no
// memory access: lane x sends (1 + SF gamma_1) psi(x), the forward hop's
// projection, to lane x - 1, and U_x(x)^+ (1 + SB gamma_1) psi(x), the
// backward hop of site x + 1 built with its own link, to lane x + 1.  The t
// hops are carried as in wilson_column; only the y and z hops load spinors.
// Requires whole warps: every lane of the warp calls this with the same
// group and t range.
template <typename T, int R, bool DAG>
DEV_INLINE void wilson_xrow(const ApplyArgs& a, long s3, int lane, int group, int t0, int t1)
{
    using A = typename Store<T>::A;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const long vol3 = a.g.stride[3];
    const int Lt = a.g.L[3], Lx = a.g.L[0];
    const int v0 = group * R;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s3, fwd, bwd, x);
    const int lane_f = lane - x[0] + (x[0] + 1 == Lx ? 0 : x[0] + 1);   // site x + 1
    const int lane_b = lane - x[0] + (x[0] == 0 ? Lx - 1 : x[0] - 1);   // site x - 1
    cx<A> pc[R][12];   // psi(t)
    cx<A> hb[R][6];    // U_t(t - 1)^+ (1 + SB gamma_4) psi(t - 1)
    {
        const long sp = s3 + vol3 * (t0 == 0 ? Lt - 1 : t0 - 1);
        cx<A> U[9];
        load_link<T>(a.links, a.g.vol, 3, sp, U);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = min(v0 + r, a.Nv - 1);
            cx<A> p[12], h[6];
            load_spinor<T, 12>(a.in, a.g.vol, v, sp, p);
            wilson_project<3, SB>(p, h);
            mat_dag_vec(U, h, hb[r]);
            mat_dag_vec(U, h + 3, hb[r] + 3);
            load_spinor<T, 12>(a.in, a.g.vol, v, s3 + vol3 * t0, pc[r]);
        }
    }
    const A mh = (A)(-0.5);
#pragma unroll 1
    for (int t = t0; t < t1; ++t) {
        const long s = s3 + vol3 * t;
        const long sn = s3 + vol3 * (t + 1 == Lt ? 0 : t + 1);
        cx<A> acc[R][12];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[r][i] = cx<A>{A(0), A(0)};
        {
            cx<A> U[9];
            load_link<T>(a.links, a.g.vol, 0, s, U);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                cx<A> h[6], w[6], q[6];
                wilson_project<0, SF>(pc[r], h);
#pragma unroll
                for (int i = 0; i < 6; ++i) q[i] = shfl_cx(h[i], lane_f);
                mat_vec(U, q, w);
                mat_vec(U, q + 3, w + 3);
                wilson_reconstruct<0, SF>(w, acc[r]);
                wilson_project<0, SB>(pc[r], h);
                mat_dag_vec(U, h, w);
                mat_dag_vec(U, h + 3, w + 3);
#pragma unroll
                for (int i = 0; i < 6; ++i) q[i] = shfl_cx(w[i], lane_b);
                wilson_reconstruct<0, SB>(q, acc[r]);
            }
        }
        wilson_hop<T, R, 1, SF, false>(a, s + fwd[1], s, v0, acc);
        wilson_hop<T, R, 1, SB, true>(a, s + bwd[1], s + bwd[1], v0, acc);
        wilson_hop<T, R, 2, SF, false>(a, s + fwd[2], s, v0, acc);
        wilson_hop<T, R, 2, SB, true>(a, s + bwd[2], s + bwd[2], v0, acc);
        cx<A> U[9];
        load_link<T>(a.links, a.g.vol, 3, s, U);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = min(v0 + r, a.Nv - 1);
            cx<A> pn[12], h[6], w[6];
            load_spinor<T, 12>(a.in, a.g.vol, v, sn, pn);
            wilson_project<3, SF>(pn, h);
            mat_vec(U, h, w);
            mat_vec(U, h + 3, w + 3);
            wilson_reconstruct<3, SF>(w, acc[r]);
            wilson_reconstruct<3, SB>(hb[r], acc[r]);
            wilson_project<3, SB>(pc[r], h);
            mat_dag_vec(U, h, hb[r]);
            mat_dag_vec(U, h + 3, hb[r] + 3);
            const A dg = diag_of<A>(a, v);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                cx<A> o;
                o.re = fma(mh, acc[r][i].re, dg * pc[r][i].re);
                o.im = fma(mh, acc[r][i].im, dg * pc[r][i].im);
                acc[r][i] = o;
                pc[r][i] = pn[i];
            }
            if (v0 + r < a.Nv) store_spinor<T, 12>(a.out, a.g.vol, v0 + r, s, acc[r]);
        }
    }
}

// ---------------------------------------------------------------- Wilson, pipelined
// The same sweep with the loads of hop h + ST - 1 in flight (cp.async into
// this thread's own shared-memory slots) while hop h is computed, so that the
// memory latency is covered without holding the data in registers.
// Hops 0..7 are (mu, +), (mu, -) for mu = 0..3; hop 8 is the site itself.
// Shared memory per thread and stage: R*K 16-byte spinor elements and the 9
// link entries; layout [stage][element][thread] (conflict-free 16-byte rows).
template <typename T, int R>
struct WilsonPipe {
    static constexpr int K = SpinorLayout<T, 12>::K;
    static constexpr int E = R * K;
    static constexpr int LB = (int)sizeof(typename Store<T>::One);
    static constexpr size_t stage_bytes_per_thread = (size_t)E * 16 + 9 * LB;
};

template <typename T, int R>
DEV_INLINE void wilson_issue(const ApplyArgs& a, int h, long nbr, long lsite, int v0, char* stage, int tid,
                             int nthr)
{
    using P = WilsonPipe<T, R>;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (v0 + r < a.Nv) {
#pragma unroll
            for (int k = 0; k < P::K; ++k) {
                const size_t gi = blk_index(a.g.vol, P::K, v0 + r, k, nbr);
                cp_async<16>(stage + ((size_t)(r * P::K + k) * nthr + tid) * 16,
                             static_cast<const char*>(a.in) + gi * 16);
            }
        }
    }
    if (h < 8) {
        char* lb = stage + (size_t)P::E * 16 * nthr;
        const int mu = h >> 1;
#pragma unroll
        for (int e = 0; e < 9; ++e)
            cp_async<P::LB>(lb + ((size_t)e * nthr + tid) * P::LB,
                            static_cast<const char*>(a.links) + blk_index(a.g.vol, 9, mu, e, lsite) * P::LB);
    }
    cp_async_commit();
}

// plain (shared-memory) reads of one complex / one 16-byte element
template <typename T> DEV_INLINE cx<typename Store<T>::A> sm_one(const char* p);
template <> DEV_INLINE cx<double> sm_one<double>(const char* p)
{
    double2 v = *reinterpret_cast<const double2*>(p);
    return {v.x, v.y};
}
template <> DEV_INLINE cx<float> sm_one<float>(const char* p)
{
    float2 v = *reinterpret_cast<const float2*>(p);
    return {v.x, v.y};
}
template <> DEV_INLINE cx<float> sm_one<__nv_bfloat16>(const char* p)
{
    return unpack2(*reinterpret_cast<const uint32_t*>(p), (__nv_bfloat16*)nullptr);
}
template <> DEV_INLINE cx<float> sm_one<__half>(const char* p)
{
    return unpack2(*reinterpret_cast<const uint32_t*>(p), (__half*)nullptr);
}
template <typename T> DEV_INLINE void sm_vec(const char* p, cx<typename Store<T>::A>* o);
template <> DEV_INLINE void sm_vec<double>(const char* p, cx<double>* o) { o[0] = sm_one<double>(p); }
template <> DEV_INLINE void sm_vec<float>(const char* p, cx<float>* o)
{
    float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = {v.x, v.y};
    o[1] = {v.z, v.w};
}
template <typename H> DEV_INLINE void sm_vec16(const char* p, cx<float>* o)
{
    uint4 v = *reinterpret_cast<const uint4*>(p);
    o[0] = unpack2(v.x, (H*)nullptr);
    o[1] = unpack2(v.y, (H*)nullptr);
    o[2] = unpack2(v.z, (H*)nullptr);
    o[3] = unpack2(v.w, (H*)nullptr);
}
template <> DEV_INLINE void sm_vec<__nv_bfloat16>(const char* p, cx<float>* o) { sm_vec16<__nv_bfloat16>(p, o); }
template <> DEV_INLINE void sm_vec<__half>(const char* p, cx<float>* o) { sm_vec16<__half>(p, o); }

template <typename T, int R, bool DAG, int H>
DEV_INLINE void wilson_pipe_hop(const ApplyArgs& a, const char* stage, int v0, int tid, int nthr,
                                cx<typename Store<T>::A> (&acc)[R][12])
{
    using A = typename Store<T>::A;
    using P = WilsonPipe<T, R>;
    using L = SpinorLayout<T, 12>;
    constexpr int MU = H >> 1;
    constexpr bool BACK = (H & 1) != 0;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int S = BACK ? -SF : SF;
    cx<A> U[9];
    const char* lb = stage + (size_t)P::E * 16 * nthr;
#pragma unroll
    for (int e = 0; e < 9; ++e) U[e] = sm_one<T>(lb + ((size_t)e * nthr + tid) * P::LB);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (v0 + r < a.Nv) {
            cx<A> p[12], h[6], w[6];
#pragma unroll
            for (int k = 0; k < P::K; ++k) {
                const char* q = stage + ((size_t)(r * P::K + k) * nthr + tid) * 16;
                if constexpr (L::CPV == 1) p[k] = sm_one<T>(q);
                else sm_vec<T>(q, p + k * L::CPV);
            }
            wilson_project<MU, S>(p, h);
            if constexpr (BACK) { mat_dag_vec(U, h, w); mat_dag_vec(U, h + 3, w + 3); }
            else { mat_vec(U, h, w); mat_vec(U, h + 3, w + 3); }
            wilson_reconstruct<MU, S>(w, acc[r]);
        }
    }
}

template <typename T, int R, bool DAG, int ST, int H>
DEV_INLINE void wilson_pipe_step(const ApplyArgs& a, const long* nb, const long* ls, int v0, char* smem, int tid,
                                 int nthr, cx<typename Store<T>::A> (&acc)[R][12])
{
    using P = WilsonPipe<T, R>;
    const size_t sb = P::stage_bytes_per_thread * nthr;
    if constexpr (H + ST - 1 <= 8) wilson_issue<T, R>(a, H + ST - 1, nb[H + ST - 1], ls[H + ST - 1], v0,
                                                      smem + ((H + ST - 1) % ST) * sb, tid, nthr);
    else cp_async_commit();
    cp_async_wait<ST - 1>();
    const char* stage = smem + (H % ST) * sb;
    if constexpr (H < 8) {
        wilson_pipe_hop<T, R, DAG, H>(a, stage, v0, tid, nthr, acc);
        wilson_pipe_step<T, R, DAG, ST, H + 1>(a, nb, ls, v0, smem, tid, nthr, acc);
    } else {
        using A = typename Store<T>::A;
        using L = SpinorLayout<T, 12>;
        const A mh = (A)(-0.5);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (v0 + r < a.Nv) {
                const A dg = diag_of<A>(a, v0 + r);
                cx<A> p[12];
#pragma unroll
                for (int k = 0; k < P::K; ++k) {
                    const char* q = stage + ((size_t)(r * P::K + k) * nthr + tid) * 16;
                    if constexpr (L::CPV == 1) p[k] = sm_one<T>(q);
                    else sm_vec<T>(q, p + k * L::CPV);
                }
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    cx<A> o;
                    o.re = fma(mh, acc[r][i].re, dg * p[i].re);
                    o.im = fma(mh, acc[r][i].im, dg * p[i].im);
                    p[i] = o;
                }
                store_spinor<T, 12>(a.out, a.g.vol, v0 + r, nb[8], p);
            }
        }
    }
}

template <typename T, int R, bool DAG, int ST>
DEV_INLINE void wilson_site_pipe(const ApplyArgs& a, long s, int group, char* smem, int tid, int nthr)
{
    using A = typename Store<T>::A;
    using P = WilsonPipe<T, R>;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s, fwd, bwd, x);
    const int v0 = group * R;
    long nb[9], ls[9];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        nb[2 * mu] = s + fwd[mu];
        ls[2 * mu] = s;
        nb[2 * mu + 1] = s + bwd[mu];
        ls[2 * mu + 1] = s + bwd[mu];
    }
    nb[8] = s;
    ls[8] = s;
    const size_t sb = P::stage_bytes_per_thread * nthr;
#pragma unroll
    for (int h = 0; h < ST - 1; ++h) wilson_issue<T, R>(a, h, nb[h], ls[h], v0, smem + h * sb, tid, nthr);
    cx<A> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[r][i] = cx<A>{A(0), A(0)};
    wilson_pipe_step<T, R, DAG, ST, 0>(a, nb, ls, v0, smem, tid, nthr, acc);
}

// ---------------------------------------------------------------- staggered
// MODE and LF as in wilson_site
template <typename T, int R, bool DAG, int MODE = 0, int LF = 0>
DEV_INLINE void staggered_site(const ApplyArgs& a, long s, int group)
{
    constexpr bool FAST = MODE != 0;
    using A = typename Store<T>::A;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s, fwd, bwd, x);
    const int v0 = group * R;
    cx<A> acc[R][3];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[r][i] = cx<A>{A(0), A(0)};
    int par = 0;  // x_0 + ... + x_{mu-1}
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const A eta = (par & 1) ? A(-1) : A(1);
        par += x[mu];
        cx<A> Uf[9], Ub[9];
        load_link_f<T, false, LF>(a.links, a.g.vol, mu, s, Uf);
        load_link_f<T, false, LF>(a.links, a.g.vol, mu, s + bwd[mu], Ub);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = FAST ? v0 + r : min(v0 + r, a.Nv - 1);   // partial group: recompute, store guarded
            cx<A> pf[3], pb[3], w[3] = {}, wb[3] = {};
            load_spinor<T, 3>(a.in, a.g.vol, v, s + fwd[mu], pf);
            load_spinor<T, 3>(a.in, a.g.vol, v, s + bwd[mu], pb);
            mat_vec(Uf, pf, w);
            mat_dag_vec(Ub, pb, wb);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<A> d = w[c] - wb[c];
                acc[r][c].re = fma(eta, d.re, acc[r][c].re);
                acc[r][c].im = fma(eta, d.im, acc[r][c].im);
            }
        }
    }
    const A hf = DAG ? A(-0.5) : A(0.5);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = FAST ? v0 + r : min(v0 + r, a.Nv - 1);
        const A dg = diag_mode<A>(a, v, MODE);
        cx<A> p[3];
        load_spinor<T, 3>(a.in, a.g.vol, v, s, p);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<A> o;
            o.re = fma(hf, acc[r][c].re, dg * p[c].re);
            o.im = fma(hf, acc[r][c].im, dg * p[c].im);
            p[c] = o;
        }
        if (FAST || v0 + r < a.Nv) store_spinor<T, 3>(a.out, a.g.vol, v0 + r, s, p);
    }
}

// staggered_site with the x hops last, by lane exchange of the site's own
// spinor (the warp layout of wilson_site_xlast: whole x-rows per warp, lane
// the thread's lane): lane x sends psi(x) to lane x - 1 for its forward hop
// and V_x(x)^+ psi(x) to lane x + 1 for its backward hop (eta_0 = 1)
template <typename T, int R, bool DAG, int MODE = 0, int LF = 0>
DEV_INLINE void staggered_site_xlast(const ApplyArgs& a, long s, int lane, int group)
{
    constexpr bool FAST = MODE != 0;
    using A = typename Store<T>::A;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s, fwd, bwd, x);
    const int Lx = a.g.L[0];
    const int lane_f = lane - x[0] + (x[0] + 1 == Lx ? 0 : x[0] + 1);   // site x + 1
    const int lane_b = lane - x[0] + (x[0] == 0 ? Lx - 1 : x[0] - 1);   // site x - 1
    const int v0 = group * R;
    cx<A> acc[R][3];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[r][i] = cx<A>{A(0), A(0)};
    int par = x[0];  // x_0 + ... + x_{mu-1}, from mu = 1 on
#pragma unroll
    for (int mu = 1; mu < 4; ++mu) {
        const A eta = (par & 1) ? A(-1) : A(1);
        par += x[mu];
        cx<A> Uf[9], Ub[9];
        load_link_f<T, false, LF>(a.links, a.g.vol, mu, s, Uf);
        load_link_f<T, false, LF>(a.links, a.g.vol, mu, s + bwd[mu], Ub);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = FAST ? v0 + r : min(v0 + r, a.Nv - 1);
            cx<A> pf[3], pb[3], w[3] = {}, wb[3] = {};
            load_spinor<T, 3>(a.in, a.g.vol, v, s + fwd[mu], pf);
            load_spinor<T, 3>(a.in, a.g.vol, v, s + bwd[mu], pb);
            mat_vec(Uf, pf, w);
            mat_dag_vec(Ub, pb, wb);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<A> d = w[c] - wb[c];
                acc[r][c].re = fma(eta, d.re, acc[r][c].re);
                acc[r][c].im = fma(eta, d.im, acc[r][c].im);
            }
        }
    }
    cx<A> U[9];
    load_link_f<T, false, LF>(a.links, a.g.vol, 0, s, U);
    const A hf = DAG ? A(-0.5) : A(0.5);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = FAST ? v0 + r : min(v0 + r, a.Nv - 1);
        cx<A> p[3], q[3], w[3], wb[3];
        load_spinor<T, 3>(a.in, a.g.vol, v, s, p);
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c] = shfl_cx(p[c], lane_f);
        mat_vec(U, q, w);          // V_x(x) psi(x + 1)
        mat_dag_vec(U, p, q);      // V_x(x)^+ psi(x): the backward hop of site x + 1
#pragma unroll
        for (int c = 0; c < 3; ++c) wb[c] = shfl_cx(q[c], lane_b);
        const A dg = diag_mode<A>(a, v, MODE);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cx<A> d = w[c] - wb[c];
            cx<A> t;
            t.re = acc[r][c].re + d.re;
            t.im = acc[r][c].im + d.im;
            cx<A> o;
            o.re = fma(hf, t.re, dg * p[c].re);
            o.im = fma(hf, t.im, dg * p[c].im);
            p[c] = o;
        }
        if (FAST || v0 + r < a.Nv) store_spinor<T, 3>(a.out, a.g.vol, v0 + r, s, p);
    }
}

// ---------------------------------------------------------------- Brillouin
// The 80 off-centre directions, each with its spin matrix
//   M = rho_k (dir . gamma) - lambda_k / 2 = [[a, rho Q], [rho Q^+, a]],
//   Q = sum_mu dir_mu B_mu,  a = -lambda_k / 2.
struct BriDir {
    signed char d[4];    // offset
    signed char rep;     // stored direction index 0..39
    signed char neg;     // 1: W_dir(x) = W_rep(x + dir)^+
    double a;            // -lambda_k / 2
    double q[8];         // rho_k Q: q00 re, im, q01 re, im, q10 re, im, q11 re, im
    float af;            // the same coefficients rounded to FP32, for the FP32 sweeps (no
    float qf[8];         // FP64 -> FP32 conversions in the inner loop)
};

template <typename A> struct BriDirA { A a; cx<A> q00, q01, q10, q11; };

template <typename A, bool DAG>
HD BriDirA<A> bri_coeffs(const BriDir& D)
{
    BriDirA<A> c;
    const A sg = DAG ? A(-1) : A(1);
    if constexpr (sizeof(A) == 4) {
        c.a = D.af;
        c.q00 = {sg * D.qf[0], sg * D.qf[1]};
        c.q01 = {sg * D.qf[2], sg * D.qf[3]};
        c.q10 = {sg * D.qf[4], sg * D.qf[5]};
        c.q11 = {sg * D.qf[6], sg * D.qf[7]};
    } else {
        c.a = (A)D.a;
        c.q00 = {sg * (A)D.q[0], sg * (A)D.q[1]};
        c.q01 = {sg * (A)D.q[2], sg * (A)D.q[3]};
        c.q10 = {sg * (A)D.q[4], sg * (A)D.q[5]};
        c.q11 = {sg * (A)D.q[6], sg * (A)D.q[7]};
    }
    return c;
}

// chi = M psi
template <typename A>
DEV_INLINE void bri_spin(const BriDirA<A>& m, const cx<A>* p, cx<A>* chi)
{
    if constexpr (sizeof(A) == 4) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<A> u0 = p[c], u1 = p[3 + c], d0 = p[6 + c], d1 = p[9 + c];
            cx<A> t;
            t = cx<A>{m.a * u0.re, m.a * u0.im}; t = cfma2(m.q00, d0, t); chi[c] = cfma2(m.q01, d1, t);
            t = cx<A>{m.a * u1.re, m.a * u1.im}; t = cfma2(m.q10, d0, t); chi[3 + c] = cfma2(m.q11, d1, t);
            t = cx<A>{m.a * d0.re, m.a * d0.im}; t = cfma2_conj(m.q00, u0, t); chi[6 + c] = cfma2_conj(m.q10, u1, t);
            t = cx<A>{m.a * d1.re, m.a * d1.im}; t = cfma2_conj(m.q01, u0, t); chi[9 + c] = cfma2_conj(m.q11, u1, t);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<A> u0 = p[c], u1 = p[3 + c], d0 = p[6 + c], d1 = p[9 + c];
            cx<A> t;
            t = scale(m.a, u0); t = cfma(m.q00, d0, t); t = cfma(m.q01, d1, t); chi[c] = t;
            t = scale(m.a, u1); t = cfma(m.q10, d0, t); t = cfma(m.q11, d1, t); chi[3 + c] = t;
            t = scale(m.a, d0); t = cfma_conj(m.q00, u0, t); t = cfma_conj(m.q10, u1, t); chi[6 + c] = t;
            t = scale(m.a, d1); t = cfma_conj(m.q01, u0, t); t = cfma_conj(m.q11, u1, t); chi[9 + c] = t;
        }
    }
}

// acc += M_d a + M_{-d} b for the pair of opposite directions d, -d, where
// a = W_d psi(x + d), b = W_{-d} psi(x - d) (colour products done) and
// M_{+-d} = lambda' +- G, G = [[0, rho Q], [rho Q^+, 0]]:
// acc += lambda' (a + b) + G (a - b)
template <typename A>
DEV_INLINE void bri_pair_acc(const BriDirA<A>& m, const cx<A>* av, const cx<A>* bv, cx<A>* acc)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<A> su0 = av[c] + bv[c], su1 = av[3 + c] + bv[3 + c];
        cx<A> sd0 = av[6 + c] + bv[6 + c], sd1 = av[9 + c] + bv[9 + c];
        cx<A> tu0 = av[c] - bv[c], tu1 = av[3 + c] - bv[3 + c];
        cx<A> td0 = av[6 + c] - bv[6 + c], td1 = av[9 + c] - bv[9 + c];
        cx<A> o;
        if constexpr (sizeof(A) == 4) {
            o = caxpy2(m.a, su0, acc[c]); o = cfma2(m.q00, td0, o); acc[c] = cfma2(m.q01, td1, o);
            o = caxpy2(m.a, su1, acc[3 + c]); o = cfma2(m.q10, td0, o); acc[3 + c] = cfma2(m.q11, td1, o);
            o = caxpy2(m.a, sd0, acc[6 + c]); o = cfma2_conj(m.q00, tu0, o); acc[6 + c] = cfma2_conj(m.q10, tu1, o);
            o = caxpy2(m.a, sd1, acc[9 + c]); o = cfma2_conj(m.q01, tu0, o); acc[9 + c] = cfma2_conj(m.q11, tu1, o);
        } else {
            o = acc[c] + scale(m.a, su0); o = cfma(m.q00, td0, o); acc[c] = cfma(m.q01, td1, o);
            o = acc[3 + c] + scale(m.a, su1); o = cfma(m.q10, td0, o); acc[3 + c] = cfma(m.q11, td1, o);
            o = acc[6 + c] + scale(m.a, sd0); o = cfma_conj(m.q00, tu0, o); acc[6 + c] = cfma_conj(m.q10, tu1, o);
            o = acc[9 + c] + scale(m.a, sd1); o = cfma_conj(m.q01, tu0, o); acc[9 + c] = cfma_conj(m.q11, tu1, o);
        }
    }
}

// out = (m0 + 15/8) psi + sum over the 40 pairs (d, -d) of the stored
// directions: the spin matrices of d and -d differ only in the sign of the
// rho part, so both colour products are formed first and one spin matrix
// application serves the pair.
// LF 0: 40 stored links, W_{-d}(x) = W_d(x - d)^+ read at the neighbour x - d;
// LF 1: all 80 stored at x, W_{-d}(x) in plane 40 + rep (local reads).
// T is the storage type of the links; TI, TO those of the input and output
// fields (the split inner solve reads 16-bit directions and writes FP32
// products, or the reverse), all with the same arithmetic type.
template <typename T, int R, bool DAG, int LF = 0, typename TI = T, typename TO = T>
DEV_INLINE void brillouin_site(const ApplyArgs& a, long s, int group, const BriDir* dirs)
{
    static_assert(std::is_same<typename Store<T>::A, typename Store<TI>::A>::value &&
                  std::is_same<typename Store<T>::A, typename Store<TO>::A>::value, "one arithmetic type");
    using A = typename Store<T>::A;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s, fwd, bwd, x);
    const int v0 = group * R;
    cx<A> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[r][i] = cx<A>{A(0), A(0)};
#pragma unroll 1
    for (int j = 0; j < 80; ++j) {
        const BriDir& D = dirs[j];
        if (D.neg) continue;   // the stored directions; -d is handled with d
        long np = s, nm = s;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            np += (D.d[mu] > 0) ? fwd[mu] : (D.d[mu] < 0 ? bwd[mu] : 0);
            nm += (D.d[mu] > 0) ? bwd[mu] : (D.d[mu] < 0 ? fwd[mu] : 0);
        }
        cx<A> Wp[9], Wm[9];
        load_link<T>(a.links, a.g.vol, D.rep, s, Wp);    // W_d(x)
        if constexpr (LF == 1) load_link<T>(a.links, a.g.vol, 40 + D.rep, s, Wm);   // W_{-d}(x)
        else load_link<T>(a.links, a.g.vol, D.rep, nm, Wm);   // W_{-d}(x) = W_d(x - d)^+
        const BriDirA<A> m = bri_coeffs<A, DAG>(D);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = min(v0 + r, a.Nv - 1);   // partial group: recompute, store guarded
            cx<A> p[12], av[12], bv[12];
            load_spinor<TI, 12>(a.in, a.g.vol, v, np, p);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) {
#pragma unroll
                for (int i = 0; i < 3; ++i) av[3 * sp + i] = cx<A>{A(0), A(0)};
                if constexpr (sizeof(A) == 4) mat_vec_acc2(Wp, p + 3 * sp, av + 3 * sp);
                else mat_vec_acc(Wp, p + 3 * sp, av + 3 * sp);
            }
            load_spinor<TI, 12>(a.in, a.g.vol, v, nm, p);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) {
#pragma unroll
                for (int i = 0; i < 3; ++i) bv[3 * sp + i] = cx<A>{A(0), A(0)};
                if constexpr (LF == 1) {
                    if constexpr (sizeof(A) == 4) mat_vec_acc2(Wm, p + 3 * sp, bv + 3 * sp);
                    else mat_vec_acc(Wm, p + 3 * sp, bv + 3 * sp);
                } else {
                    if constexpr (sizeof(A) == 4) mat_dag_vec_acc2(Wm, p + 3 * sp, bv + 3 * sp);
                    else mat_dag_vec_acc(Wm, p + 3 * sp, bv + 3 * sp);
                }
            }
            bri_pair_acc(m, av, bv, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = min(v0 + r, a.Nv - 1);
        const A dg = diag_of<A>(a, v);
        cx<A> p[12];
        load_spinor<TI, 12>(a.in, a.g.vol, v, s, p);
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            p[i].re = fma(dg, p[i].re, acc[r][i].re);
            p[i].im = fma(dg, p[i].im, acc[r][i].im);
        }
        if (v0 + r < a.Nv) store_spinor<TO, 12>(a.out, a.g.vol, v0 + r, s, p);
    }
}

}  // namespace dirac
