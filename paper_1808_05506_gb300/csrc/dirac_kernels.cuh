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

#include "dirac_common.cuh"

namespace dirac {

struct ApplyArgs {
    Geom g;
    int Nv;
    const void* in;       // internal spinor layout
    void* out;            // internal spinor layout
    const void* links;    // internal link layout (V_mu or the 40 stored W)
    double diag;          // (4 + m0) Wilson, m staggered, (m0 + 15/8) Brillouin
};

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

// one hop: acc_r += (1 + S gamma_MU) U psi_r(nbr),  U = V_MU(lsite) or its adjoint (BACK)
template <typename T, int R, int MU, int S, bool BACK>
DEV_INLINE void wilson_hop(const ApplyArgs& a, long nbr, long lsite, int v0,
                           cx<typename Store<T>::A> (&acc)[R][12])
{
    using A = typename Store<T>::A;
    cx<A> U[9];
    load_link<T>(a.links, a.g.vol, MU, lsite, U);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (v0 + r < a.Nv) {
            cx<A> p[12], h[6], w[6];
            load_spinor<T, 12>(a.in, a.g.vol, v0 + r, nbr, p);
            wilson_project<MU, S>(p, h);
            if constexpr (BACK) { mat_dag_vec(U, h, w); mat_dag_vec(U, h + 3, w + 3); }
            else { mat_vec(U, h, w); mat_vec(U, h + 3, w + 3); }
            wilson_reconstruct<MU, S>(w, acc[r]);
        }
    }
}

template <typename T, int R, bool DAG>
DEV_INLINE void wilson_site(const ApplyArgs& a, long s, int group)
{
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
    wilson_hop<T, R, 0, SF, false>(a, s + fwd[0], s, v0, acc);
    wilson_hop<T, R, 0, SB, true>(a, s + bwd[0], s + bwd[0], v0, acc);
    wilson_hop<T, R, 1, SF, false>(a, s + fwd[1], s, v0, acc);
    wilson_hop<T, R, 1, SB, true>(a, s + bwd[1], s + bwd[1], v0, acc);
    wilson_hop<T, R, 2, SF, false>(a, s + fwd[2], s, v0, acc);
    wilson_hop<T, R, 2, SB, true>(a, s + bwd[2], s + bwd[2], v0, acc);
    wilson_hop<T, R, 3, SF, false>(a, s + fwd[3], s, v0, acc);
    wilson_hop<T, R, 3, SB, true>(a, s + bwd[3], s + bwd[3], v0, acc);
    const A dg = (A)a.diag;
    const A mh = (A)(-0.5);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (v0 + r < a.Nv) {
            cx<A> p[12];
            load_spinor<T, 12>(a.in, a.g.vol, v0 + r, s, p);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                cx<A> o;
                o.re = fma(mh, acc[r][i].re, dg * p[i].re);
                o.im = fma(mh, acc[r][i].im, dg * p[i].im);
                p[i] = o;
            }
            store_spinor<T, 12>(a.out, a.g.vol, v0 + r, s, p);
        }
    }
}

// ---------------------------------------------------------------- staggered
template <typename T, int R, bool DAG>
DEV_INLINE void staggered_site(const ApplyArgs& a, long s, int group)
{
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
        load_link<T>(a.links, a.g.vol, mu, s, Uf);
        load_link<T>(a.links, a.g.vol, mu, s + bwd[mu], Ub);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (v0 + r < a.Nv) {
                cx<A> pf[3], pb[3], w[3] = {}, wb[3] = {};
                load_spinor<T, 3>(a.in, a.g.vol, v0 + r, s + fwd[mu], pf);
                load_spinor<T, 3>(a.in, a.g.vol, v0 + r, s + bwd[mu], pb);
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
    }
    const A dg = (A)a.diag;
    const A hf = DAG ? A(-0.5) : A(0.5);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (v0 + r < a.Nv) {
            cx<A> p[3];
            load_spinor<T, 3>(a.in, a.g.vol, v0 + r, s, p);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<A> o;
                o.re = fma(hf, acc[r][c].re, dg * p[c].re);
                o.im = fma(hf, acc[r][c].im, dg * p[c].im);
                p[c] = o;
            }
            store_spinor<T, 3>(a.out, a.g.vol, v0 + r, s, p);
        }
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
};

template <typename A> struct BriDirA { A a; cx<A> q00, q01, q10, q11; };

template <typename A, bool DAG>
HD BriDirA<A> bri_coeffs(const BriDir& D)
{
    BriDirA<A> c;
    const A sg = DAG ? A(-1) : A(1);
    c.a = (A)D.a;
    c.q00 = {sg * (A)D.q[0], sg * (A)D.q[1]};
    c.q01 = {sg * (A)D.q[2], sg * (A)D.q[3]};
    c.q10 = {sg * (A)D.q[4], sg * (A)D.q[5]};
    c.q11 = {sg * (A)D.q[6], sg * (A)D.q[7]};
    return c;
}

// chi = M psi
template <typename A>
HD void bri_spin(const BriDirA<A>& m, const cx<A>* p, cx<A>* chi)
{
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

template <typename T, int R, bool DAG>
DEV_INLINE void brillouin_site(const ApplyArgs& a, long s, int group, const BriDir* dirs)
{
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
        const BriDir D = dirs[j];
        long nbr = s;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) nbr += (D.d[mu] > 0) ? fwd[mu] : (D.d[mu] < 0 ? bwd[mu] : 0);
        cx<A> W[9];
        load_link<T>(a.links, a.g.vol, D.rep, D.neg ? nbr : s, W);
        const BriDirA<A> m = bri_coeffs<A, DAG>(D);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (v0 + r < a.Nv) {
                cx<A> p[12], chi[12];
                load_spinor<T, 12>(a.in, a.g.vol, v0 + r, nbr, p);
                bri_spin(m, p, chi);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    if (D.neg) mat_dag_vec_acc(W, chi + 3 * sp, acc[r] + 3 * sp);
                    else mat_vec_acc(W, chi + 3 * sp, acc[r] + 3 * sp);
                }
            }
        }
    }
    const A dg = (A)a.diag;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (v0 + r < a.Nv) {
            cx<A> p[12];
            load_spinor<T, 12>(a.in, a.g.vol, v0 + r, s, p);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                p[i].re = fma(dg, p[i].re, acc[r][i].re);
                p[i].im = fma(dg, p[i].im, acc[r][i].im);
            }
            store_spinor<T, 12>(a.out, a.g.vol, v0 + r, s, p);
        }
    }
}

}  // namespace dirac
