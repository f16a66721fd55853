// Even-odd (red-black) sweeps of the Wilson and staggered operators, for the
// Schur-complement inner solver.  Sec. 4 names the even-odd decomposition as
// the next step of tuning the Wilson kernel; the same split holds for the
// staggered operator of Sec. 3.
//
// With every extent even the hopping part H of D = a + H (a = 4 + m0 for
// Wilson, a = m for staggered) only connects sites of opposite parity
// (x + y + z + t mod 2), so on (even, odd) sites
//     D = [[a, H_eo], [H_oe, a]]
// and D e = r splits into the Schur complement on the odd sites,
//     S e_o = r_o - H_oe r_e / a,      S = a - H_oe H_eo / a,
// followed by e_e = (r_e - H_eo e_o) / a.  D^+ has the same structure with
// H^+ (Wilson: gamma5 H gamma5; staggered: -H), and S^+ = a - H^+_oe H^+_eo / a.
//
// One sweep here computes, on the sites of one parity,
//     out = alpha_v in2 + beta_v (H in)      (or H^+ in)
// per right-hand side v, with `in` a field of the other parity and `in2` one
// of the same parity (not read when null).
//
// Half fields: the sites of one parity in the internal blocked layout of a
// lattice of vol / 2 sites, with half-site index h = s / 2 (s the site index
// x + Nx (y + Ny (z + Nz t)); Nx even, so s and s + 1 share h and have
// opposite parities).  The links stay in the whole-lattice layout.
#pragma once

#include "dirac_internal.h"

namespace dirac {

struct EoArgs {
    Geom g;            // the lattice (every extent even)
    Geom gh;           // the half lattice: extents Nx / 2, Ny, Nz, Nt (h = its site index)
    long vh;           // sites of one parity: vol / 2
    int Nv;
    int par;           // parity of the output sites
    const void* in;    // half field of parity 1 - par
    const void* in2;   // half field of parity par, or null (alpha not used)
    void* out;         // half field of parity par
    const void* links; // links V_mu, whole-lattice internal layout
    const void* coef;  // arithmetic type: alpha[Nv] then beta[Nv]
    int tc;            // site order of the half lattice (site_of)
    FDiv fdc, fdt;
    // optional |out_v|^2 (of the stored values), fused into the sweep: one FP64
    // partial per warp and column, npart[v * nwarp + warp] (null: not formed);
    // nwarp = eo_norm_slots(vh, block), set by the launcher
    double* npart = nullptr;
    long nwarp = 0;
};

// partials per column of the fused norm of a sweep with `block` half sites per block
inline long eo_norm_slots(long vh, int block) { return ((vh + block - 1) / block) * (block / 32); }

// a value as the storage type T holds it (16-bit types round)
template <typename T> DEV_INLINE cx<typename Store<T>::A> stored_value(cx<typename Store<T>::A> c)
{
    if constexpr (sizeof(T) == 2) return unpack2(pack2(c, (T*)nullptr), (T*)nullptr);
    else return c;
}

// site of parity a.par with half-site index h
HD long eo_site(const EoArgs& a, long h)
{
    const uint32_t rest = fdiv(a.gh.fd[0], (uint32_t)h);   // y + Ny (z + Nz t)
    const uint32_t q1 = fdiv(a.g.fd[1], rest);
    const uint32_t q2 = fdiv(a.g.fd[2], q1);
    const int yzt = (int)(rest - q1 * (uint32_t)a.g.L[1]) + (int)(q1 - q2 * (uint32_t)a.g.L[2]) + (int)q2;
    return 2 * h + ((a.par + yzt) & 1);
}

// Storage types: TL links, TI the input field `in`, TI2 the field `in2`, TO
// the output; one arithmetic type for all (Store<TI>::A: FP64 for FP64
// fields, else FP32).  The uniform sweeps take one type for all four; the
// split inner solve mixes FP32 and 16-bit fields.

// acc_r += (1 + S gamma_MU) U psi_r(h_nbr), U = V_MU(lsite) or its adjoint (BACK)
template <typename TL, typename TI, int R, int MU, int S, bool BACK>
DEV_INLINE void eo_wilson_hop(const EoArgs& a, long hn, long lsite, int v0, cx<typename Store<TI>::A> (&acc)[R][12])
{
    using A = typename Store<TI>::A;
    cx<A> U[9];
    load_link<TL>(a.links, a.g.vol, MU, lsite, U);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cx<A> p[12], h[6], w[6];
        load_spinor<TI, 12>(a.in, a.vh, v0 + r, hn, p);
        wilson_project<MU, S>(p, h);
        if constexpr (BACK) { mat_dag_vec(U, h, w); mat_dag_vec(U, h + 3, w + 3); }
        else { mat_vec(U, h, w); mat_vec(U, h + 3, w + 3); }
        wilson_reconstruct<MU, S>(w, acc[r]);
    }
}

// out = alpha in2 + beta (H in) at one site; H = -1/2 sum_mu [(1 - gamma_mu)
// V_mu(x) psi(x + mu) + (1 + gamma_mu) V_mu(x - mu)^+ psi(x - mu)], the
// adjoint swapping the two projectors.  R divides Nv.
// q[r] = |out|^2 at this site of column v0 + r (when a.npart is set)
template <typename TL, typename TI, typename TI2, typename TO, int R, bool DAG>
DEV_INLINE void wilson_eo_site(const EoArgs& a, long h, int group, typename Store<TI>::A (&q)[R])
{
    using A = typename Store<TI>::A;
    const long s = eo_site(a, h);
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(a.g, s, fwd, bwd, x);
    const int v0 = group * R;
    cx<A> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[r][i] = cx<A>{A(0), A(0)};
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    eo_wilson_hop<TL, TI, R, 0, SF, false>(a, (s + fwd[0]) >> 1, s, v0, acc);
    eo_wilson_hop<TL, TI, R, 0, SB, true>(a, (s + bwd[0]) >> 1, s + bwd[0], v0, acc);
    eo_wilson_hop<TL, TI, R, 1, SF, false>(a, (s + fwd[1]) >> 1, s, v0, acc);
    eo_wilson_hop<TL, TI, R, 1, SB, true>(a, (s + bwd[1]) >> 1, s + bwd[1], v0, acc);
    eo_wilson_hop<TL, TI, R, 2, SF, false>(a, (s + fwd[2]) >> 1, s, v0, acc);
    eo_wilson_hop<TL, TI, R, 2, SB, true>(a, (s + bwd[2]) >> 1, s + bwd[2], v0, acc);
    eo_wilson_hop<TL, TI, R, 3, SF, false>(a, (s + fwd[3]) >> 1, s, v0, acc);
    eo_wilson_hop<TL, TI, R, 3, SB, true>(a, (s + bwd[3]) >> 1, s + bwd[3], v0, acc);
    const A* cf = static_cast<const A*>(a.coef);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + r;
        const A al = cf[v], be = A(-0.5) * cf[a.Nv + v];
        cx<A> o[12];
        if (a.in2) {
            load_spinor<TI2, 12>(a.in2, a.vh, v, h, o);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                o[i].re = fma(be, acc[r][i].re, al * o[i].re);
                o[i].im = fma(be, acc[r][i].im, al * o[i].im);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 12; ++i) o[i] = cx<A>{be * acc[r][i].re, be * acc[r][i].im};
        }
        store_spinor<TO, 12>(a.out, a.vh, v, h, o);
        if (a.npart) {
            A n2 = A(0);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const cx<A> c = stored_value<TO>(o[i]);
                n2 = fma(c.re, c.re, fma(c.im, c.im, n2));
            }
            q[r] = n2;
        }
    }
}

// out = alpha in2 + beta (H in) at one site; H = 1/2 sum_mu eta_mu(x)
// [V_mu(x) psi(x + mu) - V_mu(x - mu)^+ psi(x - mu)], H^+ = -H.  R divides Nv.
template <typename TL, typename TI, typename TI2, typename TO, int R, bool DAG>
DEV_INLINE void staggered_eo_site(const EoArgs& a, long h, int group, typename Store<TI>::A (&q)[R])
{
    using A = typename Store<TI>::A;
    const long s = eo_site(a, h);
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
        load_link<TL>(a.links, a.g.vol, mu, s, Uf);
        load_link<TL>(a.links, a.g.vol, mu, s + bwd[mu], Ub);
        const long hf = (s + fwd[mu]) >> 1, hb = (s + bwd[mu]) >> 1;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cx<A> pf[3], pb[3], w[3] = {}, wb[3] = {};
            load_spinor<TI, 3>(a.in, a.vh, v0 + r, hf, pf);
            load_spinor<TI, 3>(a.in, a.vh, v0 + r, hb, pb);
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
    const A* cf = static_cast<const A*>(a.coef);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + r;
        const A al = cf[v], be = (DAG ? A(-0.5) : A(0.5)) * cf[a.Nv + v];
        cx<A> o[3];
        if (a.in2) {
            load_spinor<TI2, 3>(a.in2, a.vh, v, h, o);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[c].re = fma(be, acc[r][c].re, al * o[c].re);
                o[c].im = fma(be, acc[r][c].im, al * o[c].im);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = cx<A>{be * acc[r][c].re, be * acc[r][c].im};
        }
        store_spinor<TO, 3>(a.out, a.vh, v, h, o);
        if (a.npart) {
            A n2 = A(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const cx<A> z = stored_value<TO>(o[c]);
                n2 = fma(z.re, z.re, fma(z.im, z.im, n2));
            }
            q[r] = n2;
        }
    }
}

// blockDim = (half sites, gy groups); block b covers a run of half sites (in
// the site order of the half lattice) and gy groups of R right-hand sides

// With a.npart the norms of the outputs are summed per warp (the 32 lanes of
// a warp share threadIdx.y, since blockDim.x >= 32): each site's |out_v|^2 in
// the arithmetic type (at most 24 squares), the warp's sum in FP64, one
// partial per warp and column; a fixed-order second pass adds the partials.
template <int OP, typename TL, typename TI, typename TI2, typename TO, int R, bool DAG>
__global__ void __launch_bounds__(192, 2) k_eo(EoArgs a, int ngroups, int gy)
{
    using A = typename Store<TI>::A;
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    if (group >= ngroups) return;   // a whole warp
    const long p = (b / nchunks) * blockDim.x + threadIdx.x;
    A q[R];
#pragma unroll
    for (int r = 0; r < R; ++r) q[r] = A(0);
    if (p < a.vh) {
        const long h = site_of(a.gh, p, a.tc, a.g.L[3], a.fdc, a.fdt);
        if constexpr (OP == OP_WILSON) wilson_eo_site<TL, TI, TI2, TO, R, DAG>(a, h, group, q);
        else staggered_eo_site<TL, TI, TI2, TO, R, DAG>(a, h, group, q);
    }
    if (a.npart) {
        const long wi = (b / nchunks) * (blockDim.x >> 5) + (threadIdx.x >> 5);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double d = (double)q[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if ((threadIdx.x & 31) == 0) a.npart[(size_t)(group * R + r) * a.nwarp + wi] = d;
        }
    }
}

// block: half sites per block (32, 64 or 128), times gy = min(192 / block,
// groups) right-hand-side groups
template <int OP, typename TL, typename TI, typename TI2, typename TO, int R, bool DAG>
cudaError_t eo_go_typed(const EoArgs& a, int block, cudaStream_t st)
{
    if (block != 32 && block != 64 && block != 128) return cudaErrorInvalidValue;
    const int ngroups = a.Nv / R;
    const int gy = groups_per_block(block, ngroups);
    const long nb = ((a.vh + block - 1) / block) * (long)((ngroups + gy - 1) / gy);
    EoArgs b = a;
    b.nwarp = eo_norm_slots(a.vh, block);
    k_eo<OP, TL, TI, TI2, TO, R, DAG><<<(unsigned)nb, dim3(block, gy), 0, st>>>(b, ngroups, gy);
    return cudaGetLastError();
}

// the uniform sweep: every field and the links in storage type T
template <int OP, typename T, int R>
cudaError_t eo_go(bool dag, const EoArgs& a, int block, cudaStream_t st)
{
    return dag ? eo_go_typed<OP, T, T, T, T, R, true>(a, block, st) : eo_go_typed<OP, T, T, T, T, R, false>(a, block, st);
}

// right-hand sides per thread R of the even-odd sweeps that are built: R
// divides Nv and fits the registers without spilling (Wilson 1, 2; staggered
// 1, 2, 4; FP64: Wilson 1, staggered 1, 2)
inline bool eo_rhs_supported(int op, int prec, int Nv, int R)
{
    if (R < 1 || Nv % R != 0) return false;
    if (op == OP_WILSON) return R == 1 || (R == 2 && prec != P_F64);
    if (op == OP_STAGGERED) return R == 1 || R == 2 || (R == 4 && prec != P_F64);
    return false;
}

// launch shape of the even-odd sweeps before tuning: the largest R built, 64
// half sites per block, t-chunks of up to 8 slices
inline LaunchCfg eo_default_config(int op, int prec, int Nv, int Nt)
{
    int R = 4;
    while (R > 1 && !eo_rhs_supported(op, prec, Nv, R)) R /= 2;
    return LaunchCfg{R, 64, 0, Nt < 8 ? Nt : 8};
}

}  // namespace dirac

namespace dirac {

// the sweep of dirac_eo.cuh with cfg.R right-hand sides per thread and
// cfg.block half sites per block (the site order is a.tc)
cudaError_t launch_eo_wilson(int prec, bool dag, const EoArgs& a, int R, int block, cudaStream_t st);
cudaError_t launch_eo_staggered(int prec, bool dag, const EoArgs& a, int R, int block, cudaStream_t st);
cudaError_t launch_eo(int op, int prec, bool dag, const EoArgs& a, LaunchCfg cfg, cudaStream_t st);

// The sweeps of the split inner solve (Wilson, 16-bit handle prec16): FP32
// links, solution, residual and operator products, 16-bit search directions.
//   EO_SPLIT_HP:  tmp(F32) = H_eo p(16)                      (no adjoint)
//   EO_SPLIT_SP:  t(F32) = a p(16) - H_oe tmp(F32) / a       (no adjoint)
//   EO_SPLIT_HR:  tmp2(16) = H^+_eo r(F32)                   (adjoint)
//   EO_SPLIT_SR:  s(16) = a r(F32) - H^+_oe tmp2(16) / a     (adjoint)
enum { EO_SPLIT_HP = 0, EO_SPLIT_SP = 1, EO_SPLIT_HR = 2, EO_SPLIT_SR = 3 };
cudaError_t launch_eo_wilson_split(int prec16, int kind, const EoArgs& a, LaunchCfg cfg, cudaStream_t st);

// arguments of a sweep over the sites of parity par (the lattice extents all
// even); tc: site order of the half lattice (0 lexicographic, else t-chunks)
EoArgs make_eo_args(const Geom& g, int Nv, int par, const void* in, const void* in2, void* out, const void* links,
                    const void* coef, int tc);

// (re, ro) = scale_v r64: a whole-lattice FP64 field split into its even and
// odd half fields in storage precision prec
cudaError_t eo_split(int prec, int nsc, const Geom& g, int Nv, const void* r64, const double* scale, void* re,
                     void* ro, cudaStream_t st);
// x64 += coef_v (ee, eo): the half fields of both parities added to a
// whole-lattice FP64 field
cudaError_t eo_axpy_to64(int prec, int nsc, const Geom& g, int Nv, const double* coef, const void* ee,
                         const void* eo, void* x64, cudaStream_t st);

// complex numbers per right-hand side of a half field (padded to whole blocks of 32 half sites)
inline size_t eo_half_n(int op, long vol) { return (size_t)nsc_of(op) * nblk_of((size_t)(vol / 2)) * 32; }

}  // namespace dirac
