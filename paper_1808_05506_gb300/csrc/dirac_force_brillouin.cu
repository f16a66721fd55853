// Link gradient of L = Re <g, D_B psi> for the Brillouin operator (Sec. 5,
// Eqs. def_bril, def_der, def_lap at c_SW = 0), PyTorch's convention
// F = dL/dRe V + i dL/dIm V.  The off-axis transporters W_dir are not kept
// between the forward and the backward pass: they are rebuilt here in FP64
// from V by the recursion of Tab. tab:off-axis (every ordering of the k hops,
// weight 1/k!, split by the first hop):
//   W_dir(x) = (1/k) sum_{hops a of dir} H_a(x) W_{dir-a}(x+a),
//   H_{+mu}(x) = V_mu(x), H_{-mu}(x) = V_mu(x-mu)^+.
// Steps (all gathers, one write per output element, no atomics):
//   1. G_dir(y) = dL/dW_dir(y) = sum_{v,s} g_v(y)_s (M_dir psi_v(y+dir))_s^+
//      for the 80 directions, M_dir = rho_k (dir . gamma) - lambda_k / 2;
//   (every step in FP64 arithmetic, whatever the storage precision)
//   2. for k = 4, 3, 2 the (k-1)-hop gradients collect what the k-hop
//      directions pass down: G_{d'}(y) += (1/k) H_a(y-a)^+ G_{d'+a}(y-a) over
//      the hops a on the axes d' does not use;
//   3. F_mu(y) = sum_{dir with +mu} (1/k) G_dir(y) W_{dir-mu}(y+mu)^+
//             + sum_{dir with -mu} (1/k) W_{dir+mu}(y) G_dir(y+mu)^+
//      (W_0 = 1: the one-hop directions).
#include "dirac_handle.h"
#include "dirac_kernels.cuh"

using namespace dirac;

namespace dirac {
namespace {

__device__ __forceinline__ void dir_of(int c, int d[4])
{
    d[0] = c % 3 - 1;
    d[1] = (c / 3) % 3 - 1;
    d[2] = (c / 9) % 3 - 1;
    d[3] = (c / 27) % 3 - 1;
}
__device__ __forceinline__ int code_of(const int d[4])
{
    return (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1) + 27 * (d[3] + 1);
}

// the spin matrix of direction d: [[a, rho Q], [rho Q^+, a]], a = -lambda_k / 2,
// Q = sum_mu d_mu B_mu (B_k = -i sigma_k, B_4 = 1); rho_k, lambda_k of Sec. 5
template <typename A>
__device__ __forceinline__ BriDirA<A> coeffs_of(const int d[4])
{
    const int k = abs(d[0]) + abs(d[1]) + abs(d[2]) + abs(d[3]);
    const double rho[5] = {0.0, 64.0 / 432.0, 16.0 / 432.0, 4.0 / 432.0, 1.0 / 432.0};
    const double lam[5] = {-240.0 / 64.0, 8.0 / 64.0, 4.0 / 64.0, 2.0 / 64.0, 1.0 / 64.0};
    const double r = rho[k];
    const double dx = d[0], dy = d[1], dz = d[2], dt = d[3];
    BriDirA<A> m;
    m.a = (A)(-0.5 * lam[k]);
    m.q00 = {(A)(r * dt), (A)(-r * dz)};
    m.q01 = {(A)(-r * dy), (A)(-r * dx)};
    m.q10 = {(A)(r * dy), (A)(-r * dx)};
    m.q11 = {(A)(r * dt), (A)(r * dz)};
    return m;
}

__device__ __forceinline__ cx<double> ld64(const double2* p, size_t i)
{
    const double2 v = p[i];
    return {v.x, v.y};
}

// C = A B, A^+ B, A B^+ (3x3)
__device__ __forceinline__ void mm(const cx<double>* Am, bool adag, const cx<double>* Bm, bool bdag, cx<double>* C)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cx<double> t{0.0, 0.0};
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const cx<double> x = adag ? conj(Am[3 * m + a]) : Am[3 * a + m];
                const cx<double> y = bdag ? conj(Bm[3 * b + m]) : Bm[3 * m + b];
                t = cfma(x, y, t);
            }
            C[3 * a + b] = t;
        }
}

// step 1: one thread per (site, direction j = 0..79).  The arithmetic is FP64
// for every storage precision: FP32 and 16-bit values are exact in FP64, so
// G is the FP64 gradient of the stored psi and g (the steps below are FP64
// as well), and F is rounded once, at its store.
template <typename T>
__global__ void __launch_bounds__(128) k_bri_gradW(Geom g, int Nv, const void* psi, const void* gv, double2* G81)
{
    using A = typename Store<T>::A;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, j), site fastest
    if (i >= 80 * g.vol) return;
    const long y = i % g.vol;
    const int j = (int)(i / g.vol);
    const int c = j < 40 ? j : j + 1;   // skip the centre code 40
    int d[4];
    dir_of(c, d);
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(g, y, fwd, bwd, x);
    long nb = y;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) nb += d[mu] > 0 ? fwd[mu] : (d[mu] < 0 ? bwd[mu] : 0);
    const BriDirA<double> m = coeffs_of<double>(d);
    cx<double> acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = cx<double>{0.0, 0.0};
    for (int v = 0; v < Nv; ++v) {
        cx<A> ps[12], gs[12];
        load_spinor<T, 12>(psi, g.vol, v, nb, ps);
        load_spinor<T, 12>(gv, g.vol, v, y, gs);
        cx<double> p[12], chi[12], gg[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            p[k] = cx<double>{(double)ps[k].re, (double)ps[k].im};
            gg[k] = cx<double>{(double)gs[k].re, (double)gs[k].im};
        }
        bri_spin(m, p, chi);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) acc[3 * a + b] = cfma_conj(chi[3 * s + b], gg[3 * s + a], acc[3 * a + b]);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) G81[((size_t)c * 9 + e) * g.vol + y] = make_double2(acc[e].re, acc[e].im);
}

struct Codes {
    int n;
    short c[32];
};

// step 2 for level k: one thread per (site, direction of k-1 hops)
__global__ void __launch_bounds__(128) k_bri_back(Geom g, Codes L, int k, const double2* __restrict__ V64,
                                                  double2* G81)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)L.n * g.vol) return;
    const long y = i % g.vol;
    const int c = L.c[i / g.vol];
    int d[4];
    dir_of(c, d);
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(g, y, fwd, bwd, x);
    cx<double> Gs[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) Gs[e] = ld64(G81, ((size_t)c * 9 + e) * g.vol + y);
    const double inv = 1.0 / k;
    for (int mu = 0; mu < 4; ++mu) {
        if (d[mu] != 0) continue;
        cx<double> U[9], Gu[9], T9[9];
        // a = +mu: (1/k) V_mu(y-mu)^+ G_{d+mu}(y-mu)
        int dp[4] = {d[0], d[1], d[2], d[3]};
        dp[mu] = 1;
        const long sm = y + bwd[mu];
        const int cp = code_of(dp);
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            U[e] = ld64(V64, ((size_t)mu * 9 + e) * g.vol + sm);
            Gu[e] = ld64(G81, ((size_t)cp * 9 + e) * g.vol + sm);
        }
        mm(U, true, Gu, false, T9);
#pragma unroll
        for (int e = 0; e < 9; ++e) Gs[e] = Gs[e] + scale(inv, T9[e]);
        // a = -mu: (1/k) V_mu(y) G_{d-mu}(y+mu)
        dp[mu] = -1;
        const long sp = y + fwd[mu];
        const int cm = code_of(dp);
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            U[e] = ld64(V64, ((size_t)mu * 9 + e) * g.vol + y);
            Gu[e] = ld64(G81, ((size_t)cm * 9 + e) * g.vol + sp);
        }
        mm(U, false, Gu, false, T9);
#pragma unroll
        for (int e = 0; e < 9; ++e) Gs[e] = Gs[e] + scale(inv, T9[e]);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) G81[((size_t)c * 9 + e) * g.vol + y] = make_double2(Gs[e].re, Gs[e].im);
}

// step 3: one thread per (site, mu); F canonical [site][mu][a][b] in the type O
template <typename O>
__global__ void __launch_bounds__(128) k_bri_dV(Geom g, const double2* __restrict__ G81,
                                                const double2* __restrict__ W81, O* F)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, mu), site fastest
    if (i >= 4 * g.vol) return;
    const long y = i % g.vol;
    const int mu = (int)(i / g.vol);
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(g, y, fwd, bwd, x);
    const long yp = y + fwd[mu];
    cx<double> acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = cx<double>{0.0, 0.0};
    for (int c = 0; c < 81; ++c) {
        int d[4];
        dir_of(c, d);
        if (d[mu] == 0) continue;
        const int k = abs(d[0]) + abs(d[1]) + abs(d[2]) + abs(d[3]);
        const double inv = 1.0 / k;
        int r[4] = {d[0], d[1], d[2], d[3]};
        r[mu] = 0;
        const int cr = code_of(r);
        cx<double> Gm[9], Wr[9], T9[9];
        if (d[mu] > 0) {
            // (1/k) G_dir(y) W_{dir-mu}(y+mu)^+
#pragma unroll
            for (int e = 0; e < 9; ++e) Gm[e] = ld64(G81, ((size_t)c * 9 + e) * g.vol + y);
            if (k == 1) {
#pragma unroll
                for (int e = 0; e < 9; ++e) T9[e] = Gm[e];
            } else {
#pragma unroll
                for (int e = 0; e < 9; ++e) Wr[e] = ld64(W81, ((size_t)cr * 9 + e) * g.vol + yp);
                mm(Gm, false, Wr, true, T9);
            }
        } else {
            // (1/k) W_{dir+mu}(y) G_dir(y+mu)^+
#pragma unroll
            for (int e = 0; e < 9; ++e) Gm[e] = ld64(G81, ((size_t)c * 9 + e) * g.vol + yp);
            if (k == 1) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) T9[3 * a + b] = conj(Gm[3 * b + a]);
            } else {
#pragma unroll
                for (int e = 0; e < 9; ++e) Wr[e] = ld64(W81, ((size_t)cr * 9 + e) * g.vol + y);
                mm(Wr, false, Gm, true, T9);
            }
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) acc[e] = acc[e] + scale(inv, T9[e]);
    }
    O* out = F + ((size_t)y * 4 + mu) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        O o;
        o.x = acc[e].re;
        o.y = acc[e].im;
        out[e] = o;
    }
}

template <typename T>
cudaError_t gradW_T(const Geom& g, int Nv, const void* psi, const void* gv, double2* G81, cudaStream_t st)
{
    const long n = 80 * g.vol;
    k_bri_gradW<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, Nv, psi, gv, G81);
    return cudaGetLastError();
}

}   // namespace

cudaError_t launch_force_brillouin(int prec, const Geom& g, int Nv, const void* psi, const void* gv,
                                   const void* V64, void* W81, void* G81, void* F, cudaStream_t st)
{
    cudaError_t e = launch_build_W81(g, V64, W81, st);
    if (e != cudaSuccess) return e;
    double2* G = static_cast<double2*>(G81);
    switch (prec) {
    case P_F64: e = gradW_T<double>(g, Nv, psi, gv, G, st); break;
    case P_F32: e = gradW_T<float>(g, Nv, psi, gv, G, st); break;
    case P_BF16: e = gradW_T<__nv_bfloat16>(g, Nv, psi, gv, G, st); break;
    case P_F16: e = gradW_T<__half>(g, Nv, psi, gv, G, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    for (int k = 4; k >= 2; --k) {
        Codes L;
        L.n = 0;
        for (int c = 0; c < 81; ++c) {
            const int d0 = c % 3 - 1, d1 = (c / 3) % 3 - 1, d2 = (c / 9) % 3 - 1, d3 = (c / 27) % 3 - 1;
            if ((d0 != 0) + (d1 != 0) + (d2 != 0) + (d3 != 0) == k - 1) L.c[L.n++] = (short)c;
        }
        const long n = (long)L.n * g.vol;
        k_bri_back<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, L, k, static_cast<const double2*>(V64), G);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const unsigned nb = (unsigned)((4 * g.vol + 127) / 128);
    if (prec == P_F64)
        k_bri_dV<double2><<<nb, 128, 0, st>>>(g, G, static_cast<const double2*>(W81), static_cast<double2*>(F));
    else
        k_bri_dV<float2><<<nb, 128, 0, st>>>(g, G, static_cast<const double2*>(W81), static_cast<float2*>(F));
    return cudaGetLastError();
}

}  // namespace dirac
