// Vector kernels of the solvers on internal-layout fields.
//
// Every field is seen as Nv contiguous segments (one per right-hand side) of
// n = NSC * vol complex numbers of its storage type, which holds for all
// internal layouts because the right-hand-side index is the slowest one.
// Arithmetic is FP32 for FP32/BF16/FP16 storage and FP64 for FP64 storage;
// every norm and dot product is accumulated in FP64: per-thread sums, warp
// shuffles, one partial per block, then a second kernel that adds the
// partials of each right-hand side in a fixed order (deterministic).  With
// FP32 arithmetic a thread first sums KF consecutive terms of its stride in
// FP32 and adds that sum to its FP64 accumulator (FP64 runs at a small
// fraction of the FP32 rate on this GPU, and one FP64 operation per term
// made the norms FP64-bound); each such FP32 sum of KF terms has a relative
// error below KF * 2^-24, which does not grow with the field size.
#include "dirac_blas.h"

namespace dirac {

constexpr int BT = 256;   // threads per block of the vector kernels

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block sum of v written to part[v_index * nblk + blockIdx.x]
__device__ __forceinline__ void block_partial(double v, double* part, size_t slot)
{
    __shared__ double sh[BT / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (BT / 32) ? sh[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) part[slot] = v;
    }
}

__global__ void k_reduce_partials(const double* __restrict__ part, int nblk, double* out, int accumulate)
{
    const int v = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += BT) s += part[(size_t)v * nblk + i];
    __shared__ double sh[BT / 32];
    s = warp_sum(s);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = s;
    __syncthreads();
    if (w == 0) {
        s = lane < (BT / 32) ? sh[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) out[v] = accumulate ? out[v] + s : s;
    }
}

int blas_blocks(size_t n)
{
    size_t b = (n + (size_t)BT * 4 - 1) / ((size_t)BT * 4);
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

size_t blas_partials(size_t n, int Nv) { return (size_t)blas_blocks(n) * Nv; }

template <typename A> __device__ __forceinline__ double norm2c(cx<A> c)
{
    return (double)c.re * (double)c.re + (double)c.im * (double)c.im;
}

constexpr int KF = 16;   // terms per FP32 partial sum

// FP64 accumulator fed by FP32 partial sums of KF terms (FP32 arithmetic), or
// plain FP64 (FP64 arithmetic)
template <typename A> struct Acc {
    double s = 0.0;
    A f = A(0);
    int c = 0;
    __device__ __forceinline__ void add(A v)
    {
        if constexpr (sizeof(A) == 8) {
            s += v;
        } else {
            f += v;
            if (++c == KF) {
                s += (double)f;
                f = A(0);
                c = 0;
            }
        }
    }
    __device__ __forceinline__ double total() const { return sizeof(A) == 8 ? s : s + (double)f; }
};

// ---------------------------------------------------------------- norms
template <typename T>
__global__ void k_norm2(size_t n, const void* __restrict__ x, double* part)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * n;
    Acc<A> s;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) {
        const cx<A> c = ld_one<T>(x, base + i);
        s.add(fma(c.re, c.re, c.im * c.im));
    }
    block_partial(s.total(), part, (size_t)v * gridDim.x + blockIdx.x);
}

// re <x, y> and im <x, y> = sum conj(x) y
template <typename T>
__global__ void k_dot(size_t n, const void* __restrict__ x, const void* __restrict__ y, double* part_re,
                      double* part_im)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * n;
    Acc<A> sr, si;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) {
        const cx<A> a = ld_one<T>(x, base + i);
        const cx<A> b = ld_one<T>(y, base + i);
        sr.add(fma(a.re, b.re, a.im * b.im));
        si.add(fma(a.re, b.im, -(a.im * b.re)));
    }
    block_partial(sr.total(), part_re, (size_t)v * gridDim.x + blockIdx.x);
    __syncthreads();
    block_partial(si.total(), part_im, (size_t)v * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------- CGLS steps
// e += alpha_v p ;  r -= alpha_v t ;  partial |r|^2
template <typename T>
__global__ void k_cgls_step(size_t n, const double* __restrict__ alpha, void* e, const void* __restrict__ p,
                            void* r, const void* __restrict__ t, double* part)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * n;
    const A a = (A)alpha[v];
    Acc<A> s;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) {
        cx<A> ev = ld_one<T>(e, base + i), pv = ld_one<T>(p, base + i);
        cx<A> rv = ld_one<T>(r, base + i), tv = ld_one<T>(t, base + i);
        ev.re = fma(a, pv.re, ev.re);
        ev.im = fma(a, pv.im, ev.im);
        rv.re = fma(-a, tv.re, rv.re);
        rv.im = fma(-a, tv.im, rv.im);
        st_one<T>(e, base + i, ev);
        st_one<T>(r, base + i, rv);
        s.add(fma(rv.re, rv.re, rv.im * rv.im));
    }
    block_partial(s.total(), part, (size_t)v * gridDim.x + blockIdx.x);
}

// p = s + beta_v p
template <typename T>
__global__ void k_xpay(size_t n, const void* __restrict__ s, const double* __restrict__ beta, void* p)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * n;
    const A b = (A)beta[v];
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) {
        cx<A> sv = ld_one<T>(s, base + i), pv = ld_one<T>(p, base + i);
        pv.re = fma(b, pv.re, sv.re);
        pv.im = fma(b, pv.im, sv.im);
        st_one<T>(p, base + i, pv);
    }
}

// ---------------------------------------------------------------- 16-byte forms
// The same three kernels on 16-byte elements (Store<T>::CPV complex numbers
// each), for segments whose length n is a multiple of CPV; m = n / CPV.
template <typename T>
__global__ void k_norm2_v(size_t m, const void* __restrict__ x, double* part)
{
    using A = typename Store<T>::A;
    constexpr int C = Store<T>::CPV;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * m;
    Acc<A> s;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < m; i += (size_t)gridDim.x * BT) {
        cx<A> c[C];
        ld_vec<T>(x, base + i, c);
        A q = A(0);
#pragma unroll
        for (int j = 0; j < C; ++j) q = fma(c[j].re, c[j].re, fma(c[j].im, c[j].im, q));
        s.add(q);
    }
    block_partial(s.total(), part, (size_t)v * gridDim.x + blockIdx.x);
}

template <typename T>
__global__ void k_cgls_step_v(size_t m, const double* __restrict__ alpha, void* e, const void* __restrict__ p,
                              void* r, const void* __restrict__ t, double* part)
{
    using A = typename Store<T>::A;
    constexpr int C = Store<T>::CPV;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * m;
    const A a = (A)alpha[v];
    Acc<A> s;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < m; i += (size_t)gridDim.x * BT) {
        cx<A> ev[C], pv[C], rv[C], tv[C];
        ld_vec<T>(e, base + i, ev);
        ld_vec<T>(p, base + i, pv);
        ld_vec<T>(r, base + i, rv);
        ld_vec<T>(t, base + i, tv);
        A q = A(0);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            ev[j].re = fma(a, pv[j].re, ev[j].re);
            ev[j].im = fma(a, pv[j].im, ev[j].im);
            rv[j].re = fma(-a, tv[j].re, rv[j].re);
            rv[j].im = fma(-a, tv[j].im, rv[j].im);
            q = fma(rv[j].re, rv[j].re, fma(rv[j].im, rv[j].im, q));
        }
        st_vec<T>(e, base + i, ev);
        st_vec<T>(r, base + i, rv);
        s.add(q);
    }
    block_partial(s.total(), part, (size_t)v * gridDim.x + blockIdx.x);
}

// The split inner solve's step: e += alpha p, r -= alpha t, |r|^2 with e, r,
// t FP32 and p in the 16-bit type H, on Wilson fields (12 complex per site).
// One 16-byte element of p holds 4 complex numbers of one site (plane k of
// 3 in its block of 32 sites); the same numbers sit in planes 2k and 2k + 1
// (of 6) of the FP32 fields, one 16-byte element each.
template <typename H>
__global__ void k_cgls_step_split(size_t m16, const double* __restrict__ alpha, void* e, const void* __restrict__ p,
                                  void* r, const void* __restrict__ t, double* part)
{
    const int v = blockIdx.y;
    const size_t base16 = (size_t)v * m16, base32 = 2 * base16;
    const float a = (float)alpha[v];
    Acc<float> s;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < m16; i += (size_t)gridDim.x * BT) {
        const size_t blk = i / 96, k = (i / 32) % 3, lane = i % 32;
        const size_t j0 = base32 + (blk * 6 + 2 * k) * 32 + lane, j1 = j0 + 32;
        cx<float> pv[4], ev[4], rv[4], tv[4];
        ld_vec<H>(p, base16 + i, pv);
        ld_vec<float>(e, j0, ev);
        ld_vec<float>(e, j1, ev + 2);
        ld_vec<float>(r, j0, rv);
        ld_vec<float>(r, j1, rv + 2);
        ld_vec<float>(t, j0, tv);
        ld_vec<float>(t, j1, tv + 2);
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ev[j].re = fmaf(a, pv[j].re, ev[j].re);
            ev[j].im = fmaf(a, pv[j].im, ev[j].im);
            rv[j].re = fmaf(-a, tv[j].re, rv[j].re);
            rv[j].im = fmaf(-a, tv[j].im, rv[j].im);
            q = fmaf(rv[j].re, rv[j].re, fmaf(rv[j].im, rv[j].im, q));
        }
        st_vec<float>(e, j0, ev);
        st_vec<float>(e, j1, ev + 2);
        st_vec<float>(r, j0, rv);
        st_vec<float>(r, j1, rv + 2);
        s.add(q);
    }
    block_partial(s.total(), part, (size_t)v * gridDim.x + blockIdx.x);
}

template <typename T>
__global__ void k_xpay_v(size_t m, const void* __restrict__ s, const double* __restrict__ beta, void* p)
{
    using A = typename Store<T>::A;
    constexpr int C = Store<T>::CPV;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * m;
    const A b = (A)beta[v];
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < m; i += (size_t)gridDim.x * BT) {
        cx<A> sv[C], pv[C];
        ld_vec<T>(s, base + i, sv);
        ld_vec<T>(p, base + i, pv);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            pv[j].re = fma(b, pv[j].re, sv[j].re);
            pv[j].im = fma(b, pv[j].im, sv[j].im);
        }
        st_vec<T>(p, base + i, pv);
    }
}

// dst = scale_v * src within one storage type, optional partial |dst|^2
template <typename T>
__global__ void k_scale_copy(size_t n, const void* __restrict__ src, const double* __restrict__ scale, void* dst,
                             double* part)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const size_t base = (size_t)v * n;
    const A c = (A)(scale ? scale[v] : 1.0);
    Acc<A> s;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) {
        auto x = ld_one<T>(src, base + i);
        cx<A> y{c * x.re, c * x.im};
        st_one<T>(dst, base + i, y);
        s.add(fma(y.re, y.re, y.im * y.im));
    }
    if (part) block_partial(s.total(), part, (size_t)v * gridDim.x + blockIdx.x);
}

// r64 = b64 - a64, partial |r|^2 (FP64 fields)
__global__ void k_residual64(size_t n, const void* __restrict__ b, const void* __restrict__ a, void* r,
                             double* part)
{
    const int v = blockIdx.y;
    const size_t base = (size_t)v * n;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) {
        cx<double> bv = ld_one<double>(b, base + i), av = ld_one<double>(a, base + i);
        cx<double> rv{bv.re - av.re, bv.im - av.im};
        st_one<double>(r, base + i, rv);
        s += rv.re * rv.re + rv.im * rv.im;
    }
    block_partial(s, part, (size_t)v * gridDim.x + blockIdx.x);
}

// r = b - a with a in double-float storage (four floats re.hi, re.lo, im.hi,
// im.lo per complex); a may alias r: each element is read (plainly, not
// through the read-only path) before the same thread writes it
__global__ void k_residual_df(size_t n, const void* __restrict__ b, const void* a, void* r, double* part)
{
    const int v = blockIdx.y;
    const size_t base = (size_t)v * n;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) {
        const cx<double> bv = ld_one<double>(b, base + i);
        const float4 q = static_cast<const float4*>(a)[base + i];
        cx<double> rv{bv.re - ((double)q.x + (double)q.y), bv.im - ((double)q.z + (double)q.w)};
        st_one<double>(r, base + i, rv);
        s += rv.re * rv.re + rv.im * rv.im;
    }
    block_partial(s, part, (size_t)v * gridDim.x + blockIdx.x);
}

// Fields of different storage types pack the complex numbers of a site into
// 16-byte elements differently, so conversions between them go site by site
// through load_spinor / store_spinor (one thread per site and right-hand side).

// dst = scale_v * src across storage types, optional partial |dst|^2
template <typename TS, typename TD, int NSC>
__global__ void k_convert(long vol, const void* __restrict__ src, const double* __restrict__ scale, void* dst,
                          double* part)
{
    using AS = typename Store<TS>::A;
    using AD = typename Store<TD>::A;
    const int v = blockIdx.y;
    const double c = scale ? scale[v] : 1.0;
    Acc<AD> s2;
    for (long s = (long)blockIdx.x * BT + threadIdx.x; s < vol; s += (long)gridDim.x * BT) {
        cx<AS> a[NSC];
        cx<AD> b[NSC];
        load_spinor<TS, NSC>(src, vol, v, s, a);
        AD q = AD(0);
#pragma unroll
        for (int k = 0; k < NSC; ++k) {
            b[k] = cx<AD>{(AD)(c * (double)a[k].re), (AD)(c * (double)a[k].im)};
            q = fma(b[k].re, b[k].re, fma(b[k].im, b[k].im, q));
        }
        s2.add(q);
        store_spinor<TD, NSC>(dst, vol, v, s, b);
    }
    if (part) block_partial(s2.total(), part, (size_t)v * gridDim.x + blockIdx.x);
}

// x64 += coef_v * e  (e in storage type T, x in FP64), site by site
template <typename T, int NSC>
__global__ void k_axpy_to64(long vol, const double* __restrict__ coef, const void* __restrict__ e, void* x64)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const double c = coef[v];
    if (c == 0.0) return;
    for (long s = (long)blockIdx.x * BT + threadIdx.x; s < vol; s += (long)gridDim.x * BT) {
        cx<A> ev[NSC];
        cx<double> xv[NSC];
        load_spinor<T, NSC>(e, vol, v, s, ev);
        load_spinor<double, NSC>(x64, vol, v, s, xv);
#pragma unroll
        for (int k = 0; k < NSC; ++k) {
            xv[k].re = fma(c, (double)ev[k].re, xv[k].re);
            xv[k].im = fma(c, (double)ev[k].im, xv[k].im);
        }
        store_spinor<double, NSC>(x64, vol, v, s, xv);
    }
}

// ---------------------------------------------------------------- launchers
#define PREC_SWITCH(prec, FN)                                  \
    switch (prec) {                                            \
    case P_F64: FN(double); break;                             \
    case P_F32: FN(float); break;                              \
    case P_BF16: FN(__nv_bfloat16); break;                     \
    case P_F16: FN(__half); break;                             \
    default: return cudaErrorInvalidValue;                     \
    }

static dim3 grid_of(size_t n, int Nv) { return dim3((unsigned)blas_blocks(n), (unsigned)Nv); }

// complex numbers per 16-byte element of a storage precision
static int cpv_of(int prec) { return prec == P_F64 ? 1 : (prec == P_F32 ? 2 : 4); }

cudaError_t blas_norm2(int prec, size_t n, int Nv, const void* x, double* part, double* out,
                       cudaStream_t st)
{
    const int C = cpv_of(prec);
    const bool vec = n % C == 0;
    dim3 g = grid_of(vec ? n / C : n, Nv);
#define GO(T) (vec ? k_norm2_v<T><<<g, BT, 0, st>>>(n / C, x, part) : k_norm2<T><<<g, BT, 0, st>>>(n, x, part))
    PREC_SWITCH(prec, GO)
#undef GO
    k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, out, 0);
    return cudaGetLastError();
}

cudaError_t blas_reduce_partials(const double* part, long nparts, int Nv, double* out, cudaStream_t st)
{
    k_reduce_partials<<<Nv, BT, 0, st>>>(part, (int)nparts, out, 0);
    return cudaGetLastError();
}

cudaError_t blas_dot(int prec, size_t n, int Nv, const void* x, const void* y, double* part,
                     double* out_re, double* out_im, cudaStream_t st)
{
    dim3 g = grid_of(n, Nv);
    double* part_im = part + (size_t)g.x * Nv;
#define GO(T) k_dot<T><<<g, BT, 0, st>>>(n, x, y, part, part_im)
    PREC_SWITCH(prec, GO)
#undef GO
    k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, out_re, 0);
    k_reduce_partials<<<Nv, BT, 0, st>>>(part_im, g.x, out_im, 0);
    return cudaGetLastError();
}

cudaError_t blas_cgls_step(int prec, size_t n, int Nv, const double* alpha, void* e, const void* p, void* r,
                           const void* t, double* part, double* rr, cudaStream_t st)
{
    const int C = cpv_of(prec);
    const bool vec = n % C == 0;
    dim3 g = grid_of(vec ? n / C : n, Nv);
#define GO(T) (vec ? k_cgls_step_v<T><<<g, BT, 0, st>>>(n / C, alpha, e, p, r, t, part) \
               : k_cgls_step<T><<<g, BT, 0, st>>>(n, alpha, e, p, r, t, part))
    PREC_SWITCH(prec, GO)
#undef GO
    k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, rr, 0);
    return cudaGetLastError();
}

cudaError_t blas_xpay(int prec, size_t n, int Nv, const void* s, const double* beta, void* p, cudaStream_t st)
{
    const int C = cpv_of(prec);
    const bool vec = n % C == 0;
    dim3 g = grid_of(vec ? n / C : n, Nv);
#define GO(T) (vec ? k_xpay_v<T><<<g, BT, 0, st>>>(n / C, s, beta, p) : k_xpay<T><<<g, BT, 0, st>>>(n, s, beta, p))
    PREC_SWITCH(prec, GO)
#undef GO
    return cudaGetLastError();
}

template <typename TS, int NSC>
static cudaError_t convert_from(int dprec, dim3 g, long vol, const void* src, const double* scale, void* dst,
                                double* part, cudaStream_t st)
{
#define GO(T) k_convert<TS, T, NSC><<<g, BT, 0, st>>>(vol, src, scale, dst, part)
    switch (dprec) {
    case P_F64: GO(double); break;
    case P_F32: GO(float); break;
    case P_BF16: GO(__nv_bfloat16); break;
    case P_F16: GO(__half); break;
    default: return cudaErrorInvalidValue;
    }
#undef GO
    return cudaGetLastError();
}

template <int NSC>
static cudaError_t convert_nsc(int sprec, int dprec, dim3 g, long vol, const void* src, const double* scale,
                               void* dst, double* part, cudaStream_t st)
{
    switch (sprec) {
    case P_F64: return convert_from<double, NSC>(dprec, g, vol, src, scale, dst, part, st);
    case P_F32: return convert_from<float, NSC>(dprec, g, vol, src, scale, dst, part, st);
    case P_BF16: return convert_from<__nv_bfloat16, NSC>(dprec, g, vol, src, scale, dst, part, st);
    case P_F16: return convert_from<__half, NSC>(dprec, g, vol, src, scale, dst, part, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t blas_convert(int sprec, int dprec, int nsc, long vol, int Nv, const void* src, const double* scale,
                         void* dst, double* part, double* nrm2, cudaStream_t st)
{
    dim3 g = grid_of((size_t)vol * 4, Nv);   // about 4 sites per thread
    cudaError_t e = (nsc == 12) ? convert_nsc<12>(sprec, dprec, g, vol, src, scale, dst, part, st)
                                : convert_nsc<3>(sprec, dprec, g, vol, src, scale, dst, part, st);
    if (e != cudaSuccess) return e;
    if (part && nrm2) k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, nrm2, 0);
    return cudaGetLastError();
}

cudaError_t blas_axpy_to64(int prec, int nsc, long vol, int Nv, const double* coef, const void* e, void* x64,
                           cudaStream_t st)
{
    dim3 g = grid_of((size_t)vol * 4, Nv);
#define GO(T) (nsc == 12 ? (k_axpy_to64<T, 12><<<g, BT, 0, st>>>(vol, coef, e, x64)) \
                         : (k_axpy_to64<T, 3><<<g, BT, 0, st>>>(vol, coef, e, x64)))
    PREC_SWITCH(prec, GO)
#undef GO
    return cudaGetLastError();
}

cudaError_t blas_scale_copy(int prec, size_t n, int Nv, const void* src, const double* scale, void* dst,
                            double* part, double* nrm2, cudaStream_t st)
{
    dim3 g = grid_of(n, Nv);
#define GO(T) k_scale_copy<T><<<g, BT, 0, st>>>(n, src, scale, dst, part)
    PREC_SWITCH(prec, GO)
#undef GO
    if (part && nrm2) k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, nrm2, 0);
    return cudaGetLastError();
}

cudaError_t blas_residual64(size_t n, int Nv, const void* b, const void* a, void* r, double* part, double* rr,
                            cudaStream_t st)
{
    dim3 g = grid_of(n, Nv);
    k_residual64<<<g, BT, 0, st>>>(n, b, a, r, part);
    k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, rr, 0);
    return cudaGetLastError();
}

cudaError_t blas_cgls_step_split(int prec16, size_t n, int Nv, const double* alpha, void* e, const void* p, void* r,
                                 const void* t, double* part, double* rr, cudaStream_t st)
{
    const size_t m16 = n / 4;
    dim3 g = grid_of(m16, Nv);
    if (prec16 == P_BF16) k_cgls_step_split<__nv_bfloat16><<<g, BT, 0, st>>>(m16, alpha, e, p, r, t, part);
    else if (prec16 == P_F16) k_cgls_step_split<__half><<<g, BT, 0, st>>>(m16, alpha, e, p, r, t, part);
    else return cudaErrorInvalidValue;
    k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, rr, 0);
    return cudaGetLastError();
}

cudaError_t blas_residual_df(size_t n, int Nv, const void* b, const void* a_df, void* r, double* part, double* rr,
                             cudaStream_t st)
{
    dim3 g = grid_of(n, Nv);
    k_residual_df<<<g, BT, 0, st>>>(n, b, a_df, r, part);
    k_reduce_partials<<<Nv, BT, 0, st>>>(part, g.x, rr, 0);
    return cudaGetLastError();
}

}  // namespace dirac
