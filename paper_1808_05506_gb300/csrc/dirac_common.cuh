// Shared device-side building blocks of the Dirac kernels: storage types,
// the internal blocked layouts, complex arithmetic, lattice geometry and the
// chiral-basis spin projectors.
//
// Internal layouts (blocked structure-of-arrays, one "element" is a 4- to
// 16-byte vector so that a warp reading 32 aligned sites issues one
// coalesced load per element; blk_index gives the position):
//   spinor   [v][site/32][k][site%32]   k = 0..K-1 element of right-hand side
//                           v at a site; Wilson/Brillouin: 12 complex (spin-
//                           major, colour-minor) split into K = 12/CPV
//                           elements of CPV complex each; staggered: 3
//                           complex, K = 3, CPV = 1.
//   links    [m][site/32][e][site%32]   m = mu (0..3) for V_mu, or one of the
//                           40 stored Brillouin directions; e = row*3 + col.
// Site index s = x + Nx (y + Ny (z + Nz t)).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#if defined(__CUDA_ARCH__)
#define DEV_INLINE __device__ __forceinline__
#else
#define DEV_INLINE inline
#endif
#define HD __host__ __device__ __forceinline__

namespace dirac {

// ---------------------------------------------------------------- complex
template <typename A> struct cx { A re, im; };

template <typename A> HD cx<A> cmk(A r, A i) { return cx<A>{r, i}; }
template <typename A> HD cx<A> operator+(cx<A> a, cx<A> b) { return {a.re + b.re, a.im + b.im}; }
template <typename A> HD cx<A> operator-(cx<A> a, cx<A> b) { return {a.re - b.re, a.im - b.im}; }
template <typename A> HD cx<A> operator-(cx<A> a) { return {-a.re, -a.im}; }
template <typename A> HD cx<A> conj(cx<A> a) { return {a.re, -a.im}; }
template <typename A> HD cx<A> times_i(cx<A> a) { return {-a.im, a.re}; }        // i a
template <typename A> HD cx<A> times_mi(cx<A> a) { return {a.im, -a.re}; }       // -i a
template <typename A> HD cx<A> scale(A s, cx<A> a) { return {s * a.re, s * a.im}; }
// acc + a*b
template <typename A> HD cx<A> cfma(cx<A> a, cx<A> b, cx<A> acc)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc + conj(a)*b
template <typename A> HD cx<A> cfma_conj(cx<A> a, cx<A> b, cx<A> acc)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}
template <typename A> HD cx<A> cmul(cx<A> a, cx<A> b) { return cfma(a, b, cx<A>{A(0), A(0)}); }

// ---------------------------------------------------------------- storage
enum Prec { P_F64 = 0, P_F32 = 1, P_BF16 = 2, P_F16 = 3 };

template <typename T> struct Store;
template <> struct Store<double> {
    using A = double;              // arithmetic type
    using Vec = double2;           // 16-byte element = 1 complex
    static constexpr int CPV = 1;
    using One = double2;           // element holding 1 complex
};
template <> struct Store<float> {
    using A = float;
    using Vec = float4;            // 16-byte element = 2 complex
    static constexpr int CPV = 2;
    using One = float2;
};
template <> struct Store<__nv_bfloat16> {
    using A = float;
    using Vec = uint4;             // 16-byte element = 4 complex
    static constexpr int CPV = 4;
    using One = uint32_t;
};
template <> struct Store<__half> {
    using A = float;
    using Vec = uint4;
    static constexpr int CPV = 4;
    using One = uint32_t;
};

// 16-bit pair <-> float complex
HD cx<float> unpack2(uint32_t w, __nv_bfloat16*)
{
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
    float2 f = __bfloat1622float2(h);
    return {f.x, f.y};
}
HD cx<float> unpack2(uint32_t w, __half*)
{
    __half2 h = *reinterpret_cast<__half2*>(&w);
    float2 f = __half22float2(h);
    return {f.x, f.y};
}
HD uint32_t pack2(cx<float> c, __nv_bfloat16*)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(c.re, c.im);
    return *reinterpret_cast<uint32_t*>(&h);
}
HD uint32_t pack2(cx<float> c, __half*)
{
    __half2 h = __floats2half2_rn(c.re, c.im);
    return *reinterpret_cast<uint32_t*>(&h);
}

// read-only / streaming memory access (plain accesses when emulated on the host)
template <typename V> DEV_INLINE V ld_ro(const V* p)
{
#if defined(__CUDA_ARCH__)
    return __ldg(p);
#else
    return *p;
#endif
}
// read-only load that does not allocate in L1 (for data no other thread of
// this SM will read soon, so that L1 keeps what will be reused)
DEV_INLINE float4 ld_na(const float4* p)
{
#if defined(__CUDA_ARCH__)
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
#else
    return *p;
#endif
}
DEV_INLINE double2 ld_na(const double2* p)
{
#if defined(__CUDA_ARCH__)
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
#else
    return *p;
#endif
}
DEV_INLINE uint4 ld_na(const uint4* p)
{
#if defined(__CUDA_ARCH__)
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
#else
    return *p;
#endif
}
DEV_INLINE float2 ld_na(const float2* p)
{
#if defined(__CUDA_ARCH__)
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
#else
    return *p;
#endif
}
DEV_INLINE uint32_t ld_na(const uint32_t* p)
{
#if defined(__CUDA_ARCH__)
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#else
    return *p;
#endif
}
template <bool NA, typename V> DEV_INLINE V ld_pol(const V* p)
{
    if constexpr (NA) return ld_na(p);
    else return ld_ro(p);
}

template <typename V> DEV_INLINE void st_cs(V* p, V v)
{
#if defined(__CUDA_ARCH__)
    __stcs(p, v);
#else
    *p = v;
#endif
}

// one complex number of storage type T at element index i
template <typename T> DEV_INLINE cx<typename Store<T>::A> ld_one(const void* base, size_t i);
template <> DEV_INLINE cx<double> ld_one<double>(const void* base, size_t i)
{
    double2 v = ld_ro(reinterpret_cast<const double2*>(base) + i);
    return {v.x, v.y};
}
template <> DEV_INLINE cx<float> ld_one<float>(const void* base, size_t i)
{
    float2 v = ld_ro(reinterpret_cast<const float2*>(base) + i);
    return {v.x, v.y};
}
template <> DEV_INLINE cx<float> ld_one<__nv_bfloat16>(const void* base, size_t i)
{
    return unpack2(ld_ro(reinterpret_cast<const uint32_t*>(base) + i), (__nv_bfloat16*)nullptr);
}
template <> DEV_INLINE cx<float> ld_one<__half>(const void* base, size_t i)
{
    return unpack2(ld_ro(reinterpret_cast<const uint32_t*>(base) + i), (__half*)nullptr);
}

template <typename T> DEV_INLINE void st_one(void* base, size_t i, cx<typename Store<T>::A> c);
template <> DEV_INLINE void st_one<double>(void* base, size_t i, cx<double> c)
{
    st_cs(reinterpret_cast<double2*>(base) + i, make_double2(c.re, c.im));
}
template <> DEV_INLINE void st_one<float>(void* base, size_t i, cx<float> c)
{
    st_cs(reinterpret_cast<float2*>(base) + i, make_float2(c.re, c.im));
}
template <> DEV_INLINE void st_one<__nv_bfloat16>(void* base, size_t i, cx<float> c)
{
    st_cs(reinterpret_cast<uint32_t*>(base) + i, pack2(c, (__nv_bfloat16*)nullptr));
}
template <> DEV_INLINE void st_one<__half>(void* base, size_t i, cx<float> c)
{
    st_cs(reinterpret_cast<uint32_t*>(base) + i, pack2(c, (__half*)nullptr));
}

// 16-byte element with CPV complex
template <typename T> DEV_INLINE void ld_vec(const void* base, size_t i, cx<typename Store<T>::A>* out);
template <> DEV_INLINE void ld_vec<double>(const void* base, size_t i, cx<double>* o)
{
    double2 v = ld_ro(reinterpret_cast<const double2*>(base) + i);
    o[0] = {v.x, v.y};
}
template <> DEV_INLINE void ld_vec<float>(const void* base, size_t i, cx<float>* o)
{
    float4 v = ld_ro(reinterpret_cast<const float4*>(base) + i);
    o[0] = {v.x, v.y};
    o[1] = {v.z, v.w};
}
template <typename H> DEV_INLINE void ld_vec16(const void* base, size_t i, cx<float>* o)
{
    uint4 v = ld_ro(reinterpret_cast<const uint4*>(base) + i);
    o[0] = unpack2(v.x, (H*)nullptr);
    o[1] = unpack2(v.y, (H*)nullptr);
    o[2] = unpack2(v.z, (H*)nullptr);
    o[3] = unpack2(v.w, (H*)nullptr);
}
template <> DEV_INLINE void ld_vec<__nv_bfloat16>(const void* b, size_t i, cx<float>* o) { ld_vec16<__nv_bfloat16>(b, i, o); }
template <> DEV_INLINE void ld_vec<__half>(const void* b, size_t i, cx<float>* o) { ld_vec16<__half>(b, i, o); }

template <typename T> DEV_INLINE void st_vec(void* base, size_t i, const cx<typename Store<T>::A>* c);
template <> DEV_INLINE void st_vec<double>(void* base, size_t i, const cx<double>* c)
{
    st_cs(reinterpret_cast<double2*>(base) + i, make_double2(c[0].re, c[0].im));
}
template <> DEV_INLINE void st_vec<float>(void* base, size_t i, const cx<float>* c)
{
    st_cs(reinterpret_cast<float4*>(base) + i, make_float4(c[0].re, c[0].im, c[1].re, c[1].im));
}
template <typename H> DEV_INLINE void st_vec16(void* base, size_t i, const cx<float>* c)
{
    uint4 v;
    v.x = pack2(c[0], (H*)nullptr);
    v.y = pack2(c[1], (H*)nullptr);
    v.z = pack2(c[2], (H*)nullptr);
    v.w = pack2(c[3], (H*)nullptr);
    st_cs(reinterpret_cast<uint4*>(base) + i, v);
}
template <> DEV_INLINE void st_vec<__nv_bfloat16>(void* b, size_t i, const cx<float>* c) { st_vec16<__nv_bfloat16>(b, i, c); }
template <> DEV_INLINE void st_vec<__half>(void* b, size_t i, const cx<float>* c) { st_vec16<__half>(b, i, c); }

// spinor of NSC complex (12 Wilson/Brillouin, 3 staggered) for rhs v at site s
template <typename T, int NSC> struct SpinorLayout {
    static constexpr int CPV = (NSC == 12) ? Store<T>::CPV : 1;
    static constexpr int K = NSC / CPV;
};

// Internal layout of the spinor and link fields: the sites go in blocks of
// 32 (what one warp reads), and inside a block the planes follow each other:
// element (plane q, site s) of a field with Q planes of one right-hand side
// (or one link set) sits at ((p * nblk + s / 32) * Q + q) * 32 + s % 32,
// p = right-hand side (or link direction), nblk = ceil(vol / 32).  A warp on
// 32 aligned sites reads 32 consecutive elements per plane, and the planes of
// one site lie at fixed offsets (32 elements apart), so one address serves a
// whole spinor or link.  The sites s >= vol of the last block are padding.
HD size_t nblk_of(size_t vol) { return (vol + 31) >> 5; }
HD size_t blk_index(size_t vol, int Q, int p, int q, long s)
{
    return (((size_t)p * nblk_of(vol) + ((size_t)s >> 5)) * Q + q) * 32 + ((size_t)s & 31);
}

template <typename T, int NSC>
DEV_INLINE void load_spinor(const void* base, size_t vol, int v, long s, cx<typename Store<T>::A>* out)
{
    using L = SpinorLayout<T, NSC>;
#pragma unroll
    for (int k = 0; k < L::K; ++k) {
        size_t idx = blk_index(vol, L::K, v, k, s);
        if constexpr (L::CPV == 1) out[k] = ld_one<T>(base, idx);
        else ld_vec<T>(base, idx, out + k * L::CPV);
    }
}

template <typename T, int NSC>
DEV_INLINE void store_spinor(void* base, size_t vol, int v, long s, const cx<typename Store<T>::A>* in)
{
    using L = SpinorLayout<T, NSC>;
#pragma unroll
    for (int k = 0; k < L::K; ++k) {
        size_t idx = blk_index(vol, L::K, v, k, s);
        if constexpr (L::CPV == 1) st_one<T>(base, idx, in[k]);
        else st_vec<T>(base, idx, in + k * L::CPV);
    }
}

// the same loads with an L1 policy (NA: do not allocate in L1)
template <typename T, bool NA> DEV_INLINE cx<typename Store<T>::A> ld_one_p(const void* base, size_t i)
{
    if constexpr (!NA) return ld_one<T>(base, i);
    else if constexpr (sizeof(T) == 8) {
        double2 v = ld_na(reinterpret_cast<const double2*>(base) + i);
        return {v.x, v.y};
    } else if constexpr (sizeof(T) == 4) {
        float2 v = ld_na(reinterpret_cast<const float2*>(base) + i);
        return {v.x, v.y};
    } else {
        return unpack2(ld_na(reinterpret_cast<const uint32_t*>(base) + i), (T*)nullptr);
    }
}
template <typename T, bool NA> DEV_INLINE void ld_vec_p(const void* base, size_t i, cx<typename Store<T>::A>* o)
{
    if constexpr (!NA) ld_vec<T>(base, i, o);
    else if constexpr (sizeof(T) == 8) {
        double2 v = ld_na(reinterpret_cast<const double2*>(base) + i);
        o[0] = {v.x, v.y};
    } else if constexpr (sizeof(T) == 4) {
        float4 v = ld_na(reinterpret_cast<const float4*>(base) + i);
        o[0] = {v.x, v.y};
        o[1] = {v.z, v.w};
    } else {
        uint4 v = ld_na(reinterpret_cast<const uint4*>(base) + i);
        o[0] = unpack2(v.x, (T*)nullptr);
        o[1] = unpack2(v.y, (T*)nullptr);
        o[2] = unpack2(v.z, (T*)nullptr);
        o[3] = unpack2(v.w, (T*)nullptr);
    }
}
template <typename T, int NSC, bool NA>
DEV_INLINE void load_spinor_p(const void* base, size_t vol, int v, long s, cx<typename Store<T>::A>* out)
{
    using L = SpinorLayout<T, NSC>;
#pragma unroll
    for (int k = 0; k < L::K; ++k) {
        size_t idx = blk_index(vol, L::K, v, k, s);
        if constexpr (L::CPV == 1) out[k] = ld_one_p<T, NA>(base, idx);
        else ld_vec_p<T, NA>(base, idx, out + k * L::CPV);
    }
}
template <typename T, bool NA>
DEV_INLINE void load_link_p(const void* base, size_t vol, int m, long s, cx<typename Store<T>::A>* U)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) U[e] = ld_one_p<T, NA>(base, blk_index(vol, 9, m, e, s));
}

// 3x3 link m at site s
template <typename T>
DEV_INLINE void load_link(const void* base, size_t vol, int m, long s, cx<typename Store<T>::A>* U)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) U[e] = ld_one<T>(base, blk_index(vol, 9, m, e, s));
}

// Two-row links (gauge compression): only rows 0 and 1 are stored (planes
// e = 0..5 of a layout with 6 planes per link); for a special unitary U the
// third row is the complex conjugate of the cross product of the first two,
// U_2c = conj(U_0a U_1b - U_0b U_1a) for (a, b, c) cyclic.
template <typename A> HD void reconstruct_row2(cx<A>* U)
{
    U[6] = conj(cmul(U[1], U[5]) - cmul(U[2], U[4]));
    U[7] = conj(cmul(U[2], U[3]) - cmul(U[0], U[5]));
    U[8] = conj(cmul(U[0], U[4]) - cmul(U[1], U[3]));
}
template <typename T, bool NA>
DEV_INLINE void load_link_2row(const void* base, size_t vol, int m, long s, cx<typename Store<T>::A>* U)
{
#pragma unroll
    for (int e = 0; e < 6; ++e) U[e] = ld_one_p<T, NA>(base, blk_index(vol, 6, m, e, s));
    reconstruct_row2(U);
}
// link m at site s in link format LF: 0 all nine entries, 1 two rows
template <typename T, bool NA, int LF>
DEV_INLINE void load_link_f(const void* base, size_t vol, int m, long s, cx<typename Store<T>::A>* U)
{
    if constexpr (LF == 1) load_link_2row<T, NA>(base, vol, m, s, U);
    else load_link_p<T, NA>(base, vol, m, s, U);
}

// ---- packed FP32 pairs: one fma.rn.f32x2 does the (re, im) halves of a
// complex update, halving the issue slots of complex arithmetic.  Used by the
// Brillouin sweep, which is issue-bound; the Wilson and staggered sweeps keep
// scalar FMAs (the register pairs cost them occupancy and they are bound by
// memory latency, not by issue)
struct f2 { float x, y; };
DEV_INLINE f2 ffma2(f2 a, f2 b, f2 c)
{
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    unsigned long long ra, rb, rc, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    f2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
#else
    return f2{fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)};
#endif
}
// acc += s * u  (s real)
DEV_INLINE cx<float> caxpy2(float s, cx<float> u, cx<float> acc)
{
    f2 r = ffma2(f2{s, s}, f2{u.re, u.im}, f2{acc.re, acc.im});
    return {r.x, r.y};
}
// acc += a * b as two packed FMAs: acc += a.re (b.re, b.im) + a.im (-b.im, b.re)
DEV_INLINE cx<float> cfma2(cx<float> a, cx<float> b, cx<float> acc)
{
    f2 r = ffma2(f2{a.re, a.re}, f2{b.re, b.im}, f2{acc.re, acc.im});
    r = ffma2(f2{a.im, a.im}, f2{-b.im, b.re}, r);
    return {r.x, r.y};
}
// acc += conj(a) * b: acc += a.re (b.re, b.im) + a.im (b.im, -b.re)
DEV_INLINE cx<float> cfma2_conj(cx<float> a, cx<float> b, cx<float> acc)
{
    f2 r = ffma2(f2{a.re, a.re}, f2{b.re, b.im}, f2{acc.re, acc.im});
    r = ffma2(f2{a.im, a.im}, f2{b.im, -b.re}, r);
    return {r.x, r.y};
}
// acc += U h (3x3 times 3) with packed FMAs: broadcast each h_b, rotate U once
DEV_INLINE void mat_vec_acc2(const cx<float>* U, const cx<float>* h, cx<float>* acc)
{
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const f2 hr{h[b].re, h[b].re}, hi{h[b].im, h[b].im};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const cx<float> u = U[3 * a + b];
            f2 r = ffma2(hr, f2{u.re, u.im}, f2{acc[a].re, acc[a].im});
            r = ffma2(hi, f2{-u.im, u.re}, r);
            acc[a] = {r.x, r.y};
        }
    }
}
// acc += U^dagger h
DEV_INLINE void mat_dag_vec_acc2(const cx<float>* U, const cx<float>* h, cx<float>* acc)
{
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const f2 hr{h[b].re, h[b].re}, hi{h[b].im, h[b].im};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const cx<float> u = U[3 * b + a];   // (U^dagger)_ab = conj(U_ba)
            f2 r = ffma2(hr, f2{u.re, -u.im}, f2{acc[a].re, acc[a].im});
            r = ffma2(hi, f2{u.im, u.re}, r);
            acc[a] = {r.x, r.y};
        }
    }
}

// value of v held by lane src of this warp (all 32 lanes take part)
template <typename A> DEV_INLINE cx<A> shfl_cx(cx<A> v, int src)
{
#if defined(__CUDA_ARCH__)
    return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
#else
    (void)src;
    return v;   // host builds of the kernel bodies have no warps
#endif
}

// w = U h  /  w = U^dagger h   (3-vectors)
template <typename A> HD void mat_vec(const cx<A>* U, const cx<A>* h, cx<A>* w)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<A> acc = cmul(U[3 * a], h[0]);
        acc = cfma(U[3 * a + 1], h[1], acc);
        acc = cfma(U[3 * a + 2], h[2], acc);
        w[a] = acc;
    }
}
template <typename A> HD void mat_dag_vec(const cx<A>* U, const cx<A>* h, cx<A>* w)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<A> acc = cmul(conj(U[a]), h[0]);
        acc = cfma_conj(U[3 + a], h[1], acc);
        acc = cfma_conj(U[6 + a], h[2], acc);
        w[a] = acc;
    }
}
// acc += U h / acc += U^dagger h
template <typename A> HD void mat_vec_acc(const cx<A>* U, const cx<A>* h, cx<A>* acc)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = cfma(U[3 * a], h[0], acc[a]);
        acc[a] = cfma(U[3 * a + 1], h[1], acc[a]);
        acc[a] = cfma(U[3 * a + 2], h[2], acc[a]);
    }
}
template <typename A> HD void mat_dag_vec_acc(const cx<A>* U, const cx<A>* h, cx<A>* acc)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = cfma_conj(U[a], h[0], acc[a]);
        acc[a] = cfma_conj(U[3 + a], h[1], acc[a]);
        acc[a] = cfma_conj(U[6 + a], h[2], acc[a]);
    }
}

// ---------------------------------------------------------------- async copies
// cp.async (global -> shared, completion tracked per thread by commit/wait
// groups).  Each thread reads back only what it copied itself, so no barrier
// is needed between the copy and the use.
template <int BYTES> DEV_INLINE void cp_async(void* smem, const void* gmem)
{
#if defined(__CUDA_ARCH__)
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    else if constexpr (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
#else
    const char* g = static_cast<const char*>(gmem);
    char* d = static_cast<char*>(smem);
    for (int i = 0; i < BYTES; ++i) d[i] = g[i];
#endif
}
DEV_INLINE void cp_async_commit()
{
#if defined(__CUDA_ARCH__)
    asm volatile("cp.async.commit_group;\n" ::: "memory");
#endif
}
template <int N> DEV_INLINE void cp_async_wait()
{
#if defined(__CUDA_ARCH__)
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
#endif
}

// ---------------------------------------------------------------- geometry
// Division by an invariant divisor as a multiply-high and a shift (Granlund
// and Montgomery, "Division by invariant integers using multiplication",
// PLDI 1994): for 0 <= n < 2^31 and 2 <= d < 2^31, with s = ceil(log2 d) and
// M = floor(2^(31+s) / d) + 1 (< 2^32), d < M d - 2^(31+s) + d <= 2^s + d
// gives floor(n / d) = floor(n M / 2^(31+s)).  Site indices are below 2^31.
struct FDiv {
    uint32_t d = 1, M = 0;
    int sh = 0;   // s - 1
};
inline FDiv make_fdiv(uint32_t d)
{
    FDiv f;
    f.d = d;
    if (d <= 1) return f;
    int s = 0;
    while ((1ull << s) < d) ++s;
    f.M = (uint32_t)((1ull << (31 + s)) / d + 1);
    f.sh = s - 1;
    return f;
}
HD uint32_t fdiv(const FDiv& f, uint32_t n)
{
    if (f.d == 1) return n;
#if defined(__CUDA_ARCH__)
    return __umulhi(n, f.M) >> f.sh;
#else
    return (uint32_t)(((uint64_t)n * f.M) >> 32) >> f.sh;
#endif
}

struct Geom {
    int L[4];        // Nx, Ny, Nz, Nt
    long stride[4];  // 1, Nx, Nx Ny, Nx Ny Nz
    long vol;
    FDiv fd[4];      // division by L[mu]
    FDiv fdP;        // division by Nx Ny
};

inline Geom make_geom(int Nx, int Ny, int Nz, int Nt)
{
    Geom g;
    g.L[0] = Nx;
    g.L[1] = Ny;
    g.L[2] = Nz;
    g.L[3] = Nt;
    g.stride[0] = 1;
    g.stride[1] = Nx;
    g.stride[2] = (long)Nx * Ny;
    g.stride[3] = (long)Nx * Ny * Nz;
    g.vol = g.stride[3] * Nt;
    for (int mu = 0; mu < 4; ++mu) g.fd[mu] = make_fdiv((uint32_t)g.L[mu]);
    g.fdP = make_fdiv((uint32_t)g.stride[2]);
    return g;
}

// Processing order of the sites of a slab of nt consecutive t-slices.  With
// tc = 0 the p-th site is site p of the slab (lexicographic).  With tc > 0
// the (z, t) planes of Lx Ly sites are visited in chunks of tc t-slices, and
// inside a chunk t runs faster than z, so a site's t-neighbours are swept a
// few planes after it rather than a whole (x, y, z) volume later; the last
// chunk may be shorter.  A bijection on 0 <= p < nt Lx Ly Lz (the offset of
// the slab is added by the caller).
// fdc, fdt: division by Lz tc and by tc
HD long site_of(const Geom& g, long p, int tc, int nt, const FDiv& fdc, const FDiv& fdt)
{
    if (tc <= 0) return p;
    const uint32_t P = (uint32_t)g.stride[2];
    const uint32_t q = fdiv(g.fdP, (uint32_t)p), w = (uint32_t)p - q * P;
    const uint32_t chunk = (uint32_t)g.L[2] * (uint32_t)tc;
    const uint32_t tb = fdiv(fdc, q);
    const uint32_t r = q - tb * chunk;
    const int t0 = (int)tb * tc;
    const int n = (nt - t0 < tc) ? nt - t0 : tc;
    uint32_t z;
    if (n == tc) z = fdiv(fdt, r);
    else z = r / (uint32_t)n;   // the shorter last chunk
    const int ti = (int)(r - z * (uint32_t)n);
    return (long)w + (long)P * ((long)z + (long)g.L[2] * (t0 + ti));
}

// neighbour offsets of site s: fwd[mu] = (s + mu) - s, bwd[mu] = (s - mu) - s (periodic)
HD void site_offsets(const Geom& g, long s, long* fwd, long* bwd, int* x)
{
    uint32_t r = (uint32_t)s;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const uint32_t q = fdiv(g.fd[mu], r);
        const int c = (int)(r - q * (uint32_t)g.L[mu]);
        r = q;
        x[mu] = c;
        fwd[mu] = (c == g.L[mu] - 1) ? -(long)(g.L[mu] - 1) * g.stride[mu] : g.stride[mu];
        bwd[mu] = (c == 0) ? (long)(g.L[mu] - 1) * g.stride[mu] : -g.stride[mu];
    }
}

}  // namespace dirac
