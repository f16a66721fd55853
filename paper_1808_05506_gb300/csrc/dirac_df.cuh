// Double-float ("df") arithmetic for the outer residual of the solvers.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <=
// ulp(hi) / 2, which carries a 48-bit significand (relative precision about
// 2^-48 = 3.6e-15) in FP32's exponent range.  FP64 arithmetic runs at a small
// fraction of the FP32 rate on this GPU, so the residual sweep r = b - D x in
// double-float costs several times less than in FP64 while resolving
// |r| / |b| far below the 1e-10 the solvers target.
//
// The operations are the classical error-free transformations: Knuth's
// two-sum (exact a + b = s + e) and the product a * b = p + e exact through
// one fused multiply-add (Dekker's two-product with an FMA), followed by a
// renormalisation (fast two-sum, valid for |s| >= |e|), as in the
// double-double arithmetic of Hida, Li and Bailey (2001), here on FP32
// halves.  The sum and the fused multiply-add are the "sloppy" forms, whose
// error bound is relative to the magnitudes of the operands (not of the
// result) -- which is what a residual sum of products needs.
//
// Storage type f64df: a complex number is four floats (re.hi, re.lo, im.hi,
// im.lo), 16 bytes, in the internal blocked layout of an FP64 field (one
// complex per element), so fields and links convert element by element.
#pragma once

#include <cmath>

#include "dirac_internal.h"

namespace dirac {

// FP32 operations that the compiler must not fuse into multiply-adds (a
// contracted a * b + c would break the error-free transformations below)
HD float df_add(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
HD float df_sub(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
HD float df_mul(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
HD float df_fma(float a, float b, float c)
{
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

// dfl and its operators live in a namespace of their own: they are found by
// argument-dependent lookup for dfl operands only, and never hide the FP32 /
// FP64 fma of the other kernel bodies from ordinary lookup
namespace dd {

struct dfl {
    float hi, lo;
    HD dfl() : hi(0.f), lo(0.f) {}
    HD dfl(float h, float l) : hi(h), lo(l) {}
    HD dfl(int v) : hi((float)v), lo(0.f) {}
    HD dfl(float v) : hi(v), lo(0.f) {}
    // exact for doubles whose significand fits 48 bits, else rounded once
    HD dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

// s + e = a + b exactly (Knuth)
HD void two_sum(float a, float b, float& s, float& e)
{
    s = df_add(a, b);
    const float bb = df_sub(s, a);
    e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
}
// s + e = a + b exactly, given |a| >= |b|
HD void fast_two_sum(float a, float b, float& s, float& e)
{
    s = df_add(a, b);
    e = df_sub(b, df_sub(s, a));
}

HD dfl operator+(dfl a, dfl b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = df_add(e, df_add(a.lo, b.lo));
    dfl r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
HD dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
HD dfl operator-(dfl a, dfl b) { return a + (-b); }

// a * b + c
HD dfl fma(dfl a, dfl b, dfl c)
{
    const float p = df_mul(a.hi, b.hi);
    float e = df_fma(a.hi, b.hi, -p);   // the rounding error of p, exactly
    e = df_fma(a.hi, b.lo, e);          // the cross terms (a.lo b.lo is below the precision)
    e = df_fma(a.lo, b.hi, e);
    float s, t;
    two_sum(p, c.hi, s, t);
    t = df_add(t, df_add(e, c.lo));
    dfl r;
    fast_two_sum(s, t, r.hi, r.lo);
    return r;
}
HD dfl operator*(dfl a, dfl b) { return fma(a, b, dfl()); }

// the double nearest to hi + lo (exact: the two halves fit 53 bits)
HD double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

}  // namespace dd

using dd::dfl;

struct f64df {
    float4 v;   // storage tag (never instantiated as data)
};
template <> struct Store<f64df> {
    using A = dfl;
    using Vec = float4;
    static constexpr int CPV = 1;
    using One = float4;
};

template <> DEV_INLINE cx<dfl> ld_one<f64df>(const void* base, size_t i)
{
    const float4 v = ld_ro(reinterpret_cast<const float4*>(base) + i);
    return {dfl(v.x, v.y), dfl(v.z, v.w)};
}
template <> DEV_INLINE void ld_vec<f64df>(const void* base, size_t i, cx<dfl>* o) { o[0] = ld_one<f64df>(base, i); }
template <> DEV_INLINE void st_one<f64df>(void* base, size_t i, cx<dfl> c)
{
    st_cs(reinterpret_cast<float4*>(base) + i, make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo));
}
template <> DEV_INLINE void st_vec<f64df>(void* base, size_t i, const cx<dfl>* c) { st_one<f64df>(base, i, c[0]); }

// launch shape of the double-float sweeps: blocks of DF_SITES sites x DF_COLS
// right-hand sides (one warp per right-hand side)
constexpr int DF_SITES = 32;
constexpr int DF_COLS = 4;

// the double-float residual sweep: out = D in (no adjoint), direct variant,
// one right-hand side per thread; in, out and links in f64df storage
cudaError_t launch_apply_df(int op, const ApplyArgs& a, cudaStream_t st);
cudaError_t launch_brillouin_df(const ApplyArgs& a, cudaStream_t st);

// n16 16-byte elements: FP64 complex (re, im) -> f64df (hi, lo pairs)
cudaError_t df_from_f64(size_t n16, const void* src, void* dst, cudaStream_t st);

}  // namespace dirac
