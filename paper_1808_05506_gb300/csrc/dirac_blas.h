// Vector kernels of the solvers (dirac_blas.cu).  n = complex numbers per
// right-hand side; every field holds Nv such contiguous segments.  The
// reductions write one FP64 value per right-hand side to a device array and
// use part (at least blas_partials(n, Nv) doubles; twice that for blas_dot)
// as scratch.
#pragma once

#include "dirac_internal.h"

namespace dirac {

int blas_blocks(size_t n);
size_t blas_partials(size_t n, int Nv);

cudaError_t blas_norm2(int prec, size_t n, int Nv, const void* x, double* part, double* out, cudaStream_t st);
cudaError_t blas_dot(int prec, size_t n, int Nv, const void* x, const void* y, double* part, double* out_re,
                     double* out_im, cudaStream_t st);
// e += alpha_v p ; r -= alpha_v t ; rr_v = |r_v|^2
cudaError_t blas_cgls_step(int prec, size_t n, int Nv, const double* alpha, void* e, const void* p, void* r,
                           const void* t, double* part, double* rr, cudaStream_t st);
// the same with e, r, t FP32 and p in the 16-bit prec16, Wilson fields (the
// split inner solve); n = complex numbers per right-hand side
cudaError_t blas_cgls_step_split(int prec16, size_t n, int Nv, const double* alpha, void* e, const void* p, void* r,
                                 const void* t, double* part, double* rr, cudaStream_t st);
// out_v = sum of the nparts partials part[v * nparts + i] (fixed order)
cudaError_t blas_reduce_partials(const double* part, long nparts, int Nv, double* out, cudaStream_t st);
// p = s + beta_v p
cudaError_t blas_xpay(int prec, size_t n, int Nv, const void* s, const double* beta, void* p, cudaStream_t st);
// dst = scale_v src within one storage type (scale NULL: 1); nrm2_v = |dst_v|^2
// if part and nrm2 are given
cudaError_t blas_scale_copy(int prec, size_t n, int Nv, const void* src, const double* scale, void* dst,
                            double* part, double* nrm2, cudaStream_t st);
// the same across storage types (site by site, since the element packing differs)
cudaError_t blas_convert(int sprec, int dprec, int nsc, long vol, int Nv, const void* src, const double* scale,
                         void* dst, double* part, double* nrm2, cudaStream_t st);
// x64 += coef_v e, site by site
cudaError_t blas_axpy_to64(int prec, int nsc, long vol, int Nv, const double* coef, const void* e, void* x64,
                           cudaStream_t st);
// r = b - a (FP64), rr_v = |r_v|^2
cudaError_t blas_residual64(size_t n, int Nv, const void* b, const void* a, void* r, double* part, double* rr,
                            cudaStream_t st);
// the same with a in double-float storage (dirac_df.cuh); a_df may alias r
cudaError_t blas_residual_df(size_t n, int Nv, const void* b, const void* a_df, void* r, double* part, double* rr,
                             cudaStream_t st);

}  // namespace dirac
