// Double-float residual sweeps (dirac_df.cuh) of the Wilson and staggered
// operators, and the FP64 -> double-float conversion of fields and links.
#include "dirac_df.cuh"

namespace dirac {

// one thread per (site, right-hand side); blockDim = (DF_SITES, DF_COLS): the
// DF_COLS right-hand sides of a block (one warp each) read the same links, so
// each link comes from L2 once per block and from L1 for the other warps
template <int OP>
__global__ void __launch_bounds__(DF_SITES * DF_COLS) k_apply_df(ApplyArgs a)
{
    const int ncb = (a.Nv + DF_COLS - 1) / DF_COLS;
    const long b = blockIdx.x;
    const int v = (int)(b % ncb) * DF_COLS + threadIdx.y;
    const long p = (b / ncb) * DF_SITES + threadIdx.x;
    if (p >= a.nsites || v >= a.Nv) return;
    const long s = slab_site(a, p);
    if constexpr (OP == OP_WILSON) wilson_site<f64df, 1, false, 0>(a, s, v);
    else staggered_site<f64df, 1, false, 0>(a, s, v);
}

cudaError_t launch_apply_df(int op, const ApplyArgs& a, cudaStream_t st)
{
    if (a.nsites == 0 || a.Nv == 0) return cudaSuccess;
    if (op == OP_BRILLOUIN) return launch_brillouin_df(a, st);
    const long nb = ((a.nsites + DF_SITES - 1) / DF_SITES) * (long)((a.Nv + DF_COLS - 1) / DF_COLS);
    const dim3 block(DF_SITES, DF_COLS);
    if (op == OP_WILSON) k_apply_df<OP_WILSON><<<(unsigned)nb, block, 0, st>>>(a);
    else if (op == OP_STAGGERED) k_apply_df<OP_STAGGERED><<<(unsigned)nb, block, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

__global__ void k_df_from_f64(size_t n16, const double2* __restrict__ src, float4* dst)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        const dfl re(v.x), im(v.y);
        dst[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}

cudaError_t df_from_f64(size_t n16, const void* src, void* dst, cudaStream_t st)
{
    if (n16 == 0) return cudaSuccess;
    size_t b = (n16 + 1023) / 1024;
    if (b > 4096) b = 4096;
    k_df_from_f64<<<(unsigned)b, 256, 0, st>>>(n16, static_cast<const double2*>(src), static_cast<float4*>(dst));
    return cudaGetLastError();
}

}  // namespace dirac
