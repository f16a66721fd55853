// Wilson D_W and D_W^+ sweeps (Sec. 4, Eq. def_wils at c_SW = 0) on the
// internal site-fastest layout.  One thread owns one site and R right-hand
// sides: every link is loaded once per thread and applied to its R spinors
// from registers, and every output element is written once.  Consecutive
// blocks cover the right-hand-side groups of the same sites, so the other
// groups find the links in L2.
#include "dirac_internal.h"

namespace dirac {

template <typename T, int R, bool DAG>
__global__ void __launch_bounds__(256) k_wilson(ApplyArgs a, int ngroups)
{
    const long b = blockIdx.x;
    const int group = (int)(b % ngroups);
    const long s = (b / ngroups) * blockDim.x + threadIdx.x;
    if (s >= a.g.vol) return;
    wilson_site<T, R, DAG>(a, s, group);
}

// V_TMARCH: blockDim = (sites, groups); a block owns a run of `block` sites of
// one t-slice (index s3 within the slice) and walks TC consecutive slices, so
// the t-neighbours and backward t-links it needs were read by this block one
// step earlier and are still in L1
template <typename T, int R, bool DAG>
__global__ void __launch_bounds__(192, 2) k_wilson_march(ApplyArgs a, int ngroups, int gy, int tc)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long vol3 = a.g.stride[3];
    const long nruns = (vol3 + blockDim.x - 1) / blockDim.x;
    long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    b /= nchunks;
    const long s3 = (b % nruns) * blockDim.x + threadIdx.x;
    const int t0 = (int)(b / nruns) * tc;
    if (s3 >= vol3 || group >= ngroups) return;
    const int t1 = min(t0 + tc, a.g.L[3]);
    for (int t = t0; t < t1; ++t) wilson_site<T, R, DAG, true>(a, s3 + vol3 * t, group);
}

// pipelined variant: the loads of later hops are in flight in shared memory
template <typename T, int R, bool DAG, int ST>
__global__ void __launch_bounds__(256) k_wilson_pipe(ApplyArgs a, int ngroups)
{
    extern __shared__ __align__(16) char smem[];
    const long b = blockIdx.x;
    const int group = (int)(b % ngroups);
    const long s = (b / ngroups) * blockDim.x + threadIdx.x;
    if (s >= a.g.vol) return;   // no block-wide synchronisation follows
    wilson_site_pipe<T, R, DAG, ST>(a, s, group, smem, threadIdx.x, blockDim.x);
}

// V_GROUPS: blockDim = (sites, groups); block b covers a run of sites and a
// chunk of gy right-hand-side groups
template <typename T, int R, bool DAG>
__global__ void __launch_bounds__(192, 2) k_wilson_groups(ApplyArgs a, int ngroups, int gy)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    const long s = (b / nchunks) * blockDim.x + threadIdx.x;
    if (s >= a.g.vol || group >= ngroups) return;
    wilson_site<T, R, DAG>(a, s, group);
}

template <typename T, int R>
static cudaError_t go(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    const int block = c.block;
    const int ngroups = (a.Nv + R - 1) / R;
    const long nblk = ((a.g.vol + block - 1) / block) * (long)ngroups;
    if (c.variant == V_GROUPS) {
        const int gy = groups_per_block(block, ngroups);
        const long nb = ((a.g.vol + block - 1) / block) * (long)((ngroups + gy - 1) / gy);
        if (dag) k_wilson_groups<T, R, true><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
        else k_wilson_groups<T, R, false><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
        return cudaGetLastError();
    }
    if (c.variant == V_TMARCH) {
        const int gy = groups_per_block(block, ngroups);
        const long vol3 = a.g.stride[3];
        const int tc = a.g.L[3] < 8 ? a.g.L[3] : 8;
        const long nb = ((vol3 + block - 1) / block) * (long)((ngroups + gy - 1) / gy) *
                        (long)((a.g.L[3] + tc - 1) / tc);
        if (dag) k_wilson_march<T, R, true><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy, tc);
        else k_wilson_march<T, R, false><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy, tc);
        return cudaGetLastError();
    }
    if (c.variant == V_PIPE3) {
        const size_t smem = WilsonPipe<T, R>::stage_bytes_per_thread * 3 * block;
        auto kern = dag ? k_wilson_pipe<T, R, true, 3> : k_wilson_pipe<T, R, false, 3>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)nblk, block, smem, st>>>(a, ngroups);
        return cudaGetLastError();
    }
    if (dag) k_wilson<T, R, true><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    else k_wilson<T, R, false><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t go_T(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    switch (c.R) {
    case 1: return go<T, 1>(dag, a, c, st);
    case 2: return go<T, 2>(dag, a, c, st);
    case 3: return go<T, 3>(dag, a, c, st);
    case 4: return go<T, 4>(dag, a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t wilson_pipe_smem(int prec, int R, int block, int stages)
{
    const size_t K = prec == P_F64 ? 12 : (prec == P_F32 ? 6 : 3);
    const size_t LB = prec == P_F64 ? 16 : (prec == P_F32 ? 8 : 4);
    return (R * K * 16 + 9 * LB) * stages * block;
}

cudaError_t launch_apply_wilson(int prec, bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    switch (prec) {
    case P_F64: return go_T<double>(dag, a, c, st);
    case P_F32: return go_T<float>(dag, a, c, st);
    case P_BF16: return go_T<__nv_bfloat16>(dag, a, c, st);
    case P_F16: return go_T<__half>(dag, a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dirac
