// Kernel templates of the Wilson sweep (Sec. 4, Eq. def_wils at c_SW = 0);
// instantiated once per storage type in apply_wilson_<type>.cu.
#pragma once

#include "dirac_internal.h"
#include <type_traits>

#include "dirac_kernels.cuh"

namespace dirac {


template <typename T, int R, bool DAG>
__global__ void __launch_bounds__(256) k_wilson(ApplyArgs a, int ngroups)
{
    const long b = blockIdx.x;
    const int group = (int)(b % ngroups);
    const long p = (b / ngroups) * blockDim.x + threadIdx.x;
    if (p >= a.nsites) return;
    wilson_site<T, R, DAG>(a, slab_site(a, p), group);
}

// V_TMARCH: blockDim = (sites, groups); a block owns a run of `block` site
// columns of the (x, y, z) volume and walks `tc` consecutive t-slices with
// the t hops carried in registers (wilson_column)
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
    const int t0 = a.t0 + (int)(b / nruns) * tc;
    if (s3 >= vol3 || group >= ngroups) return;
    wilson_column<T, R, DAG>(a, s3, group, t0, min(t0 + tc, a.t0 + a.nt));
}

// V_XROW: blockDim = (32, gy); warp y of block b takes right-hand-side group
// (b % nchunks) * gy + y on the 32-site run (b / nchunks) % nruns of the
// (x, y, z) volume and the t-chunk (b / nchunks) / nruns (wilson_xrow)
template <typename T, int R, bool DAG>
__global__ void __launch_bounds__(192, 2) k_wilson_xrow(ApplyArgs a, int ngroups, int gy, int tc)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long nruns = a.g.stride[3] / 32;
    long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    b /= nchunks;
    const long s3 = (b % nruns) * 32 + threadIdx.x;
    const int t0 = a.t0 + (int)(b / nruns) * tc;
    if (group >= ngroups) return;   // a whole warp
    wilson_xrow<T, R, DAG>(a, s3, threadIdx.x, group, t0, min(t0 + tc, a.t0 + a.nt));
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
// LF: link format (0 nine entries per link, 1 two rows, reconstructed)
template <typename T, int R, bool DAG, int MODE, int LF>
__global__ void __launch_bounds__(192, 2) k_wilson_groups(ApplyArgs a, int ngroups, int gy)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    const long p = (b / nchunks) * blockDim.x + threadIdx.x;
    if (p >= a.nsites || group >= ngroups) return;
    wilson_site<T, R, DAG, MODE, LF>(a, slab_site(a, p), group);
}

// V_XLAST: V_GROUPS with the x hops last, by lane exchange (wilson_site_xlast);
// the host checked that every warp holds whole x-rows
template <typename T, int R, bool DAG, int MODE, int LF>
__global__ void __launch_bounds__(192, 2) k_wilson_xlast(ApplyArgs a, int ngroups, int gy)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    const long p = (b / nchunks) * blockDim.x + threadIdx.x;
    if (p >= a.nsites || group >= ngroups) return;   // whole warps
    wilson_site_xlast<T, R, DAG, MODE, LF>(a, slab_site(a, p), threadIdx.x & 31, group);
}

template <typename T, int R>
cudaError_t go(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    const int block = c.block;
    const int ngroups = (a.Nv + R - 1) / R;
    const long nblk = ((a.nsites + block - 1) / block) * (long)ngroups;
    if constexpr (sizeof(T) != 8) {
    if (c.variant == V_GROUPS) {
        const int gy = groups_per_block(block, ngroups);
        const long nb = ((a.nsites + block - 1) / block) * (long)((ngroups + gy - 1) / gy);
        // whole groups of R right-hand sides: the specialised bodies
        const bool dv = sizeof(T) == 8 ? a.diag_v != nullptr : a.diag_vf != nullptr;
        const int mode = (a.Nv % R != 0 || (a.diag_v != nullptr && !dv)) ? 0 : (dv ? 2 : 1);
        auto launch_lf = [&](auto m, auto lf) {
            constexpr int M = decltype(m)::value;
            constexpr int LF = decltype(lf)::value;
            if (dag) k_wilson_groups<T, R, true, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
            else k_wilson_groups<T, R, false, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
        };
        auto launch = [&](auto m) {
            if (c.fmt == 1) launch_lf(m, std::integral_constant<int, 1>{});
            else launch_lf(m, std::integral_constant<int, 0>{});
        };
        if (mode == 1) launch(std::integral_constant<int, 1>{});
        else if (mode == 2) launch(std::integral_constant<int, 2>{});
        else launch(std::integral_constant<int, 0>{});
        return cudaGetLastError();
    }
    if constexpr (R <= 2) {
    if (c.variant == V_XLAST) {
        const int gy = groups_per_block(block, ngroups);
        const long nb = ((a.nsites + block - 1) / block) * (long)((ngroups + gy - 1) / gy);
        const bool dv = a.diag_vf != nullptr;
        const int mode = (a.Nv % R != 0 || (a.diag_v != nullptr && !dv)) ? 0 : (dv ? 2 : 1);
        auto launch_lf = [&](auto m, auto lf) {
            constexpr int M = decltype(m)::value;
            constexpr int LF = decltype(lf)::value;
            if (dag) k_wilson_xlast<T, R, true, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
            else k_wilson_xlast<T, R, false, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
        };
        auto launch = [&](auto m) {
            if (c.fmt == 1) launch_lf(m, std::integral_constant<int, 1>{});
            else launch_lf(m, std::integral_constant<int, 0>{});
        };
        if (mode == 1) launch(std::integral_constant<int, 1>{});
        else if (mode == 2) launch(std::integral_constant<int, 2>{});
        else launch(std::integral_constant<int, 0>{});
        return cudaGetLastError();
    }
    if (c.variant == V_XROW) {
        // the host checked 32 % Lx == 0 and vol3 % 32 == 0: every warp is full
        const int gy = min(c.block / 32, ngroups);
        const int tc = a.nt < 8 ? a.nt : 8;
        const long nb = (a.g.stride[3] / 32) * (long)((ngroups + gy - 1) / gy) * (long)((a.nt + tc - 1) / tc);
        if (dag) k_wilson_xrow<T, R, true><<<(unsigned)nb, dim3(32, gy), 0, st>>>(a, ngroups, gy, tc);
        else k_wilson_xrow<T, R, false><<<(unsigned)nb, dim3(32, gy), 0, st>>>(a, ngroups, gy, tc);
        return cudaGetLastError();
    }
    if (c.variant == V_TMARCH) {
        const int gy = groups_per_block(block, ngroups);
        const long vol3 = a.g.stride[3];
        const int tc = a.nt < 8 ? a.nt : 8;
        const long nb = ((vol3 + block - 1) / block) * (long)((ngroups + gy - 1) / gy) *
                        (long)((a.nt + tc - 1) / tc);
        if (dag) k_wilson_march<T, R, true><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy, tc);
        else k_wilson_march<T, R, false><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy, tc);
        return cudaGetLastError();
    }
    }   // R <= 2: the carried variants spill beyond two right-hand sides per thread
    if (c.variant == V_PIPE3) {
        const size_t smem = WilsonPipe<T, R>::stage_bytes_per_thread * 3 * block;
        auto kern = dag ? k_wilson_pipe<T, R, true, 3> : k_wilson_pipe<T, R, false, 3>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)nblk, block, smem, st>>>(a, ngroups);
        return cudaGetLastError();
    }
    }   // not FP64
    if (dag) k_wilson<T, R, true><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    else k_wilson<T, R, false><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    return cudaGetLastError();
}

template <typename T>
cudaError_t wilson_go_T(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    if constexpr (sizeof(T) == 8) {
        // FP64 sweeps are FP64-ALU bound on this GPU: only the direct variant is built
        if (c.variant != V_DIRECT) return cudaErrorInvalidValue;
    }

    switch (c.R) {
    case 1: return go<T, 1>(dag, a, c, st);
    case 2: return go<T, 2>(dag, a, c, st);
    case 3: return go<T, 3>(dag, a, c, st);
    case 4: return go<T, 4>(dag, a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dirac
