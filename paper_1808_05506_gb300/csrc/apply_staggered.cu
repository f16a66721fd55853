// Staggered D_S and D_S^+ sweeps (Sec. 3, plus a mass term) on the
// internal blocked layout.  One thread owns one site and R right-hand
// sides: every link is loaded once per thread and applied to its R spinors
// from registers, and every output element is written once.  Consecutive
// blocks cover the right-hand-side groups of the same sites, so the other
// groups find the links in L2.
#include <type_traits>

#include "dirac_internal.h"

namespace dirac {

template <typename T, int R, bool DAG>
__global__ void __launch_bounds__(256) k_staggered(ApplyArgs a, int ngroups)
{
    const long b = blockIdx.x;
    const int group = (int)(b % ngroups);
    const long p = (b / ngroups) * blockDim.x + threadIdx.x;
    if (p >= a.nsites) return;
    staggered_site<T, R, DAG>(a, slab_site(a, p), group);
}

// V_GROUPS: blockDim = (sites, groups); block b covers a run of sites and a
// chunk of gy right-hand-side groups
// LF: link format (0 nine entries per link, 1 two rows, reconstructed)
template <typename T, int R, bool DAG, int MODE, int LF>
__global__ void __launch_bounds__(192, 2) k_staggered_groups(ApplyArgs a, int ngroups, int gy)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    const long p = (b / nchunks) * blockDim.x + threadIdx.x;
    if (p >= a.nsites || group >= ngroups) return;
    staggered_site<T, R, DAG, MODE, LF>(a, slab_site(a, p), group);
}

// V_XLAST: V_GROUPS with the x hops last, by lane exchange (staggered_site_xlast);
// the host checked that every warp holds whole x-rows
template <typename T, int R, bool DAG, int MODE, int LF>
__global__ void __launch_bounds__(192, 2) k_staggered_xlast(ApplyArgs a, int ngroups, int gy)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    const long p = (b / nchunks) * blockDim.x + threadIdx.x;
    if (p >= a.nsites || group >= ngroups) return;   // whole warps
    staggered_site_xlast<T, R, DAG, MODE, LF>(a, slab_site(a, p), threadIdx.x & 31, group);
}

template <typename T, int R>
static cudaError_t go(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    const int block = c.block;
    const int ngroups = (a.Nv + R - 1) / R;
    if constexpr (sizeof(T) != 8) {
    if (c.variant == V_XLAST) {
        const int gy = groups_per_block(block, ngroups);
        const long nb = ((a.nsites + block - 1) / block) * (long)((ngroups + gy - 1) / gy);
        const bool dv = a.diag_vf != nullptr;
        const int mode = (a.Nv % R != 0 || (a.diag_v != nullptr && !dv)) ? 0 : (dv ? 2 : 1);
        auto launch_lf = [&](auto m, auto lf) {
            constexpr int M = decltype(m)::value;
            constexpr int LF = decltype(lf)::value;
            if (dag) k_staggered_xlast<T, R, true, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
            else k_staggered_xlast<T, R, false, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
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
    }
    if (c.variant == V_GROUPS) {
        const int gy = groups_per_block(block, ngroups);
        const long nb = ((a.nsites + block - 1) / block) * (long)((ngroups + gy - 1) / gy);
        const bool dv = sizeof(T) == 8 ? a.diag_v != nullptr : a.diag_vf != nullptr;
        const int mode = (a.Nv % R != 0 || (a.diag_v != nullptr && !dv)) ? 0 : (dv ? 2 : 1);
        auto launch_lf = [&](auto m, auto lf) {
            constexpr int M = decltype(m)::value;
            constexpr int LF = decltype(lf)::value;
            if (dag) k_staggered_groups<T, R, true, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
            else k_staggered_groups<T, R, false, M, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
        };
        auto launch = [&](auto m) {
            // two-row links are built for FP32 and 16-bit storage only
            if constexpr (sizeof(T) != 8) {
                if (c.fmt == 1) return launch_lf(m, std::integral_constant<int, 1>{});
            }
            launch_lf(m, std::integral_constant<int, 0>{});
        };
        if (mode == 1) launch(std::integral_constant<int, 1>{});
        else if (mode == 2) launch(std::integral_constant<int, 2>{});
        else launch(std::integral_constant<int, 0>{});
        return cudaGetLastError();
    }
    const long nblk = ((a.nsites + block - 1) / block) * (long)ngroups;
    if (dag) k_staggered<T, R, true><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    else k_staggered<T, R, false><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t go_T(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    if (c.variant != V_DIRECT && c.variant != V_GROUPS && c.variant != V_XLAST) return cudaErrorInvalidValue;
    switch (c.R) {
    case 1: return go<T, 1>(dag, a, c, st);
    case 2: return go<T, 2>(dag, a, c, st);
    case 6: return go<T, 6>(dag, a, c, st);
    case 4: return go<T, 4>(dag, a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply_staggered(int prec, bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
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
