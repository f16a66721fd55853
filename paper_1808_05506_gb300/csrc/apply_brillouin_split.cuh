// Brillouin sweeps of the split inner solve (Sec. 5, Eqs. def_bril, def_der,
// def_lap at c_SW = 0): FP32 links W (all 80 directions stored per site, link
// format 1) and FP32 arithmetic, with one of the two fields in 16 bits -- t(F32) = D p(16) for the search direction p, and
// s(16) = D^+ r(F32) for the residual r.  The product t is exact to FP32 for
// the 16-bit p that also updates the solution, so the recursive residual of
// the inner CGLS stays the true one.  Included by one translation unit per
// 16-bit type, each with its own copy of the direction table in constant
// memory (uploaded by brillouin_split_prepare before any capture).
#pragma once

#include <mutex>

#include "dirac_internal.h"

namespace dirac {
namespace {

static __constant__ BriDir c_split_dirs[80];

template <typename TI, typename TO, int R, bool DAG>
__global__ void __launch_bounds__(256) k_bri_split(ApplyArgs a, int ngroups)
{
    const long b = blockIdx.x;
    const int group = (int)(b % ngroups);
    const long p = (b / ngroups) * blockDim.x + threadIdx.x;
    if (p >= a.nsites) return;
    brillouin_site<float, R, DAG, 1, TI, TO>(a, slab_site(a, p), group, c_split_dirs);
}

template <typename TI, typename TO, int R, bool DAG>
__global__ void __launch_bounds__(192, 2) k_bri_split_groups(ApplyArgs a, int ngroups, int gy)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    const long p = (b / nchunks) * blockDim.x + threadIdx.x;
    if (p >= a.nsites || group >= ngroups) return;
    brillouin_site<float, R, DAG, 1, TI, TO>(a, slab_site(a, p), group, c_split_dirs);
}

static cudaError_t split_table(cudaStream_t st)
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    BriDir dirs[80];
    int reps[40];
    brillouin_tables(dirs, reps);
    e = cudaMemcpyToSymbolAsync(c_split_dirs, dirs, sizeof(dirs), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <typename TI, typename TO, int R, bool DAG>
static cudaError_t split_go(const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    const int ngroups = (a.Nv + R - 1) / R;
    if (c.variant == V_GROUPS && c.block <= 64) {
        const int gy = groups_per_block(c.block, ngroups);
        const long nb = ((a.nsites + c.block - 1) / c.block) * (long)((ngroups + gy - 1) / gy);
        k_bri_split_groups<TI, TO, R, DAG><<<(unsigned)nb, dim3(c.block, gy), 0, st>>>(a, ngroups, gy);
    } else {
        const int block = (c.block >= 32 && c.block <= 256 && c.block % 32 == 0) ? c.block : 128;
        const long nblk = ((a.nsites + block - 1) / block) * (long)ngroups;
        k_bri_split<TI, TO, R, DAG><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    }
    return cudaGetLastError();
}

// dag = false: a.in 16-bit (H), a.out FP32; dag = true: a.in FP32, a.out 16-bit;
// a.links FP32 W, 80 directions per site; R = min(c.R, 3)
template <typename H>
static cudaError_t split_launch(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    if (c.R >= 3) return dag ? split_go<float, H, 3, true>(a, c, st) : split_go<H, float, 3, false>(a, c, st);
    if (c.R == 2) return dag ? split_go<float, H, 2, true>(a, c, st) : split_go<H, float, 2, false>(a, c, st);
    return dag ? split_go<float, H, 1, true>(a, c, st) : split_go<H, float, 1, false>(a, c, st);
}

}  // namespace
}  // namespace dirac
