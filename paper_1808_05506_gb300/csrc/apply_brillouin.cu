// Brillouin D_B and D_B^+ sweeps (Sec. 5, Eqs. def_bril, def_der, def_lap at
// c_SW = 0) on the internal blocked layout.  One thread owns one site
// and R right-hand sides and walks the 80 off-centre directions; each stored
// link W (Tab. tab:off-axis) is loaded once per thread and applied to its R
// spinors from registers.  The direction table sits in constant memory, read
// with a warp-uniform index.
#include <cstring>
#include <type_traits>
#include <mutex>

#include "dirac_df.cuh"
#include "dirac_internal.h"

namespace dirac {

__constant__ BriDir c_bri_dirs[80];

// LF: 0 the 40 stored links, 1 all 80 directions stored at each site
template <typename T, int R, bool DAG, int LF>
__global__ void __launch_bounds__(256) k_brillouin(ApplyArgs a, int ngroups)
{
    const long b = blockIdx.x;
    const int group = (int)(b % ngroups);
    const long p = (b / ngroups) * blockDim.x + threadIdx.x;
    if (p >= a.nsites) return;
    brillouin_site<T, R, DAG, LF>(a, slab_site(a, p), group, c_bri_dirs);
}

// V_GROUPS: blockDim = (sites, groups); block b covers a run of sites and a
// chunk of gy right-hand-side groups
template <typename T, int R, bool DAG, int LF>
__global__ void __launch_bounds__(192, 2) k_brillouin_groups(ApplyArgs a, int ngroups, int gy)
{
    const int nchunks = (ngroups + gy - 1) / gy;
    const long b = blockIdx.x;
    const int group = (int)(b % nchunks) * gy + threadIdx.y;
    const long p = (b / nchunks) * blockDim.x + threadIdx.x;
    if (p >= a.nsites || group >= ngroups) return;
    brillouin_site<T, R, DAG, LF>(a, slab_site(a, p), group, c_bri_dirs);
}

template <typename T, int R, int LF>
static cudaError_t go_lf(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    const int block = c.block;
    const int ngroups = (a.Nv + R - 1) / R;
    if (c.variant == V_GROUPS) {
        const int gy = groups_per_block(block, ngroups);
        const long nb = ((a.nsites + block - 1) / block) * (long)((ngroups + gy - 1) / gy);
        if (dag) k_brillouin_groups<T, R, true, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
        else k_brillouin_groups<T, R, false, LF><<<(unsigned)nb, dim3(block, gy), 0, st>>>(a, ngroups, gy);
        return cudaGetLastError();
    }
    const long nblk = ((a.nsites + block - 1) / block) * (long)ngroups;
    if (dag) k_brillouin<T, R, true, LF><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    else k_brillouin<T, R, false, LF><<<(unsigned)nblk, block, 0, st>>>(a, ngroups);
    return cudaGetLastError();
}

template <typename T, int R>
static cudaError_t go(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    return c.fmt == 1 ? go_lf<T, R, 1>(dag, a, c, st) : go_lf<T, R, 0>(dag, a, c, st);
}

template <typename T>
static cudaError_t go_T(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    if (c.variant == V_TC) {
        // tensor cores: 16-bit storage with all 80 W stored per site
        if (sizeof(T) != 2 || c.fmt != 1) return cudaErrorInvalidValue;
        return launch_brillouin_tc(sizeof(T) == 2 && std::is_same<T, __half>::value ? P_F16 : P_BF16, dag, a, st);
    }
    if (c.variant != V_DIRECT && c.variant != V_GROUPS) return cudaErrorInvalidValue;
    switch (c.R) {
    case 1: return go<T, 1>(dag, a, c, st);
    case 2: return go<T, 2>(dag, a, c, st);
    case 3: return go<T, 3>(dag, a, c, st);
    case 4: return go<T, 4>(dag, a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply_brillouin(int prec, bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    switch (prec) {
    case P_F64: return go_T<double>(dag, a, c, st);
    case P_F32: return go_T<float>(dag, a, c, st);
    case P_BF16: return go_T<__nv_bfloat16>(dag, a, c, st);
    case P_F16: return go_T<__half>(dag, a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

// Direction table.  For dir != 0 with k = |dir|_1 nonzero components:
//   spin matrix rho_k (dir . gamma) - lambda_k/2 = [[a, rho_k Q], [rho_k Q^+, a]],
//   Q = sum_mu dir_mu B_mu, B_1 = -i sigma_1, B_2 = -i sigma_2, B_3 = -i sigma_3, B_4 = 1,
//   so Q = [[d_t - i d_z, -i d_x - d_y], [-i d_x + d_y, d_t + i d_z]].
// rho = (64, 16, 4, 1)/432 and lambda = (-240, 8, 4, 2, 1)/64 (the coefficient
// line of Sec. 5).  The stored representative of +-dir is the one whose first
// nonzero component is positive; W_dir(x) = W_{-dir}(x+dir)^+ for the others.
void brillouin_tables(BriDir dirs[80], int rep_dir81[40])
{
    static const double rho[5] = {0.0, 64.0 / 432.0, 16.0 / 432.0, 4.0 / 432.0, 1.0 / 432.0};
    static const double lam[5] = {-240.0 / 64.0, 8.0 / 64.0, 4.0 / 64.0, 2.0 / 64.0, 1.0 / 64.0};
    int nrep = 0;
    int rep_of[81];
    for (int c = 0; c < 81; ++c) rep_of[c] = -1;
    for (int c = 0; c < 81; ++c) {
        int d[4] = {c % 3 - 1, (c / 3) % 3 - 1, (c / 9) % 3 - 1, (c / 27) % 3 - 1};
        int first = 0;
        for (int mu = 0; mu < 4 && !first; ++mu) first = d[mu];
        if (first > 0) {
            rep_of[c] = nrep;
            rep_dir81[nrep++] = c;
        }
    }
    int j = 0;
    for (int c = 0; c < 81; ++c) {
        int d[4] = {c % 3 - 1, (c / 3) % 3 - 1, (c / 9) % 3 - 1, (c / 27) % 3 - 1};
        int k = 0, first = 0;
        for (int mu = 0; mu < 4; ++mu) {
            k += d[mu] != 0;
            if (!first) first = d[mu];
        }
        if (k == 0) continue;
        BriDir& D = dirs[j++];
        for (int mu = 0; mu < 4; ++mu) D.d[mu] = (signed char)d[mu];
        int mc = 80 - c;  // dir81 code of -dir
        D.neg = first < 0;
        D.rep = (signed char)(first > 0 ? rep_of[c] : rep_of[mc]);
        D.a = -0.5 * lam[k];
        const double r = rho[k];
        const double dx = d[0], dy = d[1], dz = d[2], dt = d[3];
        D.q[0] = (r * dt);  D.q[1] = (r * -dz);   // Q00
        D.q[2] = (r * -dy); D.q[3] = (r * -dx);   // Q01
        D.q[4] = (r * dy);  D.q[5] = (r * -dx);   // Q10
        D.q[6] = (r * dt);  D.q[7] = (r * dz);    // Q11
        D.af = (float)D.a;
        for (int e = 0; e < 8; ++e) D.qf[e] = (float)D.q[e];
    }
}

cudaError_t upload_brillouin_table(cudaStream_t st)
{
    // once per device: the constant bank is per device
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
    e = cudaMemcpyToSymbolAsync(c_bri_dirs, dirs, sizeof(dirs), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

// double-float residual sweep (dirac_df.cuh): one thread per (site, right-hand
// side), the DF_COLS right-hand sides of a block sharing its W through L1
__global__ void __launch_bounds__(DF_SITES * DF_COLS) k_brillouin_df(ApplyArgs a)
{
    const int ncb = (a.Nv + DF_COLS - 1) / DF_COLS;
    const long b = blockIdx.x;
    const int v = (int)(b % ncb) * DF_COLS + threadIdx.y;
    const long p = (b / ncb) * DF_SITES + threadIdx.x;
    if (p >= a.nsites || v >= a.Nv) return;
    brillouin_site<f64df, 1, false>(a, slab_site(a, p), v, c_bri_dirs);
}

cudaError_t launch_brillouin_df(const ApplyArgs& a, cudaStream_t st)
{
    cudaError_t e = upload_brillouin_table(st);
    if (e != cudaSuccess) return e;
    const long nb = ((a.nsites + DF_SITES - 1) / DF_SITES) * (long)((a.Nv + DF_COLS - 1) / DF_COLS);
    k_brillouin_df<<<(unsigned)nb, dim3(DF_SITES, DF_COLS), 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dirac
