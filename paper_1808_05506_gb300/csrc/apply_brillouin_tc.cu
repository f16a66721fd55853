// Brillouin sweep on the tensor cores (tcgen05), for BF16 and FP16 storage:
// launch variant 7.  Sec. 5, Eqs. def_bril, def_der, def_lap at c_SW = 0:
//   D_B psi(x) = (m0 + 15/8) psi(x)
//                + sum_{d != 0} W_d(x) [rho_k (d . gamma) - lambda_k / 2] psi(x + d).
// The colour and spin factors commute, so with the five coefficient classes
//   C_0(d) = -lambda_k / 2,   C_{1+mu}(d) = rho_k d_mu  (k = |d|_1),
// and T_j[c][(s, v)] = sum_{d, c'} C_j(d) W_d(x)[c][c'] psi_v(x + d)[s][c'],
//   D_B psi_v(x)[s] = (m0 + 15/8) psi_v(x)[s] + T_0[s] + sum_mu (gamma_mu T_{1+mu})[s].
// Per site the T_j are one complex product [(s, v)] x [(d, c')] . [(d, c')] x [(j, c)],
// written as a real one: with X = psi (rows (s, v)), Y = C_j W (columns (j, c)),
//   D_re = sum X_re Y_re - X_im Y_im,   D_im = sum X_re Y_im + X_im Y_re,
// the A operand holds X with K = (d, c', re/im) -- exactly the storage order of a
// 16-bit spinor, so the gathered neighbour words are copied into shared memory
// unchanged -- and the B operand holds, for output column (j, c, re), the pairs
// (Y_re, -Y_im) and for (j, c, im) the pairs (Y_im, Y_re).  M = 64 rows (4 spins x
// 16 right-hand sides), N = 32 columns (30 used), K = 480 (80 directions x 3
// colours x 2): 30 tcgen05.mma of K = 16 per site and block of 16 right-hand
// sides, BF16 or FP16 operands, FP32 accumulation in tensor memory.  The spin
// matrices gamma_mu (chiral basis) and the diagonal term are applied in the
// epilogue on CUDA cores; D^+ = gamma5 D gamma5 negates the rho classes.
// Every W is read at the site itself (link format 1: all 80 stored).
//
// Shared-memory operands use the canonical no-swizzle K-major layout: core
// matrices of 8 rows x 16 bytes (8 elements), the K-adjacent core matrices 128 B
// apart (the descriptor's leading byte offset) and the 8-row groups K / 8 x
// 128 B apart (its stride byte offset).  The M = 64 accumulator puts row m in
// tensor-memory lane (m / 16) * 32 + m % 16.
#include <algorithm>
#include <mutex>

#include "dirac.h"
#include "dirac_internal.h"

namespace dirac {
namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_VB = 16;                     // right-hand sides per work item
constexpr int TC_M = 4 * TC_VB;               // 64 rows (spin, right-hand side)
constexpr int TC_N = 32;                      // 5 classes x 3 colours x (re, im) = 30, padded
constexpr int TC_K = 480;                     // 80 directions x 3 colours x (re, im)
constexpr uint32_t TC_SBO = (TC_K / 8) * 128; // bytes between 8-row groups
constexpr uint32_t TC_A_BYTES = (TC_M / 8) * TC_SBO;   // 61440
constexpr uint32_t TC_B_BYTES = (TC_N / 8) * TC_SBO;   // 30720
constexpr uint32_t TC_T_BYTES = 4 * TC_VB * TC_N * 4;  // accumulators staged for the epilogue
constexpr size_t TC_SMEM = TC_A_BYTES + TC_B_BYTES + TC_T_BYTES + 16;
constexpr int TC_MAX_WAIT = 1 << 24;          // bounded mbarrier wait: iterations ...
constexpr unsigned long long TC_MAX_NS = 500000000ull;   // ... and half a second

struct TcDir {
    signed char d[4];
    int plane;       // W plane at the site (link format 1: rep, or 40 + rep)
    float c[5];      // C_0 .. C_4 of this direction
};
static __constant__ TcDir c_tc_dirs[80];

// byte offset of element (row r, k) of an operand in the core-matrix layout
__device__ __forceinline__ uint32_t tc_off(int r, int k)
{
    return (uint32_t)(r >> 3) * TC_SBO + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// wait for the completion of phase `parity` of the mbarrier, for at most
// TC_MAX_WAIT polls and TC_MAX_NS nanoseconds; true if it completed
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity)
{
    const unsigned long long t0 = tc_clock_ns();
    for (int it = 0; it < TC_MAX_WAIT; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(parity));
        if (done) return true;
        if ((it & 255) == 255 && tc_clock_ns() - t0 > TC_MAX_NS) return false;
    }
    return false;
}

// shared-memory matrix descriptor: no swizzle, leading byte offset 128 (K),
// stride byte offset TC_SBO (8-row groups), descriptor version 1
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(TC_SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

template <typename T> struct TcFmt;
template <> struct TcFmt<__nv_bfloat16> { static constexpr uint32_t v = 1; };
template <> struct TcFmt<__half> { static constexpr uint32_t v = 0; };

// instruction descriptor of kind::f16: FP32 accumulator, A and B of type T,
// both K-major, N = 32, M = 64
template <typename T> __device__ __forceinline__ uint32_t tc_idesc()
{
    return (1u << 4) | (TcFmt<T>::v << 7) | (TcFmt<T>::v << 10) | ((uint32_t)(TC_N >> 3) << 17) |
           ((uint32_t)(TC_M >> 4) << 24);
}

// (gamma_mu t)_sp for the chiral basis gamma_mu = [[0, B_mu], [B_mu^+, 0]],
// B_1 = -i s_x, B_2 = -i s_y, B_3 = -i s_z, B_4 = 1
__device__ __forceinline__ cx<float> gamma_row(int mu, int sp, const cx<float> (&t)[4])
{
    switch (mu) {
    case 0:   // B = [[0, -i], [-i, 0]], B^+ = [[0, i], [i, 0]]
        if (sp == 0) return times_mi(t[3]);
        if (sp == 1) return times_mi(t[2]);
        if (sp == 2) return times_i(t[1]);
        return times_i(t[0]);
    case 1:   // B = [[0, -1], [1, 0]], B^+ = [[0, 1], [-1, 0]]
        if (sp == 0) return -t[3];
        if (sp == 1) return t[2];
        if (sp == 2) return t[1];
        return -t[0];
    case 2:   // B = [[-i, 0], [0, i]], B^+ = [[i, 0], [0, -i]]
        if (sp == 0) return times_mi(t[2]);
        if (sp == 1) return times_i(t[3]);
        if (sp == 2) return times_i(t[0]);
        return times_mi(t[1]);
    default:  // B = 1
        if (sp == 0) return t[2];
        if (sp == 1) return t[3];
        if (sp == 2) return t[0];
        return t[1];
    }
}

// One CTA of 128 threads walks work items (site, block of 16 right-hand sides)
// with a stride of gridDim.x: builds the A and B operands in shared memory,
// thread 0 issues the 30 MMAs and commits them to an mbarrier, every thread
// waits (bounded), the 4 warps read their accumulator lanes, and 64 threads
// apply the spin matrices and the diagonal and store.
template <typename T, bool DAG>
__global__ void __launch_bounds__(TC_THREADS) k_brillouin_tc(ApplyArgs a, int nvb)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* As = tc_smem;
    unsigned char* Bs = tc_smem + TC_A_BYTES;
    float* Ts = reinterpret_cast<float*>(tc_smem + TC_A_BYTES + TC_B_BYTES);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_smem + TC_A_BYTES + TC_B_BYTES + TC_T_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_smem + TC_A_BYTES + TC_B_BYTES + TC_T_BYTES + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const long nitems = a.nsites * (long)nvb;
    uint32_t phase = 0;
    bool ok = true;
    for (long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const long p = item / nvb;
        const int vb0 = (int)(item - p * nvb) * TC_VB;
        const long s = slab_site(a, p);
        long fwd[4], bwd[4];
        int x[4];
        site_offsets(a.g, s, fwd, bwd, x);
        // A: row (spin, vv), K (d, c', re/im) = the spinor's own 32-bit words
        for (int idx = tid; idx < TC_VB * 80; idx += TC_THREADS) {
            const int vv = idx / 80, dd = idx - vv * 80;
            const int v = vb0 + vv;
            if (v >= a.Nv) continue;   // rows of absent right-hand sides are not stored
            const TcDir& D = c_tc_dirs[dd];
            long nb = s;
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) nb += D.d[mu] > 0 ? fwd[mu] : (D.d[mu] < 0 ? bwd[mu] : 0);
            uint32_t w[12];
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const uint4 q = ld_ro(reinterpret_cast<const uint4*>(a.in) + blk_index(a.g.vol, 3, v, kk, nb));
                w[4 * kk] = q.x;
                w[4 * kk + 1] = q.y;
                w[4 * kk + 2] = q.z;
                w[4 * kk + 3] = q.w;
            }
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    *reinterpret_cast<uint32_t*>(As + tc_off(sp * TC_VB + vv, 6 * dd + 2 * c)) = w[3 * sp + c];
        }
        // B: column (j, c, re/im), K (d, c', re/im), from W_d(x) and the class coefficients
        for (int idx = tid; idx < 80 * 3; idx += TC_THREADS) {
            const int dd = idx / 3, c = idx - dd * 3;
            const TcDir& D = c_tc_dirs[dd];
            cx<float> Wr[3];
#pragma unroll
            for (int cp = 0; cp < 3; ++cp) Wr[cp] = ld_one<T>(a.links, blk_index(a.g.vol, 9, D.plane, 3 * c + cp, s));
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float cj = (DAG && j > 0) ? -D.c[j] : D.c[j];
                const int n = (j * 3 + c) * 2;
#pragma unroll
                for (int cp = 0; cp < 3; ++cp) {
                    const cx<float> y{cj * Wr[cp].re, cj * Wr[cp].im};
                    *reinterpret_cast<uint32_t*>(Bs + tc_off(n, 6 * dd + 2 * cp)) = pack2(cx<float>{y.re, -y.im}, (T*)nullptr);
                    *reinterpret_cast<uint32_t*>(Bs + tc_off(n + 1, 6 * dd + 2 * cp)) = pack2(cx<float>{y.im, y.re}, (T*)nullptr);
                }
            }
        }
        // the generic-proxy stores must be visible to the tensor cores' reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t idesc = tc_idesc<T>();
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll 1
            for (int t = 0; t < TC_K / 16; ++t) {
                const uint64_t ad = tc_desc(a0 + 256u * t), bd = tc_desc(b0 + 256u * t);
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(t));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(mbar)));
        }
        const bool done = tc_wait(smem_u32(mbar), phase);
        // one decision for the whole CTA (every thread takes the same path to the barriers below)
        if (!__syncthreads_and((int)done)) {
            // the MMAs did not complete: record it, give them a second bounded
            // wait before tensor memory is freed below, and stop
            if (tid == 0) {
                if (a.err) atomicExch(a.err, (int)DIRAC_TIMEOUT);
                tc_wait(smem_u32(mbar), phase);
            }
            __syncthreads();
            ok = false;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) {
            // warp w holds spin w: rows w * 16 + vv in lanes 32 w + vv, vv < 16
            uint32_t r[32];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                           "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                           "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (lane < TC_VB) {
#pragma unroll
                for (int n = 0; n < 30; ++n) Ts[(warp * TC_VB + lane) * TC_N + n] = __uint_as_float(r[n]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (ok && tid < 4 * TC_VB) {
            const int sp = tid / TC_VB, vv = tid - sp * TC_VB, v = vb0 + vv;
            if (v < a.Nv) {
                const float dg = a.diag_vf ? a.diag_vf[v] : (a.diag_v ? (float)a.diag_v[v] : a.diagf);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    auto tj = [&](int j, int sp2) {
                        const float* q = Ts + (sp2 * TC_VB + vv) * TC_N + (j * 3 + c) * 2;
                        return cx<float>{q[0], q[1]};
                    };
                    cx<float> o = tj(0, sp);
#pragma unroll
                    for (int mu = 0; mu < 4; ++mu) {
                        const cx<float> t4[4] = {tj(1 + mu, 0), tj(1 + mu, 1), tj(1 + mu, 2), tj(1 + mu, 3)};
                        o = o + gamma_row(mu, sp, t4);
                    }
                    // complex i = 3 sp + c of the 16-bit field: component i % 4 of its 16-byte element i / 4
                    const int i = 3 * sp + c;
                    const size_t ei = blk_index(a.g.vol, 3, v, i >> 2, s) * 4 + (i & 3);
                    const cx<float> pc = ld_one<T>(a.in, ei);
                    o.re = fmaf(dg, pc.re, o.re);
                    o.im = fmaf(dg, pc.im, o.im);
                    st_one<T>(a.out, ei, o);
                }
            }
        }
        __syncthreads();   // the operands and the staged accumulators are reused by the next item
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

template <typename T>
cudaError_t tc_go(bool dag, const ApplyArgs& a, cudaStream_t st)
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 128;
    }
    auto kern = dag ? k_brillouin_tc<T, true> : k_brillouin_tc<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (e != cudaSuccess) return e;
    const int nvb = (a.Nv + TC_VB - 1) / TC_VB;
    const long nitems = a.nsites * (long)nvb;
    const long grid = std::min<long>(nitems, 2L * nsm);   // two CTAs per SM (~100 KB of shared memory each)
    if (grid <= 0) return cudaSuccess;
    kern<<<(unsigned)grid, TC_THREADS, TC_SMEM, st>>>(a, nvb);
    return cudaGetLastError();
}

}  // namespace

// the direction table of the tensor-core sweep (once per device, before any capture)
cudaError_t brillouin_tc_prepare(cudaStream_t st)
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
    static const double rho[5] = {0.0, 64.0 / 432.0, 16.0 / 432.0, 4.0 / 432.0, 1.0 / 432.0};
    TcDir t[80];
    for (int j = 0; j < 80; ++j) {
        int k = 0;
        for (int mu = 0; mu < 4; ++mu) {
            t[j].d[mu] = dirs[j].d[mu];
            k += dirs[j].d[mu] != 0;
        }
        t[j].plane = dirs[j].neg ? 40 + dirs[j].rep : dirs[j].rep;
        t[j].c[0] = (float)dirs[j].a;   // -lambda_k / 2
        for (int mu = 0; mu < 4; ++mu) t[j].c[1 + mu] = (float)(rho[k] * dirs[j].d[mu]);
    }
    e = cudaMemcpyToSymbolAsync(c_tc_dirs, t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

// a.links: the 80 W per site (link format 1) in the storage type; a.in, a.out
// 16-bit fields of the storage type
cudaError_t launch_brillouin_tc(int prec, bool dag, const ApplyArgs& a, cudaStream_t st)
{
    if (a.nsites == 0 || a.Nv == 0) return cudaSuccess;
    if (prec == P_BF16) return tc_go<__nv_bfloat16>(dag, a, st);
    if (prec == P_F16) return tc_go<__half>(dag, a, st);
    return cudaErrorInvalidValue;
}

}  // namespace dirac
