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
// the A operand holds X with K = (d, c', re/im) -- the storage order of a 16-bit
// spinor, so the gathered neighbour words are copied into shared memory
// unchanged -- and the B operand holds, for output column (j, c, re), the pairs
// (Y_re, -Y_im) and for (j, c, im) the pairs (Y_im, Y_re).  M = 64 rows (4 spins x
// 16 right-hand sides), N = 32 columns (30 used), BF16 or FP16 operands, FP32
// accumulation in tensor memory.  The spin matrices gamma_mu (chiral basis) and
// the diagonal term are applied in the epilogue on CUDA cores; D^+ = gamma5 D
// gamma5 negates the rho classes.  Every W is read at the site itself (link
// format 1: all 80 stored).
//
// A CTA walks whole x-rows of the lattice.  The K dimension is split into three
// blocks by d_x = -1, 0, +1, and each block into the 27 directions (d_y, d_z,
// d_t) x 3 colours x (re, im) = 162 elements, padded to 176 (11 MMAs of K = 16).
// The A block of d_x only depends on the x-coordinate p = x + d_x of the
// neighbours, so one A slot per x-position p (27 neighbour spinors per rhs)
// serves the three sites x = p + 1, p, p - 1 (as their d_x = -1, 0, +1 block):
// one chain of 11 MMAs with N = 96 columns, B = [B(p - 1, d_x = +1), B(p, 0),
// B(p + 1, -1)], adds to the accumulators of the three sites at once.  The B
// blocks sit in a ring of entries, entry p holding exactly those three, so each
// site's builder writes its three blocks into three consecutive entries.  The
// accumulators form a ring of 16 x 32 tensor-memory columns (all 512), one per
// site; a chain whose sites wrap around the ring is split in two.  An MMA
// always accumulates: the epilogue clears each accumulator after reading it.
// At the ends of a row a slot serves only the sites that exist (N = 32 or 64).
//
// The CTA is warp-specialised, its roles linked by mbarriers (every wait
// bounded in time; a wait that runs out stops the whole CTA and records
// DIRAC_TIMEOUT):
//   warps 0-3   epilogue: accumulator -> registers (each warp its lane
//               quadrant = one spin), clear, spin matrices, diagonal, store;
//   warp 4      one thread issues the MMA chains and commits them to the
//               barriers that free the A slot and the B entry and hand
//               completed accumulators to the epilogue;
//   warps 5-12  fill the A slots two x-positions at a time (adjacent lanes
//               load the adjacent 16-byte pieces of the two sites, one 32-byte
//               sector), the loads issued before waiting for the slots;
//   warps 13-20 the B blocks of each site from its 80 W (thread = direction x
//               colour row, both re/im rows), the links of the next site loaded
//               while the current one is built; the blocks for d_x = -1, 0 go
//               first, so that the entry they complete is ready while the one
//               for d_x = +1 still waits for its entry to be free.
// The B entries C_j(d) W are formed in the storage arithmetic (packed 16-bit
// multiplies, rounded to nearest): C_0 = -lambda_k / 2 is a power of two, so
// that product is exact; rho_k is rounded to the storage type first, which
// keeps the rho classes within two units in the last place of C_j W.
// The padding of K, the d = 0 entries of B, the entries of the classes that
// vanish for a direction (d_mu = 0) and the rows of absent right-hand sides
// stay zero from the start.
//
// Shared-memory operands use the canonical no-swizzle K-major layout: core
// matrices of 8 rows x 16 bytes (8 elements), the K-adjacent core matrices 128 B
// apart (the descriptor's leading byte offset) and the 8-row groups 22 x 128 B
// apart (its stride byte offset).  The M = 64 accumulator puts row m in
// tensor-memory lane (m / 16) * 32 + m % 16.
#include <algorithm>
#include <mutex>

#include "dirac.h"
#include "dirac_internal.h"

namespace dirac {
namespace {

constexpr int TC_VB = 16;                               // right-hand sides per work item
constexpr int TC_M = 4 * TC_VB;                         // 64 rows (spin, right-hand side)
constexpr int TC_N = 32;                                // per site: 5 classes x 3 colours x (re, im) = 30, padded
constexpr int TC_KS = 176;                              // K of one slot: 27 x 3 x 2 = 162, padded
constexpr int TC_KSTEPS = TC_KS / 16;                   // MMAs per chain
constexpr uint32_t TC_SBO = (TC_KS / 8) * 128;          // bytes between 8-row groups (2816)
constexpr uint32_t TC_ASLOT = (TC_M / 8) * TC_SBO;      // one A slot (22528 B)
constexpr uint32_t TC_BBLK = (TC_N / 8) * TC_SBO;       // one site's block of B (11264 B)
constexpr uint32_t TC_BENT = 3 * TC_BBLK;               // one B entry (33792 B)
constexpr int TC_NS = 4;                                // A slots
constexpr int TC_NR = 3;                                // B entries
constexpr int TC_NACC = 16;                             // accumulators (512 columns)
constexpr int TC_TS = 25;                               // staged row stride (floats): classes 1..4
constexpr uint32_t TC_TBUF = TC_M * TC_TS * 4;          // one staging buffer (6400 B)
constexpr uint32_t TC_A_OFF = 0;
constexpr uint32_t TC_B_OFF = TC_A_OFF + TC_NS * TC_ASLOT;   // 90112
constexpr uint32_t TC_T_OFF = TC_B_OFF + TC_NR * TC_BENT;    // 191488
constexpr uint32_t TC_BAR_OFF = TC_T_OFF + 2 * TC_TBUF;      // 204288
// barriers: full / empty A slot, full / empty B entry, full / empty accumulator, drain
constexpr int TC_BAR_FA = 0, TC_BAR_EA = TC_NS, TC_BAR_FB = 2 * TC_NS, TC_BAR_EB = 2 * TC_NS + TC_NR,
              TC_BAR_FC = 2 * TC_NS + 2 * TC_NR, TC_BAR_EC = TC_BAR_FC + TC_NACC, TC_BAR_DR = TC_BAR_EC + TC_NACC,
              TC_NBARS = TC_BAR_DR + 1;
constexpr size_t TC_SMEM = TC_BAR_OFF + 8 * TC_NBARS + 16;
constexpr int TC_EPI_WARPS = 4, TC_MMA_WARP = 4, TC_GATHER_WARP0 = 5, TC_B_WARP0 = 13, TC_WARPS = 21;
constexpr int TC_THREADS = TC_WARPS * 32;
constexpr int TC_BTHREADS = (TC_WARPS - TC_B_WARP0) * 32;    // 256 B builders, 240 with work
constexpr int TC_GTHREADS = (TC_B_WARP0 - TC_GATHER_WARP0) * 32;   // 256 gatherers
constexpr int TC_GROUNDS = 28;                          // gather rounds of a pair: 2 x 8 rhs x 14 x 2 directions
constexpr int TC_GPT = (TC_GROUNDS + 7) / 8;            // gather rounds per thread (8 warps)
constexpr int TC_MAX_WAIT = 1 << 24;                    // bounded mbarrier wait: polls ...
constexpr unsigned long long TC_MAX_NS = 500000000ull;  // ... and half a second
constexpr uint32_t TC_SUSPEND_NS = 20000;               // suspend-time hint of one poll

static_assert(TC_SMEM <= 227 * 1024, "shared memory of one CTA");
static_assert((TC_BAR_OFF & 7) == 0, "mbarrier alignment");

// the 80 directions ordered by d_x block, then rest index (bank-friendly B stores)
struct TcDir {
    signed char g;   // d_x + 1
    signed char r;   // rest index (d_y + 1) + 3 (d_z + 1) + 9 (d_t + 1)
    short plane;     // W plane at the site (link format 1: rep, or 40 + rep)
    float c0;        // C_0 = -lambda_k / 2
    float rho;       // rho_k: C_{1+mu} = rho_k d_mu
    int nz;          // bit mu: d_mu != 0
    int neg;         // bit mu: d_mu < 0
};
static __constant__ TcDir c_tc_dirs[80];

// byte offset of element (row, k) of one K block in the core-matrix layout
__device__ __forceinline__ uint32_t tc_off(int row, int k)
{
    return (uint32_t)(row >> 3) * TC_SBO + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// wait for the completion of phase `parity` of the mbarrier, for at most
// TC_MAX_WAIT polls and TC_MAX_NS nanoseconds, and only while no other role of
// the CTA has given up (*abort); true if it completed.  A wait that runs out
// sets *abort, so that every other role stops at its next wait.
__device__ __noinline__ bool tc_wait_slow(uint32_t bar, uint32_t parity, volatile int* abort)
{
    const unsigned long long t0 = tc_clock_ns();
    for (int it = 0; it < TC_MAX_WAIT; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(parity), "r"(TC_SUSPEND_NS) : "memory");
        if (done) return true;
        if ((it & 7) == 7) {
            if (*abort) return false;
            if (tc_clock_ns() - t0 > TC_MAX_NS) break;
        }
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int* abort)
{
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done ? true : tc_wait_slow(bar, parity, abort);
}

// shared memory by 32-bit address (an immediate offset where the call gives one)
template <int OFF = 0> __device__ __forceinline__ void tc_sts32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0+%2], %1;" ::"r"(a), "r"(v), "n"(OFF));
}
__device__ __forceinline__ void tc_sts64(uint32_t a, uint32_t v0, uint32_t v1)
{
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(v0), "r"(v1));
}
__device__ __forceinline__ float tc_ldsf(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void tc_stsf(uint32_t a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v)); }

// packed 16-bit product, rounded to nearest
__device__ __forceinline__ uint32_t tc_mul2(uint32_t x, uint32_t y, __nv_bfloat16*)
{
    const __nv_bfloat162 r = __hmul2(*reinterpret_cast<const __nv_bfloat162*>(&x), *reinterpret_cast<const __nv_bfloat162*>(&y));
    return *reinterpret_cast<const uint32_t*>(&r);
}
__device__ __forceinline__ uint32_t tc_mul2(uint32_t x, uint32_t y, __half*)
{
    const __half2 r = __hmul2(*reinterpret_cast<const __half2*>(&x), *reinterpret_cast<const __half2*>(&y));
    return *reinterpret_cast<const uint32_t*>(&r);
}

__device__ __forceinline__ void tc_bar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void tc_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_arrive_n(uint32_t bar, uint32_t n)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(n) : "memory");
}

// the mbarrier receives one arrival when every MMA this thread issued so far is complete
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// the generic-proxy shared-memory stores of this thread become visible to the tensor cores
__device__ __forceinline__ void tc_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// barrier 1 over the 128 epilogue threads, and of their flags
__device__ __forceinline__ bool tc_epi_and(bool v)
{
    int r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.s32 p, %1, 0;\nbar.red.and.pred q, 1, 128, p;\nselp.s32 %0, 1, 0, q;\n}"
                 : "=r"(r) : "r"((int)v) : "memory");
    return r != 0;
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
// both K-major, N columns, M = 64
template <typename T> __device__ __forceinline__ uint32_t tc_idesc(int n)
{
    return (1u << 4) | (TcFmt<T>::v << 7) | (TcFmt<T>::v << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(TC_M >> 4) << 24);
}

// complex element index of component i (= 3 spin + colour) of rhs v at site s
template <typename TO> __device__ __forceinline__ size_t tc_out_index(size_t vol, int v, int i, long s)
{
    constexpr int CPV = Store<TO>::CPV;
    return blk_index(vol, 12 / CPV, v, i / CPV, s) * CPV + i % CPV;
}

// The work schedule every role walks: items (x-row, block of 16 right-hand
// sides) blockIdx.x, blockIdx.x + gridDim.x, ...; per item Lx + 2 slot fills
// (positions -1 .. Lx) and Lx sites.
struct TcRow {
    long base;   // site of x = 0
    int vb0;     // first right-hand side of the block
};

__device__ __forceinline__ TcRow tc_row(const ApplyArgs& a, long item, int nvb)
{
    const long row = item / nvb;
    return TcRow{slab_site(a, row * (long)a.g.L[0]), (int)(item - row * nvb) * TC_VB};
}

// site of x-position q of the row (periodic, -1 <= q <= Lx)
__device__ __forceinline__ long tc_site_at(long base, int q, int Lx)
{
    int x = q;
    if (x < 0) x += Lx;
    if (x >= Lx) x -= Lx;
    return base + x;
}

// Gatherers (warps 5-12): the fills of a row are position -1, then the pairs
// (0, 1), (2, 3), ..., and what is left; lane bit 0 picks the position of the
// pair, bits 1..3 the rhs vv & 7 and bit 4 the rest index r & 1, rounds
// wr = warp + 8 k the rest (vv / 8 = wr & 1, r / 2 = wr / 2).
template <typename T>
__device__ void tc_gather_role(const ApplyArgs& a, int nvb, uint32_t As, uint32_t bars, volatile int* abort, int gwarp,
                               int lane)
{
    const int Lx = a.g.L[0];
    const long nitems = (a.nsites / Lx) * (long)nvb;
    const size_t nblk = nblk_of((size_t)a.g.vol);
    const int po = lane & 1;
    int g_r[TC_GPT], g_vv[TC_GPT];
    uint32_t g_sb[TC_GPT][3];   // slot offset of (spin 0, rhs vv) at the K of colour c
#pragma unroll
    for (int k = 0; k < TC_GPT; ++k) {
        const int wr = gwarp + 8 * k;
        g_r[k] = wr < TC_GROUNDS ? 2 * (wr >> 1) + (lane >> 4) : 27;   // 27: none
        g_vv[k] = ((lane >> 1) & 7) + 8 * (wr & 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) g_sb[k][c] = tc_off(g_vv[k], 6 * (g_r[k] < 27 ? g_r[k] : 0) + 2 * c);
    }
    long f0 = 0;
    bool ok = true;
    for (long item = blockIdx.x; item < nitems && ok; item += gridDim.x, f0 += Lx + 2) {
        const TcRow R = tc_row(a, item, nvb);
        long fwd[4], bwd[4];
        int xc[4];
        site_offsets(a.g, R.base, fwd, bwd, xc);
        long g_off[TC_GPT];
        size_t g_v[TC_GPT];
        bool g_on[TC_GPT];
#pragma unroll
        for (int k = 0; k < TC_GPT; ++k) {
            const int r = g_r[k];
            const int dy = r % 3 - 1, dz = (r / 3) % 3 - 1, dt = r / 9 - 1;
            g_off[k] = (dy > 0 ? fwd[1] : (dy < 0 ? bwd[1] : 0)) + (dz > 0 ? fwd[2] : (dz < 0 ? bwd[2] : 0)) +
                       (dt > 0 ? fwd[3] : (dt < 0 ? bwd[3] : 0));
            g_on[k] = r < 27 && R.vb0 + g_vv[k] < a.Nv;
            g_v[k] = (size_t)(R.vb0 + g_vv[k]) * nblk;
        }
        for (int p = -1; p <= Lx && ok;) {
            const int np = (p >= 0 && p + 1 <= Lx) ? 2 : 1;   // positions in this fill
            const bool lane_on = po < np;
            const long sq = tc_site_at(R.base, p + po, Lx);
            uint4 w[TC_GPT][3];
#pragma unroll
            for (int k = 0; k < TC_GPT; ++k) {
                if (!(g_on[k] && lane_on)) continue;
                const long nb = sq + g_off[k];
                const uint4* q = reinterpret_cast<const uint4*>(a.in) + (g_v[k] + (size_t)(nb >> 5)) * 96 + (nb & 31);
                w[k][0] = ld_ro(q);
                w[k][1] = ld_ro(q + 32);
                w[k][2] = ld_ro(q + 64);
            }
            const long F = f0 + p + 1;   // fill of position p
            for (int j = 0; j < np && ok; ++j)
                if (F + j >= TC_NS)
                    ok = tc_wait(bars + 8u * (TC_BAR_EA + (int)((F + j) % TC_NS)), (uint32_t)(((F + j) / TC_NS - 1) & 1), abort);
            if (!ok) break;
            const uint32_t S = As + (uint32_t)((F + po) % TC_NS) * TC_ASLOT;
#pragma unroll
            for (int k = 0; k < TC_GPT; ++k) {
                if (!(g_on[k] && lane_on)) continue;
                const uint32_t wv[12] = {w[k][0].x, w[k][0].y, w[k][0].z, w[k][0].w, w[k][1].x, w[k][1].y,
                                         w[k][1].z, w[k][1].w, w[k][2].x, w[k][2].y, w[k][2].z, w[k][2].w};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // rows spin * 16 + vv: 2 spin 8-row groups further down
                    const uint32_t at = S + g_sb[k][c];
                    tc_sts32<0>(at, wv[c]);
                    tc_sts32<2 * TC_SBO>(at, wv[3 + c]);
                    tc_sts32<4 * TC_SBO>(at, wv[6 + c]);
                    tc_sts32<6 * TC_SBO>(at, wv[9 + c]);
                }
            }
            tc_fence_async();
            for (int j = 0; j < np; ++j) tc_arrive(bars + 8u * (TC_BAR_FA + (int)((F + j) % TC_NS)));
            p += np;
        }
    }
    // tail: the last releases of the slots arrive before the CTA may exit
    if (ok && gwarp == 0 && lane == 0) {
        for (long g = f0 - TC_NS; g < f0; ++g)
            if (g >= 0 && !tc_wait(bars + 8u * (TC_BAR_EA + (int)(g % TC_NS)), (uint32_t)((g / TC_NS) & 1), abort)) break;
    }
}

// number of arrivals site x of a row of Lx sites brings to the B entry x + g:
// its own, plus those of the sites -2, -1 (site 0) or Lx, Lx + 1 (site Lx - 1)
// that do not exist, so that every entry completes with 3 arrivals per builder
__device__ __forceinline__ uint32_t tc_b_count(int x, int g, int Lx)
{
    const int e = x + g;
    uint32_t n = 1;
    if (x == 0) n += (uint32_t)max(0, 2 - e);
    if (x == Lx - 1) n += (uint32_t)max(0, e - (Lx - 1));
    return n;
}

// three consecutive words (colours c' = 0, 1, 2 of one direction) of one row of
// a B block: 6 r + 2 c' are element offsets along K, so for even r the first two
// words share an aligned 8-byte pair, for odd r the last two
__device__ __forceinline__ void tc_st3(uint32_t at, uint32_t ka, uint32_t kb, bool odd, uint32_t w0, uint32_t w1,
                                       uint32_t w2)
{
    if (!odd) {
        tc_sts64(at + ka, w0, w1);
        tc_sts32(at + kb, w2);
    } else {
        tc_sts32(at + ka, w0);
        tc_sts64(at + kb, w1, w2);
    }
}

// B builders (warps 13-20): thread t < 240 owns direction t / 3 (order of
// c_tc_dirs) and colour row c = t % 3, both its re and im rows; it reads the
// three words W_d(x)[c][c'] from the site-major copy (a warp's loads for a
// site are about 100 consecutive words).  Site x's block for d_x = g - 1 goes
// to sub-block 2 - g of the entry of fill f0 + x + g.  Only the classes that do
// not vanish for the direction are written, the rho classes as one product
// with the sign bits of both halves flipped where C_{1+mu} < 0 (rounding to
// nearest is odd in its argument).
template <typename T, bool DAG>
__device__ void tc_b_role(const ApplyArgs& a, int nvb, uint32_t Bs, uint32_t bars, volatile int* abort, int btid)
{
    const int Lx = a.g.L[0];
    const long nitems = (a.nsites / Lx) * (long)nvb;
    const bool on = btid < 240;
    const int d = on ? btid / 3 : 0, c = btid % 3;
    const TcDir D = c_tc_dirs[d];
    const int g_own = D.g, nz = D.nz, neg = DAG ? (D.neg ^ 0xF) : D.neg;
    const bool odd = D.r & 1;
    const uint32_t sub = (uint32_t)(2 - D.g) * TC_BBLK;
    const uint32_t ka = sub + tc_off(0, 6 * D.r), kb = sub + tc_off(0, odd ? 6 * D.r + 2 : 6 * D.r + 4);
    const uint32_t c0x2 = pack2(cx<float>{D.c0, D.c0}, (T*)nullptr);
    const uint32_t rhox2 = pack2(cx<float>{D.rho, D.rho}, (T*)nullptr);
    uint32_t rowoff[2][5];   // rows 6 j + 2 c + ri
#pragma unroll
    for (int ri = 0; ri < 2; ++ri)
#pragma unroll
        for (int j = 0; j < 5; ++j) rowoff[ri][j] = tc_off(6 * j + 2 * c + ri, 0);
    const int woff = 9 * d + 3 * c;
    auto load = [&](long s, uint32_t (&w)[3]) {
        if (!on) return;
        const uint32_t* W = reinterpret_cast<const uint32_t*>(a.links) + (size_t)s * 720 + woff;
        w[0] = ld_ro(W);
        w[1] = ld_ro(W + 1);
        w[2] = ld_ro(W + 2);
    };
    uint32_t wn[3] = {0u, 0u, 0u};
    if ((long)blockIdx.x < nitems) load(tc_row(a, blockIdx.x, nvb).base, wn);
    long f0 = 0;
    bool ok = true;
    for (long item = blockIdx.x; item < nitems && ok; item += gridDim.x, f0 += Lx + 2) {
        const TcRow R = tc_row(a, item, nvb);
        for (int x = 0; x < Lx; ++x) {
            const uint32_t wc[3] = {wn[0], wn[1], wn[2]};
            // the links of the next site, in flight while this one is built
            if (x + 1 < Lx) load(R.base + x + 1, wn);
            else if (item + (long)gridDim.x < nitems) load(tc_row(a, item + gridDim.x, nvb).base, wn);
            // the blocks for g = 0, 1, 2 in turn, each after its entry is free
            // (the entries of g = 0, 1 were already free for site x - 1)
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const long F = f0 + x + g;
                if ((g == 2 || x == 0) && F >= TC_NR &&
                    !tc_wait(bars + 8u * (TC_BAR_EB + (int)(F % TC_NR)), (uint32_t)((F / TC_NR - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                if (on && g == g_own) {
                    const uint32_t base = Bs + (uint32_t)(F % TC_NR) * TC_BENT;
                    uint32_t p0[2][3], p1[2][3];
#pragma unroll
                    for (int cp = 0; cp < 3; ++cp) {
                        const uint32_t e0 = wc[cp] ^ 0x80000000u;          // (re, -im)
                        const uint32_t e1 = __byte_perm(wc[cp], 0, 0x1032); // (im, re)
                        p0[0][cp] = tc_mul2(e0, c0x2, (T*)nullptr);
                        p0[1][cp] = tc_mul2(e1, c0x2, (T*)nullptr);
                        p1[0][cp] = tc_mul2(e0, rhox2, (T*)nullptr);
                        p1[1][cp] = tc_mul2(e1, rhox2, (T*)nullptr);
                    }
#pragma unroll
                    for (int ri = 0; ri < 2; ++ri) {
                        tc_st3(base + rowoff[ri][0], ka, kb, odd, p0[ri][0], p0[ri][1], p0[ri][2]);
#pragma unroll
                        for (int mu = 0; mu < 4; ++mu) {
                            if (!((nz >> mu) & 1)) continue;
                            const uint32_t m = ((neg >> mu) & 1) ? 0x80008000u : 0u;
                            tc_st3(base + rowoff[ri][1 + mu], ka, kb, odd, p1[ri][0] ^ m, p1[ri][1] ^ m, p1[ri][2] ^ m);
                        }
                    }
                    tc_fence_async();
                }
                tc_arrive_n(bars + 8u * (TC_BAR_FB + (int)(F % TC_NR)), tc_b_count(x, g, Lx));
            }
            if (!ok) break;
        }
    }
    // tail: the last releases of the entries arrive before the CTA may exit
    if (ok && btid == 0) {
        for (long F = f0 - TC_NR; F < f0; ++F)
            if (F >= 0 && !tc_wait(bars + 8u * (TC_BAR_EB + (int)(F % TC_NR)), (uint32_t)((F / TC_NR) & 1), abort)) break;
    }
}

// one chain of MMAs: A slot a0 (K = 176) times the sub-blocks of B from b0, n
// columns, into tensor-memory columns d
template <typename T>
__device__ __forceinline__ void tc_chain(uint32_t d, uint32_t a0, uint32_t b0, int n)
{
    const uint32_t idesc = tc_idesc<T>(n);
#pragma unroll
    for (int t = 0; t < TC_KSTEPS; ++t) {
        const uint64_t ad = tc_desc(a0 + 256u * t), bd = tc_desc(b0 + 256u * t);
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                     ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "n"(1));
    }
}

// The MMA issuer (one thread of warp 4): per slot p of a row (fill f0 + p + 1),
// once its A slot and its B entry are there and the accumulator of the site it
// opens (p + 1) is free, the chain (or two, where the sites wrap around the
// accumulator ring); then the commits that free the slot and the entry and
// hand site p - 1, now complete, to the epilogue.
template <typename T>
__device__ void tc_mma_role(const ApplyArgs& a, int nvb, uint32_t a_base, uint32_t b_base, uint32_t tmem,
                            uint32_t bars, volatile int* abort)
{
    const int Lx = a.g.L[0];
    const long nitems = (a.nsites / Lx) * (long)nvb;
    long f0 = 0, i0 = 0;
    bool ok = true;
    for (long item = blockIdx.x; item < nitems && ok; item += gridDim.x, f0 += Lx + 2, i0 += Lx) {
        for (int p = -1; p <= Lx; ++p) {
            const long F = f0 + p + 1;
            ok = tc_wait(bars + 8u * (TC_BAR_FA + (int)(F % TC_NS)), (uint32_t)((F / TC_NS) & 1), abort);
            if (ok) ok = tc_wait(bars + 8u * (TC_BAR_FB + (int)(F % TC_NR)), (uint32_t)((F / TC_NR) & 1), abort);
            if (ok && p + 1 < Lx && i0 + p + 1 >= TC_NACC) {
                const long in = i0 + p + 1;
                ok = tc_wait(bars + 8u * (TC_BAR_EC + (int)(in % TC_NACC)), (uint32_t)((in / TC_NACC - 1) & 1), abort);
            }
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int xlo = max(p - 1, 0), xhi = min(p + 1, Lx - 1);
            const uint32_t a0 = a_base + (uint32_t)(F % TC_NS) * TC_ASLOT;
            const uint32_t e0 = b_base + (uint32_t)(F % TC_NR) * TC_BENT;
            // sites xlo .. xhi: sub-blocks x - p + 1, accumulators (i0 + x) % 16
            const int c0 = (int)((i0 + xlo) % TC_NACC), cnt = xhi - xlo + 1;
            const int run = min(cnt, TC_NACC - c0);
            tc_chain<T>(tmem + 32u * c0, a0, e0 + (uint32_t)(xlo - p + 1) * TC_BBLK, 32 * run);
            if (run < cnt) tc_chain<T>(tmem, a0, e0 + (uint32_t)(xlo + run - p + 1) * TC_BBLK, 32 * (cnt - run));
            tc_commit(bars + 8u * (TC_BAR_EA + (int)(F % TC_NS)));
            tc_commit(bars + 8u * (TC_BAR_EB + (int)(F % TC_NR)));
            if (p >= 1) tc_commit(bars + 8u * (TC_BAR_FC + (int)((i0 + p - 1) % TC_NACC)));
        }
    }
    // every MMA issued here is complete before tensor memory is freed
    tc_commit(bars + 8u * TC_BAR_DR);
    volatile int never = 0;
    tc_wait(bars + 8u * TC_BAR_DR, 0u, &never);
}

// Epilogue (warps 0-3): warp w reads lanes 32 w .. 32 w + 15 of the site's
// accumulator (rows w * 16 + vv: spin w, rhs vv) and clears it; T_1 .. T_4 go
// through shared memory to the spins that need them, and each (spin, rhs)
// forms T_0 + sum_mu gamma_mu T_{1+mu} (chiral basis: gamma_1, gamma_2 couple
// spin s to 3 - s, gamma_3, gamma_4 to s ^ 2), adds the diagonal and stores.
// psi(x) for the diagonal is loaded one site ahead.
template <typename T>
__device__ void tc_epi_role(const ApplyArgs& a, int nvb, uint32_t Ts, uint32_t tmem, uint32_t bars, volatile int* abort,
                            int tid)
{
    static_assert(Store<T>::CPV == 4, "16-bit fields");
    const int Lx = a.g.L[0];
    const long nitems = (a.nsites / Lx) * (long)nvb;
    const size_t nblk = nblk_of((size_t)a.g.vol);
    const int sp = tid >> 5, lane = tid & 31, vv = lane & 15;
    const bool lane_on = lane < TC_VB;
    const uint32_t zero = 0u;
    // factors of the couplings: gamma_1 (-i / +i), gamma_2 (-1 / +1), gamma_3 (-i / +i)
    const float s1 = sp < 2 ? -1.f : 1.f;
    const float s2 = (sp == 0 || sp == 3) ? -1.f : 1.f;
    // complex 3 sp + c of rhs v at site s: ((v nblk + s / 32) 3 + i / 4) 128 + (s % 32) 4 + i % 4
    uint32_t ioff[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ioff[c] = (uint32_t)(((3 * sp + c) >> 2) * 128 + ((3 * sp + c) & 3));
    // staged rows: own (written), spin 3 - sp and spin sp ^ 2 (read)
    const uint32_t t_own = (uint32_t)((sp * TC_VB + vv) * TC_TS * 4);
    const uint32_t t_a = (uint32_t)(((3 - sp) * TC_VB + vv) * TC_TS * 4);
    const uint32_t t_b = (uint32_t)(((sp ^ 2) * TC_VB + vv) * TC_TS * 4);
    const uint32_t* in = reinterpret_cast<const uint32_t*>(a.in);
    auto site_part = [](long s) { return (size_t)(s >> 5) * 384 + (size_t)(s & 31) * 4; };
    auto load_own = [&](const TcRow& R, long s, uint32_t (&w)[3]) {
        const int v = R.vb0 + vv;
        if (!lane_on || v >= a.Nv) return;
        const uint32_t* q = in + (size_t)v * nblk * 384 + site_part(s);
        w[0] = ld_ro(q + ioff[0]);
        w[1] = ld_ro(q + ioff[1]);
        w[2] = ld_ro(q + ioff[2]);
    };
    uint32_t own_n[3] = {0u, 0u, 0u};
    if ((long)blockIdx.x < nitems) {
        const TcRow R0 = tc_row(a, blockIdx.x, nvb);
        load_own(R0, R0.base, own_n);
    }
    long i = 0;
    bool ok = true;
    for (long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const TcRow R = tc_row(a, item, nvb);
        const int v = R.vb0 + vv;
        const bool v_on = lane_on && v < a.Nv;
        const float dg = v_on ? (a.diag_vf ? a.diag_vf[v] : (a.diag_v ? (float)a.diag_v[v] : a.diagf)) : 0.f;
        uint32_t* out = reinterpret_cast<uint32_t*>(a.out) + (size_t)(v_on ? v : 0) * nblk * 384;
        for (int x = 0; x < Lx; ++x, ++i) {
            const uint32_t own[3] = {own_n[0], own_n[1], own_n[2]};
            if (x + 1 < Lx) load_own(R, R.base + x + 1, own_n);
            else if (item + (long)gridDim.x < nitems) {
                const TcRow Rn = tc_row(a, item + gridDim.x, nvb);
                load_own(Rn, Rn.base, own_n);
            }
            const int ac = (int)(i % TC_NACC);
            bool w_ok = tc_wait(bars + 8u * (TC_BAR_FC + ac), (uint32_t)((i / TC_NACC) & 1), abort);
            w_ok = __all_sync(0xffffffffu, w_ok);
            const uint32_t Tb = Ts + (uint32_t)(i & 1) * TC_TBUF;
            uint32_t r[32];
            if (w_ok) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t taddr = tmem + 32u * ac + ((uint32_t)(sp * 32) << 16);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                             "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                               "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                               "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                               "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // clear the accumulator for the site that takes it next
                asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
                             "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr), "r"(zero) : "memory");
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                tc_arrive(bars + 8u * (TC_BAR_EC + ac));
                if (lane_on) {
#pragma unroll
                    for (int n = 6; n < 30; ++n) tc_stsf(Tb + t_own + 4u * (n - 6), __uint_as_float(r[n]));
                }
            }
            if (!tc_epi_and(w_ok)) {
                ok = false;
                break;
            }
            if (v_on) {
                const size_t sp_idx = site_part(R.base + x);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // T_0[sp] + s1 i T_1[3 - sp] + s2 T_2[3 - sp] + s2 i T_3[sp ^ 2] + T_4[sp ^ 2]
                    const float t1r = tc_ldsf(Tb + t_a + 8u * c), t1i = tc_ldsf(Tb + t_a + 8u * c + 4);
                    const float t2r = tc_ldsf(Tb + t_a + 24u + 8u * c), t2i = tc_ldsf(Tb + t_a + 28u + 8u * c);
                    const float t3r = tc_ldsf(Tb + t_b + 48u + 8u * c), t3i = tc_ldsf(Tb + t_b + 52u + 8u * c);
                    const float t4r = tc_ldsf(Tb + t_b + 72u + 8u * c), t4i = tc_ldsf(Tb + t_b + 76u + 8u * c);
                    cx<float> o{__uint_as_float(r[2 * c]), __uint_as_float(r[2 * c + 1])};
                    o.re += -s1 * t1i + s2 * t2r - s2 * t3i + t4r;
                    o.im += s1 * t1r + s2 * t2i + s2 * t3r + t4i;
                    const cx<float> pc = unpack2(own[c], (T*)nullptr);
                    o.re = fmaf(dg, pc.re, o.re);
                    o.im = fmaf(dg, pc.im, o.im);
                    st_cs(out + sp_idx + ioff[c], pack2(o, (T*)nullptr));
                }
            }
        }
    }
}

template <typename T, bool DAG>
__global__ void __launch_bounds__(TC_THREADS, 1) k_brillouin_tc(ApplyArgs a, int nvb)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* As = tc_smem + TC_A_OFF;
    unsigned char* Bs = tc_smem + TC_B_OFF;
    float* Ts = reinterpret_cast<float*>(tc_smem + TC_T_OFF);
    const uint32_t bars = smem_u32(tc_smem + TC_BAR_OFF);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_smem + TC_BAR_OFF + 8 * TC_NBARS);
    volatile int* abort = reinterpret_cast<volatile int*>(tc_smem + TC_BAR_OFF + 8 * TC_NBARS + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // operands start at zero: K padding, vanishing classes, the d = 0 entries of B, absent rows
    for (uint32_t i = tid; i < TC_T_OFF / 16; i += TC_THREADS)
        reinterpret_cast<uint4*>(tc_smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    tc_fence_async();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < TC_NS; ++s) {
            tc_bar_init(bars + 8u * (TC_BAR_FA + s), TC_GTHREADS);   // the gatherers
            tc_bar_init(bars + 8u * (TC_BAR_EA + s), 1);     // one commit
        }
        for (int b = 0; b < TC_NR; ++b) {
            tc_bar_init(bars + 8u * (TC_BAR_FB + b), 3 * TC_BTHREADS);   // three sites' builders
            tc_bar_init(bars + 8u * (TC_BAR_EB + b), 1);
        }
        for (int c = 0; c < TC_NACC; ++c) {
            tc_bar_init(bars + 8u * (TC_BAR_FC + c), 1);
            tc_bar_init(bars + 8u * (TC_BAR_EC + c), 128);   // the epilogue
        }
        tc_bar_init(bars + 8u * TC_BAR_DR, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (warp < TC_EPI_WARPS) {
        // all accumulators start at zero (every MMA accumulates)
        const uint32_t zero = 0u;
        for (int c = 0; c < TC_NACC; ++c)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
                         "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
                         ::"r"(tmem + 32u * c + ((uint32_t)(warp * 32) << 16)), "r"(zero) : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (warp < TC_EPI_WARPS) tc_epi_role<T>(a, nvb, smem_u32(Ts), tmem, bars, abort, tid);
    else if (warp == TC_MMA_WARP) {
        if (lane == 0) tc_mma_role<T>(a, nvb, smem_u32(As), smem_u32(Bs), tmem, bars, abort);
    } else if (warp < TC_B_WARP0) {
        tc_gather_role<T>(a, nvb, smem_u32(As), bars, abort, warp - TC_GATHER_WARP0, lane);
    } else {
        tc_b_role<T, DAG>(a, nvb, smem_u32(Bs), bars, abort, tid - TC_B_WARP0 * 32);
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort && a.err) atomicExch(a.err, (int)DIRAC_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
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
    const long nitems = (a.nsites / a.g.L[0]) * (long)nvb;
    // one CTA per SM: ~200 KB of shared memory and all 512 tensor-memory columns
    const long grid = std::min<long>(nitems, nsm);
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
    int n = 0;
    for (int g = 0; g < 3; ++g)
        for (int r = 0; r < 27; ++r)
            for (int j = 0; j < 80; ++j) {
                const signed char* d = dirs[j].d;
                if (d[0] + 1 != g || (d[1] + 1) + 3 * (d[2] + 1) + 9 * (d[3] + 1) != r) continue;
                int k = 0;
                for (int m = 0; m < 4; ++m) k += d[m] != 0;
                TcDir& D = t[n++];
                D.g = (signed char)g;
                D.r = (signed char)r;
                D.plane = (short)(dirs[j].neg ? 40 + dirs[j].rep : dirs[j].rep);
                D.c0 = (float)dirs[j].a;   // -lambda_k / 2
                D.rho = (float)rho[k];
                D.nz = 0;
                D.neg = 0;
                for (int m = 0; m < 4; ++m) {
                    D.nz |= (d[m] != 0) << m;
                    D.neg |= (d[m] < 0) << m;
                }
            }
    if (n != 80) return cudaErrorInvalidValue;
    e = cudaMemcpyToSymbolAsync(c_tc_dirs, t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

// the site-major copy: element (s, d, e) = W plane of direction d (tensor-core
// order), entry e, at site s; 16-bit complex words copied unchanged
__global__ void k_brillouin_tc_links(size_t vol, size_t nsite, const uint32_t* __restrict__ w80, uint32_t* __restrict__ wtc)
{
    const size_t n = nsite * 720;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = i / 720;
        const int r = (int)(i - s * 720), d = r / 9, e = r - 9 * d;
        wtc[i] = w80[blk_index(vol, 9, c_tc_dirs[d].plane, e, (long)s)];
    }
}

cudaError_t launch_brillouin_tc_links(const Geom& g, const void* w80, void* wtc, cudaStream_t st)
{
    const size_t nsite = nblk_of((size_t)g.vol) * 32;
    const size_t n = nsite * 720;
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 65535);
    k_brillouin_tc_links<<<grid, 256, 0, st>>>((size_t)g.vol, nsite, static_cast<const uint32_t*>(w80),
                                               static_cast<uint32_t*>(wtc));
    return cudaGetLastError();
}

// a.links: the 80 W of each site, site-major in the order of c_tc_dirs
// (launch_brillouin_tc_links), 16-bit; a.in, a.out 16-bit fields of the storage type
cudaError_t launch_brillouin_tc(int prec, bool dag, const ApplyArgs& a, cudaStream_t st)
{
    if (a.nsites == 0 || a.Nv == 0) return cudaSuccess;
    if (prec == P_BF16) return tc_go<__nv_bfloat16>(dag, a, st);
    if (prec == P_F16) return tc_go<__half>(dag, a, st);
    return cudaErrorInvalidValue;
}

}  // namespace dirac
