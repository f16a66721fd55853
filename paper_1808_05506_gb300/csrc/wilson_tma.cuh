// Wilson sweep with its operands staged by the Tensor Memory Accelerator.
//
// A CTA owns tiles of `ny` complete x-rows of one xy-plane (S = Lx * ny
// sites, one consumer thread per site and sub-group).  For each round of RB
// right-hand sides it streams seven stages through a ring of shared-memory
// buffers: the tile itself (with the forward x-links), the y+1 / y-1 rows,
// the z+1 / z-1 and t+1 / t-1 tiles, each with the link planes its hop needs.
// One producer thread issues two tensor copies per stage (cp.async.bulk.tensor
// over 5-D views of the spinor and link arrays, completion counted in bytes
// on an mbarrier); the consumer warps wait for a stage, apply its hop to R
// right-hand sides from shared memory, and release the buffer.  The loads
// therefore stay in flight without occupying registers or the LSU.
// Tensor copies do not wrap around the periodic boundary: where a y stage
// crosses it, the box row outside the lattice is zero-filled and the threads
// of that row read their neighbour from global memory instead.
//
// Stage buffer layout: spinor planes [RB][K][S] of 16-byte elements, then the
// 9 link planes [9][S] of one complex each.  The x-hops use the centre tile
// with the x index rotated inside its row.
//
// Every wait is bounded: after ~1 s without progress a thread records
// DIRAC_TIMEOUT in the handle's error word and stops; the producer first
// waits (bounded) for the copies it issued, so no copy lands in freed
// shared memory.
#pragma once

#include <cuda.h>
#include <type_traits>

#include "dirac_kernels.cuh"

namespace dirac {

constexpr int TMA_STAGES_PER_ROUND = 7;   // centre, y+, y-, z+, z-, t+, t-
constexpr unsigned TMA_SPIN_LIMIT = 1u << 25;   // about 1-2 s with the 32 ns back-off

struct TmaArgs {
    ApplyArgs a;
    int P;           // spinor planes per stage = RB * K
    int ny;          // rows per tile
    int S;           // sites per tile = Lx * ny
    long ntiles;     // number of tiles = vol / S
    int rounds;      // ceil(Nv / RB)
    int* err;        // device error word
};

// ---- PTX wrappers (host emulation: copies happen at issue time, waits pass)
DEV_INLINE unsigned smem_u32(const void* p)
{
#if defined(__CUDA_ARCH__)
    return (unsigned)__cvta_generic_to_shared(p);
#else
    return 0u;
#endif
}

DEV_INLINE void mbar_init(uint64_t* bar, unsigned count)
{
#if defined(__CUDA_ARCH__)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
#else
    (void)bar;
    (void)count;
#endif
}

DEV_INLINE void mbar_fence_init()
{
#if defined(__CUDA_ARCH__)
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#endif
}

DEV_INLINE void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
#if defined(__CUDA_ARCH__)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
#else
    (void)bar;
    (void)bytes;
#endif
}

DEV_INLINE void mbar_arrive(uint64_t* bar)
{
#if defined(__CUDA_ARCH__)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
#else
    (void)bar;
#endif
}

// true once the phase with this parity has completed
DEV_INLINE bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
#if defined(__CUDA_ARCH__)
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
#else
    (void)bar;
    (void)parity;
    return true;
#endif
}

// bounded wait; false on timeout
DEV_INLINE bool mbar_wait(uint64_t* bar, unsigned parity)
{
    for (unsigned it = 0; it < TMA_SPIN_LIMIT; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
#if defined(__CUDA_ARCH__)
        if (it > 256) __nanosleep(32);
#endif
    }
    return false;
}

// bulk copy global -> shared, completion counted on bar; bytes % 16 == 0
DEV_INLINE void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
#if defined(__CUDA_ARCH__)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
#else
    const char* s = static_cast<const char*>(src);
    char* d = static_cast<char*>(dst);
    for (unsigned i = 0; i < bytes; ++i) d[i] = s[i];
    (void)bar;
#endif
}

// 5-D tensor copy global -> shared (box given by the tensor map)
DEV_INLINE void tensor_copy5(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4, uint64_t* bar)
{
#if defined(__CUDA_ARCH__)
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
#else
    (void)dst; (void)map; (void)c0; (void)c1; (void)c2; (void)c3; (void)c4; (void)bar;
#endif
}

template <typename T, int RB>
struct TmaLayout {
    static constexpr int K = SpinorLayout<T, 12>::K;
    static constexpr int LB = (int)sizeof(typename Store<T>::One);
    // bytes of one stage for a tile of S sites
    static HD size_t stage_bytes(int S) { return (size_t)RB * K * S * 16 + (size_t)9 * S * LB; }
};

// Sites and links a stage covers.  For stage d of tile (plane base p0, first
// row y0): returns the site of the tile's row j shifted by the stage's hop.
struct TmaTile {
    long plane0;   // site index of (x=0, y=0) of the tile's xy-plane
    int y0;        // first row
    int z, t;
};

DEV_INLINE TmaTile tma_tile(const Geom& g, int ny, long tile)
{
    const int rows_per_plane = g.L[1] / ny;
    TmaTile T;
    const long plane = tile / rows_per_plane;     // (z, t) plane index
    T.y0 = (int)(tile % rows_per_plane) * ny;
    T.z = (int)(plane % g.L[2]);
    T.t = (int)(plane / g.L[2]);
    T.plane0 = plane * g.stride[2];
    return T;
}

// first site of row j of the tile as seen from stage d (the neighbour row /
// tile the stage holds), and the site of the link plane the stage holds
DEV_INLINE long tma_row_site(const Geom& g, const TmaTile& T, int j, int d)
{
    int y = T.y0 + j, z = T.z, t = T.t;
    switch (d) {
    case 1: y = (y + 1) % g.L[1]; break;
    case 2: y = (y + g.L[1] - 1) % g.L[1]; break;
    case 3: z = (z + 1) % g.L[2]; break;
    case 4: z = (z + g.L[2] - 1) % g.L[2]; break;
    case 5: t = (t + 1) % g.L[3]; break;
    case 6: t = (t + g.L[3] - 1) % g.L[3]; break;
    default: break;
    }
    return ((long)t * g.L[2] + z) * g.stride[2] + (long)y * g.L[0];
}
// link planes of stage d: forward links (own rows) for d = 0, 1, 3, 5; the
// backward hop's link V_mu(x - mu) sits at the neighbour rows for d = 2, 4, 6
DEV_INLINE long tma_link_row_site(const Geom& g, const TmaTile& T, int j, int d)
{
    return (d == 2 || d == 4 || d == 6) ? tma_row_site(g, T, j, d) : tma_row_site(g, T, j, 0);
}
DEV_INLINE int tma_link_mu(int d) { return (d + 1) / 2; }   // 0:x 1,2:y 3,4:z 5,6:t

// zt coordinate and first y row of the box stage d holds for tile T (y may be
// -1 or Ly - ny + 1 .. Ly: the row outside the lattice is zero-filled)
DEV_INLINE void tma_stage_coords(const Geom& g, const TmaTile& T, int d, int* y, int* zt)
{
    int yy = T.y0, z = T.z, t = T.t;
    switch (d) {
    case 1: yy += 1; break;
    case 2: yy -= 1; break;
    case 3: z = (z + 1) % g.L[2]; break;
    case 4: z = (z + g.L[2] - 1) % g.L[2]; break;
    case 5: t = (t + 1) % g.L[3]; break;
    case 6: t = (t + g.L[3] - 1) % g.L[3]; break;
    default: break;
    }
    *y = yy;
    *zt = z + g.L[2] * t;
}

// Producer: issue the two tensor copies of stage d of round q for tile T.
template <typename T_, int RB>
DEV_INLINE void tma_issue_stage(const TmaArgs& ta, const CUtensorMap* mspin, const CUtensorMap* mlink,
                                const TmaTile& T, int q, int d, char* buf, uint64_t* full)
{
    using Lay = TmaLayout<T_, RB>;
    mbar_arrive_expect_tx(full, (unsigned)Lay::stage_bytes(ta.S));
    int y, zt;
    tma_stage_coords(ta.a.g, T, d, &y, &zt);
#if !defined(__CUDA_ARCH__)
    {
        // host emulation of the two boxes (rows outside the lattice read as zero)
        const Geom& g = ta.a.g;
        const int Lx = g.L[0];
        auto box = [&](const char* src, size_t plane_bytes, int row_bytes, int plane0, int nplanes, int nvalid,
                       int yb, int ztb, char* dst) {
            for (int p = 0; p < nplanes; ++p)
                for (int j = 0; j < ta.ny; ++j) {
                    char* o = dst + ((size_t)p * ta.ny + j) * row_bytes;
                    const int yy = yb + j;
                    if (plane0 + p >= nvalid || yy < 0 || yy >= g.L[1]) {
                        for (int b = 0; b < row_bytes; ++b) o[b] = 0;
                        continue;
                    }
                    const char* s2 = src + (size_t)(plane0 + p) * plane_bytes +
                                     ((size_t)ztb * g.L[1] + yy) * (size_t)row_bytes;
                    for (int b = 0; b < row_bytes; ++b) o[b] = s2[b];
                }
        };
        box(static_cast<const char*>(ta.a.in), (size_t)g.vol * 16, Lx * 16, q * ta.P, ta.P,
            ta.a.Nv * Lay::K, y, zt, buf);
        int ly = y, lzt = zt;
        if (d == 1 || d == 3 || d == 5) tma_stage_coords(g, T, 0, &ly, &lzt);
        box(static_cast<const char*>(ta.a.links), (size_t)g.vol * Lay::LB, Lx * Lay::LB, tma_link_mu(d) * 9, 9, 36,
            ly, lzt, buf + (size_t)ta.P * ta.S * 16);
        (void)mspin;
        (void)mlink;
        return;
    }
#endif
    // spinor planes [q*RB*K, q*RB*K + P) of the box rows; planes past Nv*K read as zero
    tensor_copy5(buf, mspin, 0, 0, y, zt, q * ta.P, full);
    // link planes mu*9 .. mu*9+8 of the forward rows (d = 0, 1, 3, 5) or of the
    // neighbour rows (d = 2, 4, 6: the backward hop's V_mu(x - mu))
    int ly = y, lzt = zt;
    if (d == 1 || d == 3 || d == 5) tma_stage_coords(ta.a.g, T, 0, &ly, &lzt);
    tensor_copy5(buf + (size_t)ta.P * ta.S * 16, mlink, 0, 0, ly, lzt, tma_link_mu(d) * 9, full);
}

// Consumer: apply stage d of the current round to this thread's R
// right-hand sides (sub-group sub covers r_local = sub * R .. sub * R + R - 1).
// gsite >= 0: this thread's neighbour row fell outside the box (a y stage
// crossing the periodic boundary): read the spinors at site gsite and, for
// the backward y hop, the link at gsite from global memory instead
template <typename T_, int R, int RB, bool DAG>
DEV_INLINE void tma_consume_stage(const TmaArgs& ta, int d, const char* buf, int i, int sub, int q,
                                  cx<typename Store<T_>::A> (&acc)[R][12], long gsite = -1)
{
    using A = typename Store<T_>::A;
    using Lay = TmaLayout<T_, RB>;
    using L = SpinorLayout<T_, 12>;
    const int S = ta.S, Lx = ta.a.g.L[0];
    const char* lbase = buf + (size_t)RB * Lay::K * S * 16;
    auto spinor = [&](int rl, int idx, cx<A>* p) {
        if (gsite >= 0) {
            load_spinor<T_, 12>(ta.a.in, ta.a.g.vol, min(q * RB + rl, ta.a.Nv - 1), gsite, p);
            return;
        }
#pragma unroll
        for (int k = 0; k < Lay::K; ++k) {
            const char* src = buf + (((size_t)rl * Lay::K + k) * S + idx) * 16;
            if constexpr (L::CPV == 1) p[k] = sm_one<T_>(src);
            else sm_vec<T_>(src, p + k * L::CPV);
        }
    };
    auto link = [&](int idx, cx<A>* U) {
        if (gsite >= 0 && d == 2) {
            load_link<T_>(ta.a.links, ta.a.g.vol, 1, gsite, U);
            return;
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) U[e] = sm_one<T_>(lbase + ((size_t)e * S + idx) * Lay::LB);
    };
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    auto hop = [&](auto mu_c, auto s_c, auto back_c, int sidx, int lidx) {
        constexpr int MU = decltype(mu_c)::value;
        constexpr int S_ = decltype(s_c)::value;
        constexpr bool BACK = decltype(back_c)::value;
        cx<A> U[9];
        link(lidx, U);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cx<A> p[12], h[6], w[6];
            spinor(sub * R + r, sidx, p);
            wilson_project<MU, S_>(p, h);
            if constexpr (BACK) { mat_dag_vec(U, h, w); mat_dag_vec(U, h + 3, w + 3); }
            else { mat_vec(U, h, w); mat_vec(U, h + 3, w + 3); }
            wilson_reconstruct<MU, S_>(w, acc[r]);
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using BF = std::integral_constant<bool, false>;
    using BT = std::integral_constant<bool, true>;
    using SFc = std::integral_constant<int, SF>;
    using SBc = std::integral_constant<int, SB>;
    if (d == 0) {
        // start the sum with -2 diag psi(x) (out = -1/2 acc at the end), then both x hops
        const int x = i % Lx, rowb = i - x;
        const int ixp = rowb + (x + 1 == Lx ? 0 : x + 1);
        const int ixm = rowb + (x == 0 ? Lx - 1 : x - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = min(q * RB + sub * R + r, ta.a.Nv - 1);
            const A m2d = (A)(-2) * diag_of<A>(ta.a, v);
            cx<A> p[12];
            spinor(sub * R + r, i, p);
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[r][c] = cx<A>{m2d * p[c].re, m2d * p[c].im};
        }
        hop(I0{}, SFc{}, BF{}, ixp, i);
        hop(I0{}, SBc{}, BT{}, ixm, ixm);
    } else if (d == 1) hop(I1{}, SFc{}, BF{}, i, i);
    else if (d == 2) hop(I1{}, SBc{}, BT{}, i, i);
    else if (d == 3) hop(I2{}, SFc{}, BF{}, i, i);
    else if (d == 4) hop(I2{}, SBc{}, BT{}, i, i);
    else if (d == 5) hop(I3{}, SFc{}, BF{}, i, i);
    else hop(I3{}, SBc{}, BT{}, i, i);
}

}  // namespace dirac
