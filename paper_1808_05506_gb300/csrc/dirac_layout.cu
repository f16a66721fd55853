// Layout conversion (canonical <-> internal blocked layout) and the
// Brillouin off-axis link build of Tab. tab:off-axis.
#include "dirac_internal.h"

namespace dirac {

// ---------------------------------------------------------------- spinors
// canonical complex numbers c of one (site, rhs): NSC contiguous complex of type CT,
// read and written with the widest aligned vector (float4 = 2 complex when the
// 8 * NSC-byte run is 16-byte aligned, else one complex at a time)
template <int NSC, typename CT, typename A>
__device__ __forceinline__ void canon_load(const CT* src, cx<A>* p)
{
    if constexpr (sizeof(CT) == 4 && NSC % 2 == 0) {
        const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int j = 0; j < NSC / 2; ++j) {
            float4 v = q[j];
            p[2 * j] = cx<A>{(A)v.x, (A)v.y};
            p[2 * j + 1] = cx<A>{(A)v.z, (A)v.w};
        }
    } else if constexpr (sizeof(CT) == 4) {
        const float2* q = reinterpret_cast<const float2*>(src);
#pragma unroll
        for (int j = 0; j < NSC; ++j) {
            float2 v = q[j];
            p[j] = cx<A>{(A)v.x, (A)v.y};
        }
    } else {
        const double2* q = reinterpret_cast<const double2*>(src);
#pragma unroll
        for (int j = 0; j < NSC; ++j) {
            double2 v = q[j];
            p[j] = cx<A>{(A)v.x, (A)v.y};
        }
    }
}

template <int NSC, typename CT, typename A>
__device__ __forceinline__ void canon_store(CT* dst, const cx<A>* p)
{
    if constexpr (sizeof(CT) == 4 && NSC % 2 == 0) {
        float4* q = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int j = 0; j < NSC / 2; ++j)
            q[j] = make_float4((float)p[2 * j].re, (float)p[2 * j].im, (float)p[2 * j + 1].re, (float)p[2 * j + 1].im);
    } else if constexpr (sizeof(CT) == 4) {
        float2* q = reinterpret_cast<float2*>(dst);
#pragma unroll
        for (int j = 0; j < NSC; ++j) q[j] = make_float2((float)p[j].re, (float)p[j].im);
    } else {
        double2* q = reinterpret_cast<double2*>(dst);
#pragma unroll
        for (int j = 0; j < NSC; ++j) q[j] = make_double2((double)p[j].re, (double)p[j].im);
    }
}

// canon holds the sites site0 .. site0 + nsites - 1 (a t-slab, or the whole lattice)
template <typename T, int NSC, typename CT>
__global__ void k_pack(Geom g, int Nv, const CT* __restrict__ canon, void* internal, long site0, long nsites)
{
    using A = typename Store<T>::A;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, v), v fastest
    if (i >= nsites * Nv) return;
    const long s = site0 + i / Nv;
    const int v = (int)(i % Nv);
    cx<A> p[NSC];
    canon_load<NSC, CT, A>(canon + (size_t)i * NSC * 2, p);
    store_spinor<T, NSC>(internal, g.vol, v, s, p);
}

template <typename T, int NSC, typename CT>
__global__ void k_unpack(Geom g, int Nv, const void* internal, CT* __restrict__ canon, long site0, long nsites)
{
    using A = typename Store<T>::A;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsites * Nv) return;
    const long s = site0 + i / Nv;
    const int v = (int)(i % Nv);
    cx<A> p[NSC];
    load_spinor<T, NSC>(internal, g.vol, v, s, p);
    canon_store<NSC, CT, A>(canon + (size_t)i * NSC * 2, p);
}

template <typename T, int NSC>
static cudaError_t pack_T(const Geom& g, int Nv, const void* canon, bool f64, void* internal,
                          cudaStream_t st, long site0, long nsites)
{
    const long n = nsites * Nv;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (f64) k_pack<T, NSC, double><<<nb, 256, 0, st>>>(g, Nv, (const double*)canon, internal, site0, nsites);
    else k_pack<T, NSC, float><<<nb, 256, 0, st>>>(g, Nv, (const float*)canon, internal, site0, nsites);
    return cudaGetLastError();
}

template <typename T, int NSC>
static cudaError_t unpack_T(const Geom& g, int Nv, const void* internal, void* canon, bool f64,
                            cudaStream_t st, long site0, long nsites)
{
    const long n = nsites * Nv;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (f64) k_unpack<T, NSC, double><<<nb, 256, 0, st>>>(g, Nv, internal, (double*)canon, site0, nsites);
    else k_unpack<T, NSC, float><<<nb, 256, 0, st>>>(g, Nv, internal, (float*)canon, site0, nsites);
    return cudaGetLastError();
}

#define DISPATCH_PREC_NSC(FN, ...)                                                        \
    switch (prec) {                                                                       \
    case P_F64: return nsc == 12 ? FN<double, 12>(__VA_ARGS__) : FN<double, 3>(__VA_ARGS__); \
    case P_F32: return nsc == 12 ? FN<float, 12>(__VA_ARGS__) : FN<float, 3>(__VA_ARGS__);   \
    case P_BF16:                                                                          \
        return nsc == 12 ? FN<__nv_bfloat16, 12>(__VA_ARGS__) : FN<__nv_bfloat16, 3>(__VA_ARGS__); \
    case P_F16: return nsc == 12 ? FN<__half, 12>(__VA_ARGS__) : FN<__half, 3>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue;                                                \
    }

cudaError_t launch_pack_spinor(int prec, int nsc, const Geom& g, int Nv, const void* canon,
                               bool canon_f64, void* internal, cudaStream_t st, long site0, long nsites)
{
    if (nsites < 0) nsites = g.vol;
    if (nsites * Nv == 0) return cudaSuccess;
    DISPATCH_PREC_NSC(pack_T, g, Nv, canon, canon_f64, internal, st, site0, nsites)
}

cudaError_t launch_unpack_spinor(int prec, int nsc, const Geom& g, int Nv, const void* internal,
                                 void* canon, bool canon_f64, cudaStream_t st, long site0, long nsites)
{
    if (nsites < 0) nsites = g.vol;
    if (nsites * Nv == 0) return cudaSuccess;
    DISPATCH_PREC_NSC(unpack_T, g, Nv, internal, canon, canon_f64, st, site0, nsites)
}

// one column c of a canonical FP64 field with Nsrc right-hand sides <-> slot v
// of an internal FP64 field (the batched solver's queue of systems)
template <int NSC>
__global__ void k_pack_column(Geom g, int Nsrc, int c, const double* __restrict__ canon, int v, void* internal)
{
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.vol) return;
    const double* src = canon + ((size_t)s * Nsrc + c) * NSC * 2;
    cx<double> p[NSC];
#pragma unroll
    for (int k = 0; k < NSC; ++k) p[k] = cx<double>{src[2 * k], src[2 * k + 1]};
    store_spinor<double, NSC>(internal, g.vol, v, s, p);
}

template <int NSC>
__global__ void k_unpack_column(Geom g, int v, const void* internal, int Nsrc, int c, double* __restrict__ canon)
{
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.vol) return;
    cx<double> p[NSC];
    load_spinor<double, NSC>(internal, g.vol, v, s, p);
    double* dst = canon + ((size_t)s * Nsrc + c) * NSC * 2;
#pragma unroll
    for (int k = 0; k < NSC; ++k) {
        dst[2 * k] = p[k].re;
        dst[2 * k + 1] = p[k].im;
    }
}

cudaError_t launch_pack_column64(int nsc, const Geom& g, int Nsrc, int c, const void* canon, int v, void* internal,
                                 cudaStream_t st)
{
    const unsigned nb = (unsigned)((g.vol + 255) / 256);
    if (nsc == 12) k_pack_column<12><<<nb, 256, 0, st>>>(g, Nsrc, c, (const double*)canon, v, internal);
    else k_pack_column<3><<<nb, 256, 0, st>>>(g, Nsrc, c, (const double*)canon, v, internal);
    return cudaGetLastError();
}

cudaError_t launch_unpack_column64(int nsc, const Geom& g, int v, const void* internal, int Nsrc, int c, void* canon,
                                   cudaStream_t st)
{
    const unsigned nb = (unsigned)((g.vol + 255) / 256);
    if (nsc == 12) k_unpack_column<12><<<nb, 256, 0, st>>>(g, v, internal, Nsrc, c, (double*)canon);
    else k_unpack_column<3><<<nb, 256, 0, st>>>(g, v, internal, Nsrc, c, (double*)canon);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- links
template <typename CT>
__global__ void k_links_to_f64(Geom g, const CT* __restrict__ canon, double2* V64)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, mu)
    if (i >= g.vol * 4) return;
    const long s = i / 4;
    const int mu = (int)(i % 4);
    const CT* src = canon + (size_t)i * 18;
#pragma unroll
    for (int e = 0; e < 9; ++e)
        V64[((size_t)mu * 9 + e) * g.vol + s] = make_double2((double)src[2 * e], (double)src[2 * e + 1]);
}

cudaError_t launch_links_to_f64(const Geom& g, const void* canon, bool canon_f64, void* V64,
                                cudaStream_t st)
{
    const unsigned nb = (unsigned)((g.vol * 4 + 255) / 256);
    if (canon_f64) k_links_to_f64<double><<<nb, 256, 0, st>>>(g, (const double*)canon, (double2*)V64);
    else k_links_to_f64<float><<<nb, 256, 0, st>>>(g, (const float*)canon, (double2*)V64);
    return cudaGetLastError();
}

// FP64 links [m][e][site] -> storage-precision links in the blocked layout
template <typename T>
__global__ void k_convert_links(long vol, long n, const double2* __restrict__ src, void* dst)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (m, e, site), site fastest
    if (i >= n) return;
    const long s = i % vol;
    const long me = i / vol;
    double2 v = src[i];
    using A = typename Store<T>::A;
    st_one<T>(dst, blk_index((size_t)vol, 9, (int)(me / 9), (int)(me % 9), s), cx<A>{(A)v.x, (A)v.y});
}

cudaError_t launch_convert_links(int prec, const Geom& g, int nmat, const void* src64, void* dst,
                                 cudaStream_t st)
{
    const long n = g.vol * 9L * nmat;
    const unsigned nb = (unsigned)((n + 255) / 256);
    const double2* s = (const double2*)src64;
    switch (prec) {
    case P_F64: k_convert_links<double><<<nb, 256, 0, st>>>(g.vol, n, s, dst); break;
    case P_F32: k_convert_links<float><<<nb, 256, 0, st>>>(g.vol, n, s, dst); break;
    case P_BF16: k_convert_links<__nv_bfloat16><<<nb, 256, 0, st>>>(g.vol, n, s, dst); break;
    case P_F16: k_convert_links<__half><<<nb, 256, 0, st>>>(g.vol, n, s, dst); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- W build
// Tab. tab:off-axis defines W_dir(x) as the average of the path products over
// the k! orderings of the k unit hops of dir.  Splitting off the first hop a
// gives the recursion W_dir(x) = (1/k) sum_{hops a of dir} V_a(x) W_{dir-a}(x+a)
// with V_{-mu}(x) = V_mu(x-mu)^+; it is evaluated level by level (k = 1..4)
// in FP64 over all 80 directions, with tmp81 laid out [dir81][9][site].
__device__ __forceinline__ int dir81_of(const int d[4])
{
    return (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1) + 27 * (d[3] + 1);
}

__global__ void k_wbuild_level1(Geom g, const double2* __restrict__ V64, double2* tmp)
{
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.vol) return;
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(g, s, fwd, bwd, x);
    for (int mu = 0; mu < 4; ++mu) {
        int dp[4] = {0, 0, 0, 0}, dm[4] = {0, 0, 0, 0};
        dp[mu] = 1;
        dm[mu] = -1;
        const int cp = dir81_of(dp), cm = dir81_of(dm);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                tmp[((size_t)cp * 9 + a * 3 + b) * g.vol + s] = V64[((size_t)mu * 9 + a * 3 + b) * g.vol + s];
                double2 u = V64[((size_t)mu * 9 + b * 3 + a) * g.vol + s + bwd[mu]];
                tmp[((size_t)cm * 9 + a * 3 + b) * g.vol + s] = make_double2(u.x, -u.y);
            }
    }
}

struct DirList {
    int n;
    int k;
    short code[32];
};

__global__ void k_wbuild_level(Geom g, DirList L, double2* tmp)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, j), site fastest
    if (i >= g.vol * L.n) return;
    const long s = i % g.vol;
    const int j = (int)(i / g.vol);
    const int c = L.code[j];
    int d[4] = {c % 3 - 1, (c / 3) % 3 - 1, (c / 9) % 3 - 1, (c / 27) % 3 - 1};
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(g, s, fwd, bwd, x);
    cx<double> acc[9];
    for (int e = 0; e < 9; ++e) acc[e] = cx<double>{0.0, 0.0};
    for (int mu = 0; mu < 4; ++mu) {
        if (d[mu] == 0) continue;
        int a[4] = {0, 0, 0, 0};
        a[mu] = d[mu];
        int rest[4] = {d[0], d[1], d[2], d[3]};
        rest[mu] = 0;
        const int ca = dir81_of(a), cr = dir81_of(rest);
        const long sa = s + (d[mu] > 0 ? fwd[mu] : bwd[mu]);
        cx<double> Va[9], Wr[9];
        for (int e = 0; e < 9; ++e) {
            double2 u = tmp[((size_t)ca * 9 + e) * g.vol + s];
            double2 w = tmp[((size_t)cr * 9 + e) * g.vol + sa];
            Va[e] = {u.x, u.y};
            Wr[e] = {w.x, w.y};
        }
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) {
                cx<double> t = acc[r * 3 + q];
                for (int m = 0; m < 3; ++m) t = cfma(Va[r * 3 + m], Wr[m * 3 + q], t);
                acc[r * 3 + q] = t;
            }
    }
    const double inv = 1.0 / L.k;
    for (int e = 0; e < 9; ++e)
        tmp[((size_t)c * 9 + e) * g.vol + s] = make_double2(acc[e].re * inv, acc[e].im * inv);
}

struct RepList {
    short code[40];
};

__global__ void k_wbuild_store(Geom g, RepList R, const double2* __restrict__ tmp, double2* W64)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, rep), site fastest
    if (i >= g.vol * 40) return;
    const long s = i % g.vol;
    const int r = (int)(i / g.vol);
    for (int e = 0; e < 9; ++e) W64[((size_t)r * 9 + e) * g.vol + s] = tmp[((size_t)R.code[r] * 9 + e) * g.vol + s];
}

// all 80 directions of W (FP64, [dir81][9][site]; the centre code 40 is not written)
cudaError_t launch_build_W81(const Geom& g, const void* V64, void* tmp81, cudaStream_t st)
{
    double2* tmp = (double2*)tmp81;
    unsigned nb = (unsigned)((g.vol + 255) / 256);
    k_wbuild_level1<<<nb, 256, 0, st>>>(g, (const double2*)V64, tmp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int k = 2; k <= 4; ++k) {
        DirList L;
        L.n = 0;
        L.k = k;
        for (int c = 0; c < 81; ++c) {
            int d[4] = {c % 3 - 1, (c / 3) % 3 - 1, (c / 9) % 3 - 1, (c / 27) % 3 - 1};
            int kk = (d[0] != 0) + (d[1] != 0) + (d[2] != 0) + (d[3] != 0);
            if (kk == k) L.code[L.n++] = (short)c;
        }
        const long n = g.vol * L.n;
        k_wbuild_level<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, L, tmp);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_build_W(const Geom& g, const void* V64, void* tmp81, void* W64, cudaStream_t st)
{
    double2* tmp = (double2*)tmp81;
    cudaError_t e = launch_build_W81(g, V64, tmp81, st);
    if (e != cudaSuccess) return e;
    BriDir dirs[80];
    int reps[40];
    brillouin_tables(dirs, reps);
    RepList R;
    for (int r = 0; r < 40; ++r) R.code[r] = (short)reps[r];
    const long n = g.vol * 40;
    k_wbuild_store<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, R, tmp, (double2*)W64);
    return cudaGetLastError();
}

}  // namespace dirac

// ---------------------------------------------------------------- link formats
namespace dirac {

// two-row links: planes e = 0..5 of each storage link, in a layout with 6 planes
template <typename T>
__global__ void k_links_2row(long vol, long n, const void* __restrict__ src, void* dst)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (mu, e < 6, site), site fastest
    if (i >= n) return;
    const long s = i % vol;
    const long me = i / vol;
    const int mu = (int)(me / 6), e = (int)(me % 6);
    st_one<T>(dst, blk_index((size_t)vol, 6, mu, e, s), ld_one<T>(src, blk_index((size_t)vol, 9, mu, e, s)));
}

cudaError_t launch_links_2row(int prec, const Geom& g, const void* links, void* out, cudaStream_t st)
{
    const long n = g.vol * 4L * 6;
    const unsigned nb = (unsigned)((n + 255) / 256);
    switch (prec) {
    case P_F32: k_links_2row<float><<<nb, 256, 0, st>>>(g.vol, n, links, out); break;
    case P_BF16: k_links_2row<__nv_bfloat16><<<nb, 256, 0, st>>>(g.vol, n, links, out); break;
    case P_F16: k_links_2row<__half><<<nb, 256, 0, st>>>(g.vol, n, links, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// max over the links of |U_2c - conj(U_0 x U_1)_c| in FP64 (non-negative
// doubles order like their bit patterns, so the maximum is an integer atomic)
__global__ void k_su3_deviation(long vol, const double2* __restrict__ V64, unsigned long long* dev)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (mu, site), site fastest
    double m = 0.0;
    if (i < 4 * vol) {
        const long s = i % vol;
        const int mu = (int)(i / vol);
        cx<double> U[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const double2 v = V64[((size_t)mu * 9 + e) * vol + s];
            U[e] = cx<double>{v.x, v.y};
        }
        cx<double> R[9];
#pragma unroll
        for (int e = 0; e < 6; ++e) R[e] = U[e];
        reconstruct_row2(R);
#pragma unroll
        for (int c = 6; c < 9; ++c) {
            const cx<double> d = R[c] - U[c];
            m = fmax(m, sqrt(d.re * d.re + d.im * d.im));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dev, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_su3_deviation(const Geom& g, const void* V64, double* dev, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(dev, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    const long n = 4 * g.vol;
    k_su3_deviation<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g.vol, (const double2*)V64,
                                                                 (unsigned long long*)dev);
    return cudaGetLastError();
}

struct RepDirs {
    signed char d[40][4];
};

// all 80 Brillouin directions per site: plane j < 40 is the stored W_{d_j}(x),
// plane 40 + j is W_{-d_j}(x) = W_{d_j}(x - d_j)^+ (Tab. tab:off-axis caption),
// both in the storage precision (a copy and a conjugate transpose: no rounding)
// planes j0..79 (j0 = 40 when src and dst are the same array: only the
// adjoint planes are written, read from the stored ones)
template <typename T>
__global__ void k_brillouin_w80(Geom g, RepDirs R, int j0, long n, const void* __restrict__ src, void* dst)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (plane - j0, e, site), site fastest
    if (i >= n) return;
    const long s = i % g.vol;
    const long pe = i / g.vol;
    const int j = j0 + (int)(pe / 9), e = (int)(pe % 9);
    using A = typename Store<T>::A;
    cx<A> v;
    if (j < 40) {
        v = ld_one<T>(src, blk_index((size_t)g.vol, 9, j, e, s));
    } else {
        const int rep = j - 40;
        long r = s, sn = 0;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int L = g.L[mu];
            const int x = (int)(r % L);
            r /= L;
            const int xm = (x - R.d[rep][mu] + L) % L;
            sn += (long)xm * g.stride[mu];
        }
        const int a = e / 3, b = e % 3;   // (W^+)_ab = conj(W_ba)
        v = conj(ld_one<T>(src, blk_index((size_t)g.vol, 9, rep, 3 * b + a, sn)));
    }
    st_one<T>(dst, blk_index((size_t)g.vol, 9, j, e, s), v);
}

cudaError_t launch_brillouin_w80(int prec, const Geom& g, const void* links, void* out, cudaStream_t st)
{
    BriDir dirs[80];
    int reps[40];
    brillouin_tables(dirs, reps);
    RepDirs R;
    for (int r = 0; r < 40; ++r) {
        const int c = reps[r];
        R.d[r][0] = (signed char)(c % 3 - 1);
        R.d[r][1] = (signed char)((c / 3) % 3 - 1);
        R.d[r][2] = (signed char)((c / 9) % 3 - 1);
        R.d[r][3] = (signed char)((c / 27) % 3 - 1);
    }
    const int j0 = links == out ? 40 : 0;
    const long n = g.vol * (80L - j0) * 9;
    const unsigned nb = (unsigned)((n + 255) / 256);
    switch (prec) {
    case P_F64: k_brillouin_w80<double><<<nb, 256, 0, st>>>(g, R, j0, n, links, out); break;
    case P_F32: k_brillouin_w80<float><<<nb, 256, 0, st>>>(g, R, j0, n, links, out); break;
    case P_BF16: k_brillouin_w80<__nv_bfloat16><<<nb, 256, 0, st>>>(g, R, j0, n, links, out); break;
    case P_F16: k_brillouin_w80<__half><<<nb, 256, 0, st>>>(g, R, j0, n, links, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dirac
