// Host side of the even-odd sweeps and the two kernels that move fields
// between the whole-lattice FP64 layout of the outer solver and the half
// fields (one parity each) of the even-odd inner solver (dirac_eo.cuh).
#include "dirac_eo.cuh"

namespace dirac {

constexpr int EO_BT = 256;

// parity of site s
DEV_INLINE int site_parity(const Geom& g, long s)
{
    uint32_t r = (uint32_t)s;
    int sum = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const uint32_t q = fdiv(g.fd[mu], r);
        sum += (int)(r - q * (uint32_t)g.L[mu]);
        r = q;
    }
    return (sum + (int)r) & 1;
}

template <typename T, int NSC>
__global__ void k_eo_split(Geom g, long vh, const void* __restrict__ r64, const double* __restrict__ scale, void* re,
                           void* ro)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const double c = scale ? scale[v] : 1.0;
    for (long s = (long)blockIdx.x * EO_BT + threadIdx.x; s < g.vol; s += (long)gridDim.x * EO_BT) {
        cx<double> a[NSC];
        cx<A> b[NSC];
        load_spinor<double, NSC>(r64, g.vol, v, s, a);
#pragma unroll
        for (int k = 0; k < NSC; ++k) b[k] = cx<A>{(A)(c * a[k].re), (A)(c * a[k].im)};
        store_spinor<T, NSC>(site_parity(g, s) ? ro : re, vh, v, s >> 1, b);
    }
}

template <typename T, int NSC>
__global__ void k_eo_axpy_to64(Geom g, long vh, const double* __restrict__ coef, const void* __restrict__ ee,
                               const void* __restrict__ eo, void* x64)
{
    using A = typename Store<T>::A;
    const int v = blockIdx.y;
    const double c = coef[v];
    if (c == 0.0) return;
    for (long s = (long)blockIdx.x * EO_BT + threadIdx.x; s < g.vol; s += (long)gridDim.x * EO_BT) {
        cx<A> ev[NSC];
        cx<double> xv[NSC];
        load_spinor<T, NSC>(site_parity(g, s) ? eo : ee, vh, v, s >> 1, ev);
        load_spinor<double, NSC>(x64, g.vol, v, s, xv);
#pragma unroll
        for (int k = 0; k < NSC; ++k) {
            xv[k].re = fma(c, (double)ev[k].re, xv[k].re);
            xv[k].im = fma(c, (double)ev[k].im, xv[k].im);
        }
        store_spinor<double, NSC>(x64, g.vol, v, s, xv);
    }
}

static dim3 eo_grid(long vol, int Nv)
{
    long b = (vol + (long)EO_BT * 4 - 1) / ((long)EO_BT * 4);   // about 4 sites per thread
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return dim3((unsigned)b, (unsigned)Nv);
}

#define EO_PREC_SWITCH(prec, FN)          \
    switch (prec) {                       \
    case P_F64: FN(double); break;        \
    case P_F32: FN(float); break;         \
    case P_BF16: FN(__nv_bfloat16); break; \
    case P_F16: FN(__half); break;        \
    default: return cudaErrorInvalidValue; \
    }

cudaError_t eo_split(int prec, int nsc, const Geom& g, int Nv, const void* r64, const double* scale, void* re,
                     void* ro, cudaStream_t st)
{
    const dim3 gr = eo_grid(g.vol, Nv);
    const long vh = g.vol / 2;
#define GO(T) (nsc == 12 ? (k_eo_split<T, 12><<<gr, EO_BT, 0, st>>>(g, vh, r64, scale, re, ro)) \
                         : (k_eo_split<T, 3><<<gr, EO_BT, 0, st>>>(g, vh, r64, scale, re, ro)))
    EO_PREC_SWITCH(prec, GO)
#undef GO
    return cudaGetLastError();
}

cudaError_t eo_axpy_to64(int prec, int nsc, const Geom& g, int Nv, const double* coef, const void* ee,
                         const void* eo, void* x64, cudaStream_t st)
{
    const dim3 gr = eo_grid(g.vol, Nv);
    const long vh = g.vol / 2;
#define GO(T) (nsc == 12 ? (k_eo_axpy_to64<T, 12><<<gr, EO_BT, 0, st>>>(g, vh, coef, ee, eo, x64)) \
                         : (k_eo_axpy_to64<T, 3><<<gr, EO_BT, 0, st>>>(g, vh, coef, ee, eo, x64)))
    EO_PREC_SWITCH(prec, GO)
#undef GO
    return cudaGetLastError();
}

EoArgs make_eo_args(const Geom& g, int Nv, int par, const void* in, const void* in2, void* out, const void* links,
                    const void* coef, int tc)
{
    EoArgs a;
    a.g = g;
    a.gh = make_geom(g.L[0] / 2, g.L[1], g.L[2], g.L[3]);
    a.vh = g.vol / 2;
    a.Nv = Nv;
    a.par = par;
    a.in = in;
    a.in2 = in2;
    a.out = out;
    a.links = links;
    a.coef = coef;
    a.tc = tc < 0 ? 0 : (tc > g.L[3] ? g.L[3] : tc);
    a.fdc = make_fdiv((uint32_t)(g.L[2] * (a.tc > 0 ? a.tc : 1)));
    a.fdt = make_fdiv((uint32_t)(a.tc > 0 ? a.tc : 1));
    return a;
}

cudaError_t launch_eo(int op, int prec, bool dag, const EoArgs& a, LaunchCfg cfg, cudaStream_t st)
{
    if (a.vh == 0 || a.Nv == 0) return cudaSuccess;
    if (!eo_rhs_supported(op, prec, a.Nv, cfg.R)) return cudaErrorInvalidValue;
    if (op == OP_WILSON) return launch_eo_wilson(prec, dag, a, cfg.R, cfg.block, st);
    if (op == OP_STAGGERED) return launch_eo_staggered(prec, dag, a, cfg.R, cfg.block, st);
    return cudaErrorInvalidValue;
}

}  // namespace dirac
