// Link gradient of L = Re <g, D psi> = Re sum_x g(x)^+ (D psi)(x) for the
// operators that couple through single links, with PyTorch's convention for
// a real loss of complex variables, F = dL/dRe V + i dL/dIm V.  A term
// Re tr(V M) of L contributes M^+ to F and a term Re tr(V^+ M) contributes M.
//   Wilson (Sec. 4, def_wils; V_mu(x) enters the forward hop from x and the
//   backward hop from x+mu):
//     F_mu(x) = -1/2 sum_v sum_s [(1 - gamma_mu) g_v(x)]_s psi_v(x+mu)_s^+
//               -1/2 sum_v sum_s psi_v(x)_s [(1 + gamma_mu) g_v(x+mu)]_s^+
//     Each spin sum runs over the two components of the rank-2 projection:
//     sum_s [(1 + S gamma) a]_s b_s^+ = sum_{c=0,1} h_c k_c^+ with
//     h = a_up + S B a_down, k = b_up + S B b_down.
//   staggered (Sec. 3; eta_mu(x + mu) = eta_mu(x)):
//     F_mu(x) = 1/2 eta_mu(x) sum_v [g_v(x) psi_v(x+mu)^+ - psi_v(x) g_v(x+mu)^+]
// One thread owns one link (x, mu), gathers both hops that touch it and
// writes it once (no atomics).  The Brillouin gradient, through the composite
// transporters W, is in dirac_force_brillouin.cu.
#include "dirac_handle.h"
#include "dirac_kernels.cuh"

using namespace dirac;

namespace dirac {

// acc[a][b] += c * sum_{comp} u_comp[a] conj(w_comp[b]) for ncomp 3-vectors
template <typename A>
__device__ __forceinline__ void outer_acc(cx<A>* acc, const cx<A>* u, const cx<A>* w, int ncomp, A c)
{
    for (int k = 0; k < ncomp; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                cx<A> t = cfma_conj(w[3 * k + b], u[3 * k + a], cx<A>{A(0), A(0)});   // u conj(w)
                acc[3 * a + b].re = fma(c, t.re, acc[3 * a + b].re);
                acc[3 * a + b].im = fma(c, t.im, acc[3 * a + b].im);
            }
}

template <typename T, int MU>
__device__ __forceinline__ void wilson_force_link(const Geom& g, int Nv, const void* psi, const void* gv,
                                                  long s, long sp, cx<typename Store<T>::A>* acc)
{
    using A = typename Store<T>::A;
    for (int v = 0; v < Nv; ++v) {
        cx<A> a[12], b[12], h[6], k[6];
        load_spinor<T, 12>(gv, g.vol, v, s, a);
        load_spinor<T, 12>(psi, g.vol, v, sp, b);
        wilson_project<MU, -1>(a, h);
        wilson_project<MU, -1>(b, k);
        outer_acc(acc, h, k, 2, A(-0.5));
        load_spinor<T, 12>(psi, g.vol, v, s, a);
        load_spinor<T, 12>(gv, g.vol, v, sp, b);
        wilson_project<MU, +1>(a, k);
        wilson_project<MU, +1>(b, h);
        outer_acc(acc, k, h, 2, A(-0.5));
    }
}

template <typename T, bool STAG>
__global__ void __launch_bounds__(128) k_force(Geom g, int Nv, const void* psi, const void* gv, void* F)
{
    using A = typename Store<T>::A;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // (mu, site), site fastest
    if (i >= 4 * g.vol) return;
    const long s = i % g.vol;
    const int mu = (int)(i / g.vol);
    long fwd[4], bwd[4];
    int x[4];
    site_offsets(g, s, fwd, bwd, x);
    const long sp = s + fwd[mu];
    cx<A> acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = cx<A>{A(0), A(0)};
    if constexpr (STAG) {
        int par = 0;
        for (int nu = 0; nu < mu; ++nu) par += x[nu];
        const A eta = (par & 1) ? A(-0.5) : A(0.5);
        for (int v = 0; v < Nv; ++v) {
            cx<A> a[3], b[3];
            load_spinor<T, 3>(gv, g.vol, v, s, a);
            load_spinor<T, 3>(psi, g.vol, v, sp, b);
            outer_acc(acc, a, b, 1, eta);
            load_spinor<T, 3>(psi, g.vol, v, s, a);
            load_spinor<T, 3>(gv, g.vol, v, sp, b);
            outer_acc(acc, a, b, 1, -eta);
        }
    } else {
        switch (mu) {
        case 0: wilson_force_link<T, 0>(g, Nv, psi, gv, s, sp, acc); break;
        case 1: wilson_force_link<T, 1>(g, Nv, psi, gv, s, sp, acc); break;
        case 2: wilson_force_link<T, 2>(g, Nv, psi, gv, s, sp, acc); break;
        default: wilson_force_link<T, 3>(g, Nv, psi, gv, s, sp, acc); break;
        }
    }
    using O = typename Store<A>::One;   // float2 or double2
    O* out = reinterpret_cast<O*>(F) + ((size_t)s * 4 + mu) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        O o;
        o.x = acc[e].re;
        o.y = acc[e].im;
        out[e] = o;
    }
}

template <typename T>
static cudaError_t force_T(int op, const Geom& g, int Nv, const void* psi, const void* gv, void* F, cudaStream_t st)
{
    const unsigned nb = (unsigned)((4 * g.vol + 127) / 128);
    if (op == OP_STAGGERED) k_force<T, true><<<nb, 128, 0, st>>>(g, Nv, psi, gv, F);
    else k_force<T, false><<<nb, 128, 0, st>>>(g, Nv, psi, gv, F);
    return cudaGetLastError();
}

cudaError_t launch_force(int op, int prec, const Geom& g, int Nv, const void* psi, const void* gv, void* F,
                         cudaStream_t st)
{
    switch (prec) {
    case P_F64: return force_T<double>(op, g, Nv, psi, gv, F, st);
    case P_F32: return force_T<float>(op, g, Nv, psi, gv, F, st);
    case P_BF16: return force_T<__nv_bfloat16>(op, g, Nv, psi, gv, F, st);
    case P_F16: return force_T<__half>(op, g, Nv, psi, gv, F, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dirac

extern "C" DIRAC_API dirac_status dirac_force(dirac_handle* h, void* F, const void* psi, const void* g,
                                              dirac_layout layout)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!F || !psi || !g || F == psi || F == g)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_force: NULL or aliased pointers");
    if (layout != DIRAC_CANONICAL && layout != DIRAC_INTERNAL)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_force: unknown layout");
    if (!dirac_check_device_ptr(F) || !dirac_check_device_ptr(psi) || !dirac_check_device_ptr(g))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_force: F, psi and g must be device pointers");
    dirac_status st;
    const void *pi = psi, *gi = g;
    if (layout == DIRAC_CANONICAL) {
        if ((st = h->ensure_workspace())) return st;
        if ((st = dirac_pack(h, h->ws_in, psi))) return st;
        if ((st = dirac_pack(h, h->ws_out, g))) return st;
        pi = h->ws_in;
        gi = h->ws_out;
    }
    if (h->op == OP_BRILLOUIN) {
        // the transporters are rebuilt from V in FP64 (not kept from the forward pass)
        void *w81 = nullptr, *g81 = nullptr;
        const size_t fb = (size_t)h->g.vol * 81 * 9 * 16;
        if ((st = h->alloc(&w81, fb, "Brillouin force scratch"))) return st;
        if ((st = h->alloc(&g81, fb, "Brillouin force scratch"))) {
            h->release(w81);
            return st;
        }
        st = h->cuda(launch_force_brillouin(h->prec, h->g, h->Nv, pi, gi, h->links64, w81, g81, F, h->stream),
                     "Brillouin force kernels");
        h->release_after_sync(w81);
        h->release_after_sync(g81);
        return st;
    }
    return h->cuda(launch_force(h->op, h->prec, h->g, h->Nv, pi, gi, F, h->stream), "force kernel launch");
}
