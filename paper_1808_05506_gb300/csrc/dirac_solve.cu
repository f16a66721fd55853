// Defect-correction (iterative-refinement) solvers for D x = b: one system
// with Nv right-hand sides (dirac_solve), and a queue of systems with their
// own Nv and masses sharing one gauge field (dirac_solve_batched).  Every
// right-hand side has its own scalars and convergence test.
//
// Outer loop, FP64 on the GPU (the only FP64 steps): r = b - D x with FP64
// links and an FP64 sweep, per-right-hand-side |r|^2 and |b|^2, stop when
// |r| / |b| <= tol; otherwise normalise r_hat = r sqrt(n) / |r| (unit RMS,
// safe for 16-bit storage), solve D e = r_hat approximately in the storage
// precision, and update x += (|r| / sqrt(n)) e in FP64.
// Inner solver: CGLS, i.e. conjugate gradients on D^+ D e = D^+ r_hat written
// to carry the true residual r = r_hat - D e of the unsymmetric system:
//     r = r_hat, s = D^+ r, p = s, gamma = |s|^2
//     loop: t = D p, delta = |t|^2, alpha = gamma / delta,
//           e += alpha p, r -= alpha t, s = D^+ r, gamma' = |s|^2,
//           beta = gamma' / gamma, p = s + beta p,
//           a right-hand side stops (alpha = beta = 0 from then on) once
//           |r| <= inner_tol |r_hat|.
// Fields are stored in the handle's precision; arithmetic is FP32 (FP64 for
// FP64 handles); norms are FP64.  The scalars and the stopping masks live on
// the device, so groups of 8 iterations are captured once as a CUDA graph
// and replayed; the host looks at one counter per group.
// Batched systems share every sweep: all resident right-hand sides are one
// multi-right-hand-side field, and the sweep takes a per-right-hand-side
// diagonal (the mass of its system).  A queue admits the columns of the
// systems into free slots and writes each column back as soon as it
// converges.
// Even-odd inner solves (Wilson and staggered, every extent even, nonzero
// diagonal; dirac_eo.cuh): r_hat is split into its even and odd half fields,
// the inner iteration runs on the Schur complement S = a - H_oe H_eo / a of
// the odd sites (CGLS for Wilson; plain CG for staggered, whose S = m +
// H_eo^+ H_eo / m is hermitian and definite), and the even half follows as
// e_e = (r_e - H_eo e_o) / a.  The residual of D e = r_hat is then the Schur
// residual on the odd sites (zero on the even ones), so the stopping test and
// the FP64 outer loop are unchanged.  Each application of S is two
// half-lattice sweeps.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <vector>

#include "dirac_blas.h"
#include "dirac_df.cuh"
#include "dirac_eo.cuh"
#include "dirac_handle.h"

using namespace dirac;

namespace dirac {

constexpr int GRAPH_ITERS = 8;

// DIRAC_TRACE=1 in the environment prints the refinement history to stderr
static bool trace_on()
{
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("DIRAC_TRACE");
        on = (e && *e && *e != '0') ? 1 : 0;
    }
    return on == 1;
}

// per right-hand side: alpha = gamma / delta for active ones (else 0); flags breakdown
__global__ void k_cgls_alpha(int Nv, const double* gamma, const double* delta, const int* active,
                             double* alpha, int* breakdown)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= Nv) return;
    double a = 0.0;
    if (active[v]) {
        const double d = delta[v];
        if (!(d > 0.0) || !isfinite(d) || !isfinite(gamma[v])) *breakdown = 1;
        else a = gamma[v] / d;
    }
    alpha[v] = a;
}

// the same for CG on a hermitian definite operator of either sign: delta =
// <p, S p> may be negative, only zero or non-finite values are a breakdown
__global__ void k_cg_alpha(int Nv, const double* gamma, const double* delta, const int* active, double* alpha,
                           int* breakdown)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= Nv) return;
    double a = 0.0;
    if (active[v]) {
        const double d = delta[v];
        if (d == 0.0 || !isfinite(d) || !isfinite(gamma[v])) *breakdown = 1;
        else a = gamma[v] / d;
    }
    alpha[v] = a;
}

// beta = gamma' / gamma for active ones (else 0); gamma <- gamma'
__global__ void k_cgls_beta(int Nv, const double* gnew, double* gamma, const int* active, double* beta)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= Nv) return;
    double b = 0.0;
    if (active[v] && gamma[v] > 0.0) b = gnew[v] / gamma[v];
    beta[v] = b;
    gamma[v] = gnew[v];
}

// stop the right-hand sides that reached |r|^2 <= tol2 |r_hat|^2 (or went
// non-finite), then count the active ones
__global__ void k_cgls_mask(int Nv, const double* rr, const double* rr0, const double* tol2, int* active,
                            int* nactive)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int mine = 0;
    for (int v = threadIdx.x; v < Nv; v += blockDim.x) {
        if (active[v] && !(rr[v] > tol2[0] * rr0[v])) active[v] = 0;
        mine += active[v];
    }
    atomicAdd(&cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) *nactive = cnt;
}

// coefficient sets (alpha_v, beta_v) of the even-odd sweeps out = alpha in2 + beta H in
enum { EO_HOP = 0,   // (0, 1): H_eo p
       EO_S = 1,     // (a, -1/a): S p = a p - H_oe (H_eo p) / a
       EO_RHS = 2,   // (1, -1/a): r_o - H_oe r_e / a
       EO_REC = 3,   // (1/a, -1/a): e_e = (r_e - H_eo e_o) / a
       EO_NSETS = 4 };

struct SolverWS {
    int W = 0;
    int prec = 0;
    bool eo = false;                                          // even-odd inner solve (half fields)
    bool cg = false;                                          // CG on the hermitian Schur complement
    bool split = false;                                       // split fields (see dirac_set_inner_fields)
    int pa = 0, pd = 0;   // precision of e, r, t, tmp, re, ro (pa) and of p, s, tmp2 (pd); = prec unless split
    void *b64 = nullptr, *x64 = nullptr, *r64 = nullptr;     // FP64 internal fields
    // inner fields: whole-lattice fields, or odd half fields when eo
    void *e = nullptr, *r = nullptr, *s = nullptr, *p = nullptr, *t = nullptr;
    void *tmp = nullptr, *re = nullptr, *ro = nullptr;        // eo: even scratch, r_hat halves
    void* tmp2 = nullptr;                                     // split: the adjoint sweep's intermediate
    void* xdf = nullptr;                                      // x in double-float storage (lazy)
    size_t n = 0;                                             // complex numbers per rhs of the inner fields
    double* part = nullptr;                                   // reduction partials
    double* npart = nullptr;                                  // eo: fused-norm partials (W x eo_norm_slots)
    double* scal = nullptr;                                   // per-rhs scalar slots
    int* iflags = nullptr;                                    // active[W], breakdown, nactive
    double *bb, *rr64, *scale, *coef, *rr0, *rr, *gamma, *gnew, *delta, *alpha, *beta, *diag_v, *dim, *itol2;
    float* diag_vf;                                           // diag_v in FP32 for the FP32-arithmetic sweeps
    void* eoc = nullptr;                                      // eo: EO_NSETS x (alpha[W], beta[W]), arithmetic type
    std::vector<double> dh;                                   // host copy of the per-slot diagonal
    cudaStream_t cs = nullptr;          // private stream: graphs cannot be captured on the legacy stream
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // what the graph was captured with
    LaunchCfg g_cfg{0, 0, 0};
    LaunchCfg g_eo_cfg{0, 0, 0};
    const void* g_links = nullptr;
    const void* g_alt = nullptr;
    const void* g_tc = nullptr;
    int g_fmt = 0;
    const double* g_diag = nullptr;
    double g_dval = 0.0;
};

}  // namespace dirac

void dirac_handle::free_solver_workspace()
{
    SolverWS* w = (SolverWS*)sw;
    if (!w) return;
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->cs) cudaStreamDestroy(w->cs);
    void** ptrs[] = {&w->b64, &w->x64, &w->r64, &w->e, &w->r, &w->s, &w->p, &w->t, &w->tmp, &w->re, &w->ro, &w->xdf,
                     &w->tmp2};
    for (void** q : ptrs) release(*q);
    void* pp = w->part;
    release(pp);
    pp = w->npart;
    release(pp);
    pp = w->scal;
    release(pp);
    pp = w->iflags;
    release(pp);
    delete w;
    sw = nullptr;
    sw_bytes = 0;
    sw_nv = 0;
}

static dirac_status ensure_solver_ws(dirac_handle* h, bool eo, bool split, SolverWS** out)
{
    SolverWS* w = (SolverWS*)h->sw;
    if (w && w->W == h->Nv && w->prec == h->prec && w->eo == eo && w->split == split) {
        *out = w;
        return DIRAC_OK;
    }
    h->free_solver_workspace();
    w = new SolverWS();
    h->sw = w;
    w->W = h->Nv;
    w->prec = h->prec;
    w->eo = eo;
    w->split = split;
    w->cg = eo && h->op == OP_STAGGERED;
    w->pa = split ? P_F32 : h->prec;
    w->pd = h->prec;
    const size_t nfull = (size_t)nsc_of(h->op) * nblk_of((size_t)h->g.vol) * 32;
    w->n = eo ? eo_half_n(h->op, h->g.vol) : nfull;
    const size_t f64 = nfull * h->Nv * 16, fa = w->n * h->Nv * cbytes(w->pa), fd = w->n * h->Nv * cbytes(w->pd);
    dirac_status st;
    if ((st = h->alloc(&w->b64, f64, "solver b"))) return st;
    if ((st = h->alloc(&w->x64, f64, "solver x"))) return st;
    if ((st = h->alloc(&w->r64, f64, "solver r"))) return st;
    // e, r, t, tmp, re, ro in pa; s, p, tmp2 in pd
    void** inner[] = {&w->e, &w->r, &w->t, &w->s, &w->p, &w->tmp, &w->re, &w->ro, &w->tmp2};
    const bool in_pa[] = {true, true, true, false, false, true, true, true, false};
    const int ninner = split && eo ? 9 : (eo ? 8 : 5);
    size_t inner_bytes = 0;
    for (int i = 0; i < ninner; ++i) {
        const size_t fb = in_pa[i] ? fa : fd;
        if ((st = h->alloc(inner[i], fb, "solver inner field"))) return st;
        if ((st = h->cuda(cudaMemset(*inner[i], 0, fb), "solver field clear"))) return st;
        inner_bytes += fb;
    }
    // the padding sites of the last block of 32 stay zero (the vector kernels
    // run over whole blocks; the sweeps and packs write only real sites)
    void** fields64[] = {&w->b64, &w->x64, &w->r64};
    for (void** q : fields64)
        if ((st = h->cuda(cudaMemset(*q, 0, f64), "solver field clear"))) return st;
    void* pp = nullptr;
    if ((st = h->alloc(&pp, 2 * blas_partials(nfull, h->Nv) * sizeof(double), "solver partials"))) return st;
    w->part = (double*)pp;
    if (eo) {
        // one partial per warp and column for every launch shape of the even-odd sweeps (32..128 half sites)
        const long vh = h->g.vol / 2;
        if ((st = h->alloc(&pp, (size_t)h->Nv * (size_t)((vh + 31) / 32 + 4) * sizeof(double), "solver norm partials")))
            return st;
        w->npart = (double*)pp;
    }
    const int nslots = 13;
    const size_t nscal = (size_t)nslots * h->Nv + 1 + ((size_t)h->Nv + 1) / 2 + (size_t)EO_NSETS * 2 * h->Nv;
    if ((st = h->alloc(&pp, nscal * sizeof(double), "solver scalars"))) return st;
    w->scal = (double*)pp;
    double** slots[] = {&w->bb, &w->rr64, &w->scale, &w->coef, &w->rr0, &w->rr, &w->gamma,
                        &w->gnew, &w->delta, &w->alpha, &w->beta, &w->diag_v, &w->dim};
    for (int i = 0; i < nslots; ++i) *slots[i] = w->scal + (size_t)i * h->Nv;
    w->itol2 = w->scal + (size_t)nslots * h->Nv;
    w->diag_vf = reinterpret_cast<float*>(w->scal + (size_t)nslots * h->Nv + 1);
    w->eoc = w->scal + (size_t)nslots * h->Nv + 1 + ((size_t)h->Nv + 1) / 2;
    if ((st = h->alloc(&pp, ((size_t)h->Nv + 2) * sizeof(int), "solver flags"))) return st;
    w->iflags = (int*)pp;
    if (split && !eo && (st = h->cuda(brillouin_split_prepare(w->pd, h->stream), "solver: direction table")))
        return st;
    if ((st = h->cuda(cudaStreamCreateWithFlags(&w->cs, cudaStreamNonBlocking), "solver stream"))) return st;
    if ((st = h->cuda(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming), "solver event"))) return st;
    h->sw_bytes = 3 * f64 + inner_bytes;
    h->sw_nv = h->Nv;
    w->dh.assign(h->Nv, h->diag);
    *out = w;
    return DIRAC_OK;
}

// coefficient set k of the even-odd sweeps (device, arithmetic type of the inner fields)
static const void* eo_coef(SolverWS* w, int k)
{
    const size_t esz = w->prec == P_F64 ? sizeof(double) : sizeof(float);
    return (const char*)w->eoc + (size_t)k * 2 * w->W * esz;
}

// uploads the even-odd coefficient sets for the per-slot diagonal w->dh
static dirac_status upload_eo_coef(dirac_handle* h, SolverWS* w)
{
    const int W = w->W;
    std::vector<double> c((size_t)EO_NSETS * 2 * W);
    for (int v = 0; v < W; ++v) {
        const double a = w->dh[v];
        const double al[EO_NSETS] = {0.0, a, 1.0, 1.0 / a};
        const double be[EO_NSETS] = {1.0, -1.0 / a, -1.0 / a, -1.0 / a};
        for (int k = 0; k < EO_NSETS; ++k) {
            c[(size_t)k * 2 * W + v] = al[k];
            c[(size_t)k * 2 * W + W + v] = be[k];
        }
    }
    if (w->prec == P_F64)
        return h->cuda(cudaMemcpyAsync(w->eoc, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice,
                                       h->stream), "solve: even-odd coefficients");
    // pageable source: the copy completes before cudaMemcpyAsync returns, so c may go
    std::vector<float> cf(c.begin(), c.end());
    return h->cuda(cudaMemcpyAsync(w->eoc, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream),
                   "solve: even-odd coefficients");
}

// one even-odd sweep out = alpha in2 + beta H in (or H^+) on the sites of parity par
static LaunchCfg eo_cfg_of(const dirac_handle* h, const SolverWS* w)
{
    LaunchCfg c = h->eo_cfg;
    if (c.R == 0 || !eo_rhs_supported(h->op, w->prec, w->W, c.R))
        c = eo_default_config(h->op, w->prec, w->W, h->g.L[3]);
    return c;
}

// one even-odd sweep with every field in precision w->pa (the links of that
// precision: the handle's, or the FP32 copy of the split solve)
static dirac_status eo_sweep(dirac_handle* h, SolverWS* w, bool dag, int par, void* out, const void* in,
                             const void* in2, int set, double* nrm = nullptr)
{
    const LaunchCfg c = eo_cfg_of(h, w);
    const void* L = h->links;
    dirac_status st;
    if (w->split && (st = h->ensure_links32(&L))) return st;
    EoArgs a = make_eo_args(h->g, w->W, par, in, in2, out, L, eo_coef(w, set), c.order);
    if (nrm) a.npart = w->npart;
    if ((st = h->cuda(launch_eo(h->op, w->pa, dag, a, c, h->stream), "solve: even-odd sweep"))) return st;
    if (!nrm) return DIRAC_OK;
    return h->cuda(blas_reduce_partials(w->npart, eo_norm_slots(a.vh, c.block), w->W, nrm, h->stream),
                   "solve: fused norm");
}

// one sweep of the split solve (EO_SPLIT_*); nrm: |out_v|^2 fused into the sweep
static dirac_status eo_split_sweep(dirac_handle* h, SolverWS* w, int kind, int par, void* out, const void* in,
                                   const void* in2, int set, double* nrm = nullptr)
{
    const LaunchCfg c = eo_cfg_of(h, w);
    const void* L = nullptr;
    dirac_status st;
    if ((st = h->ensure_links32(&L))) return st;
    EoArgs a = make_eo_args(h->g, w->W, par, in, in2, out, L, eo_coef(w, set), c.order);
    if (nrm) a.npart = w->npart;
    if ((st = h->cuda(launch_eo_wilson_split(w->pd, kind, a, c, h->stream), "solve: even-odd sweep"))) return st;
    if (!nrm) return DIRAC_OK;
    return h->cuda(blas_reduce_partials(w->npart, eo_norm_slots(a.vh, c.block), w->W, nrm, h->stream),
                   "solve: fused norm");
}

// out = D in (or D^+ in) on the whole lattice (the inner operator without the
// even-odd split)
static dirac_status apply_inner_whole(dirac_handle* h, SolverWS* w, bool dag, void* out, const void* in,
                                      const double* diag_v)
{
    // the handle's launch shape and link format (a captured graph is
    // rebuilt when either changes, and the format-1 links keep their
    // address across dirac_set_links)
    LaunchCfg c0 = h->cfg;
    if (!w->split)
        return h->run_apply(dag, out, in, w->W, h->diag, h->links, w->prec, c0, diag_v, 0, 0,
                            diag_v ? w->diag_vf : nullptr);
    // split Brillouin fields: t(F32) = D p(16), s(16) = D^+ r(F32) with the
    // FP32 W copy of the split solve, all 80 directions per site (format 1)
    const void* L32 = nullptr;
    dirac_status st;
    if ((st = h->ensure_links32(&L32))) return st;
    ApplyArgs a = h->args(out, in, w->W, h->diag);
    a.links = L32;
    a.diag_v = diag_v;
    a.diag_vf = diag_v ? w->diag_vf : nullptr;
    a.tc = (c0.variant == V_DIRECT || c0.variant == V_GROUPS) ? c0.order : 0;
    if (a.tc > 0) {
        a.fdc = make_fdiv((uint32_t)(h->g.L[2] * a.tc));
        a.fdt = make_fdiv((uint32_t)a.tc);
    }
    return h->cuda(launch_brillouin_split(w->pd, dag, a, c0, h->stream), "solve: split Brillouin sweep");
}

// the Schur complement S (or S^+) on the odd half fields: two half sweeps;
// nrm: |out_v|^2 fused into the second
static dirac_status apply_inner_eo(dirac_handle* h, SolverWS* w, bool dag, void* out, const void* in, double* nrm)
{
    dirac_status st;
    if (w->split) {
        if (!dag) {
            if ((st = eo_split_sweep(h, w, EO_SPLIT_HP, 0, w->tmp, in, nullptr, EO_HOP))) return st;
            return eo_split_sweep(h, w, EO_SPLIT_SP, 1, out, w->tmp, in, EO_S, nrm);
        }
        if ((st = eo_split_sweep(h, w, EO_SPLIT_HR, 0, w->tmp2, in, nullptr, EO_HOP))) return st;
        return eo_split_sweep(h, w, EO_SPLIT_SR, 1, out, w->tmp2, in, EO_S, nrm);
    }
    if ((st = eo_sweep(h, w, dag, 0, w->tmp, in, nullptr, EO_HOP))) return st;   // H_eo in
    return eo_sweep(h, w, dag, 1, out, w->tmp, in, EO_S, nrm);                    // a in - H_oe (.) / a
}

// out = A in (or A^+ in), A the operator of the inner solve: D on the whole
// lattice, or the Schur complement S on the odd half fields.  Split fields:
// A p reads p in 16 bits and writes t in FP32; A^+ r reads r in FP32 and
// writes s in 16 bits.  nrm (optional): |out_v|^2 per right-hand side, fused
// into the second half sweep on the even-odd path, a separate pass on the
// whole lattice.
static dirac_status apply_inner(dirac_handle* h, SolverWS* w, bool dag, void* out, const void* in,
                                const double* diag_v, double* nrm = nullptr)
{
    if (!w->eo) {
        dirac_status st = apply_inner_whole(h, w, dag, out, in, diag_v);
        if (st || !nrm) return st;
        return h->cuda(blas_norm2(dag ? w->pd : w->pa, w->n, w->W, out, w->part, nrm, h->stream), "solve: norm");
    }
    return apply_inner_eo(h, w, dag, out, in, nrm);
}

// one inner iteration over all W right-hand sides (kernel launches only, so it
// can be captured): CGLS on A, or CG when A is hermitian (w->cg)
static dirac_status enqueue_iteration(dirac_handle* h, SolverWS* w, const double* diag_v)
{
    const int W = w->W, P = w->prec;
    const size_t n = w->n;
    cudaStream_t S = h->stream;
    int* active = w->iflags;
    int* breakdown = w->iflags + W;
    int* nactive = w->iflags + W + 1;
    const unsigned sb = (unsigned)((W + 127) / 128);
    dirac_status st;
    if ((st = apply_inner(h, w, false, w->t, w->p, diag_v, w->cg ? nullptr : w->delta))) return st;
    if (w->cg) {
        // t = A p, delta = <p, t>, e += alpha p, r -= alpha t, gamma' = |r|^2, p = r + beta p
        if ((st = h->cuda(blas_dot(P, n, W, w->p, w->t, w->part, w->delta, w->dim, S), "solve: <p, t>")))
            return st;
        k_cg_alpha<<<sb, 128, 0, S>>>(W, w->gamma, w->delta, active, w->alpha, breakdown);
        if ((st = h->cuda(blas_cgls_step(P, n, W, w->alpha, w->e, w->p, w->r, w->t, w->part, w->rr, S),
                          "solve: step")))
            return st;
        k_cgls_beta<<<sb, 128, 0, S>>>(W, w->rr, w->gamma, active, w->beta);
        if ((st = h->cuda(blas_xpay(P, n, W, w->r, w->beta, w->p, S), "solve: p = r + beta p"))) return st;
    } else {
        // t = A p (pa), delta = |t|^2, e += alpha p, r -= alpha t (pa; p in pd),
        // s = A^+ r (pd), gamma' = |s|^2, p = s + beta p (pd); the norms of t
        // and s come with the sweeps that write them
        k_cgls_alpha<<<sb, 128, 0, S>>>(W, w->gamma, w->delta, active, w->alpha, breakdown);
        const cudaError_t ce =
            w->split ? blas_cgls_step_split(w->pd, n, W, w->alpha, w->e, w->p, w->r, w->t, w->part, w->rr, S)
                     : blas_cgls_step(P, n, W, w->alpha, w->e, w->p, w->r, w->t, w->part, w->rr, S);
        if ((st = h->cuda(ce, "solve: step"))) return st;
        if ((st = apply_inner(h, w, true, w->s, w->r, diag_v, w->gnew))) return st;
        k_cgls_beta<<<sb, 128, 0, S>>>(W, w->gnew, w->gamma, active, w->beta);
        if ((st = h->cuda(blas_xpay(w->pd, n, W, w->s, w->beta, w->p, S), "solve: p = s + beta p"))) return st;
    }
    k_cgls_mask<<<1, 256, 0, S>>>(W, w->rr, w->rr0, w->itol2, active, nactive);
    return h->cuda(cudaGetLastError(), "solve: scalar kernels");
}

static dirac_status ensure_graph(dirac_handle* h, SolverWS* w, const double* diag_v)
{
    auto same = [](const LaunchCfg& a, const LaunchCfg& b) {
        return a.R == b.R && a.block == b.block && a.variant == b.variant && a.order == b.order;
    };
    // the whole-lattice sweeps take the handle's diagonal by value (dirac_set_mass may change it)
    if (w->gexec && same(w->g_cfg, h->cfg) && same(w->g_eo_cfg, h->eo_cfg) && w->g_links == h->links &&
        w->g_alt == h->links_alt && w->g_tc == h->links_tc && w->g_fmt == h->link_fmt && w->g_diag == diag_v && w->g_dval == h->diag)
        return DIRAC_OK;
    if (w->gexec) {
        cudaGraphExecDestroy(w->gexec);
        w->gexec = nullptr;
    }
    dirac_status st;
    if ((st = h->cuda(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "solve: begin capture")))
        return st;
    dirac_status est = DIRAC_OK;
    for (int i = 0; i < GRAPH_ITERS && est == DIRAC_OK; ++i) est = enqueue_iteration(h, w, diag_v);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (est) {
        if (graph) cudaGraphDestroy(graph);
        return est;
    }
    if ((st = h->cuda(ce, "solve: end capture"))) return st;
    ce = cudaGraphInstantiate(&w->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if ((st = h->cuda(ce, "solve: graph instantiate"))) return st;
    w->g_cfg = h->cfg;
    w->g_eo_cfg = h->eo_cfg;
    w->g_links = h->links;
    w->g_alt = h->links_alt;
    w->g_tc = h->links_tc;
    w->g_fmt = h->link_fmt;
    w->g_diag = diag_v;
    w->g_dval = h->diag;
    return DIRAC_OK;
}

// Inner solve on the active right-hand sides.  On entry: r holds the
// right-hand side of the inner system (r_hat, or the Schur right-hand side),
// rr0 = |r|^2, active[] is set on the device.  e is zeroed here.  Sweeps are
// counted in whole-lattice equivalents (an application of S is two half
// sweeps: one).
static dirac_status inner_cgls(dirac_handle* h, SolverWS* w, const double* diag_v, int max_inner, double inner_tol,
                               dirac_solve_stats* S_, bool* breakdown_out)
{
    const int W = w->W, P = w->prec;
    const size_t n = w->n;
    cudaStream_t S = h->stream;
    dirac_status st;
    *breakdown_out = false;
    const double itol2 = inner_tol * inner_tol;
    if ((st = h->cuda(cudaMemcpyAsync(w->itol2, &itol2, sizeof(double), cudaMemcpyHostToDevice, S), "solve: copy")))
        return st;
    if ((st = h->cuda(cudaMemsetAsync(w->iflags + W, 0, 2 * sizeof(int), S), "solve: memset"))) return st;
    if ((st = h->cuda(cudaMemsetAsync(w->e, 0, n * W * cbytes(w->pa), S), "solve: e = 0"))) return st;
    if (w->cg) {
        // p = r, gamma = |r|^2
        if ((st = h->cuda(blas_scale_copy(P, n, W, w->r, nullptr, w->p, w->part, w->gamma, S), "solve: p = r")))
            return st;
    } else {
        // s = A^+ r, p = s, gamma = |s|^2
        if ((st = apply_inner(h, w, true, w->s, w->r, diag_v))) return st;
        S_->sweeps++;
        if ((st = h->cuda(blas_scale_copy(w->pd, n, W, w->s, nullptr, w->p, w->part, w->gamma, S), "solve: p = s")))
            return st;
    }
    const int sweeps_per_it = w->cg ? 1 : 2;
    int done = 0, first = 1;
    while (done < max_inner) {
        const int chunk = std::min(GRAPH_ITERS, max_inner - done);
        if (chunk == GRAPH_ITERS && !first) {
            if ((st = ensure_graph(h, w, diag_v))) return st;
            if ((st = h->cuda(cudaGraphLaunch(w->gexec, S), "solve: graph launch"))) return st;
        } else {
            for (int i = 0; i < chunk; ++i)
                if ((st = enqueue_iteration(h, w, diag_v))) return st;
        }
        first = 0;
        done += chunk;
        S_->inner_iterations += chunk;
        S_->sweeps += sweeps_per_it * chunk;
        int flags[2] = {0, 0};   // breakdown, nactive
        if ((st = h->cuda(cudaMemcpyAsync(flags, w->iflags + W, 2 * sizeof(int), cudaMemcpyDeviceToHost, S),
                          "solve: copy")))
            return st;
        if ((st = h->cuda(cudaStreamSynchronize(S), "solve: sync"))) return st;
        if (flags[0]) {
            // a zero or non-finite curvature on an active right-hand side: stop the
            // inner solve and let the FP64 outer residual decide on the update
            *breakdown_out = true;
            break;
        }
        if (trace_on()) {
            std::vector<double> rr(W), rr0(W);
            cudaMemcpy(rr.data(), w->rr, W * sizeof(double), cudaMemcpyDeviceToHost);
            cudaMemcpy(rr0.data(), w->rr0, W * sizeof(double), cudaMemcpyDeviceToHost);
            double mx = 0;
            for (int v = 0; v < W; ++v)
                if (rr0[v] > 0) mx = std::max(mx, std::sqrt(rr[v] / rr0[v]));
            fprintf(stderr, "[dirac] inner it %d: active %d, max |r|/|r_hat| %.3e\n", done, flags[1], mx);
        }
        if (flags[1] == 0) break;
    }
    return DIRAC_OK;
}

// prepare r_hat from r64 for the active right-hand sides and run the inner solve
static dirac_status refine_step(dirac_handle* h, SolverWS* w, const double* diag_v, const std::vector<int>& act,
                                const std::vector<double>& rr64, int max_inner, double inner_tol,
                                dirac_solve_stats* S_)
{
    const int W = w->W;
    const size_t n = (size_t)nsc_of(h->op) * nblk_of((size_t)h->g.vol) * 32;
    cudaStream_t S = h->stream;
    dirac_status st;
    std::vector<double> scale(W), coef(W);
    for (int v = 0; v < W; ++v) {
        scale[v] = act[v] ? std::sqrt((double)n / rr64[v]) : 0.0;
        coef[v] = act[v] ? 1.0 / scale[v] : 0.0;
    }
    if ((st = h->cuda(cudaMemcpyAsync(w->scale, scale.data(), W * sizeof(double), cudaMemcpyHostToDevice, S), "copy")))
        return st;
    if ((st = h->cuda(cudaMemcpyAsync(w->coef, coef.data(), W * sizeof(double), cudaMemcpyHostToDevice, S), "copy")))
        return st;
    if ((st = h->cuda(cudaMemcpyAsync(w->iflags, act.data(), W * sizeof(int), cudaMemcpyHostToDevice, S), "copy")))
        return st;
    bool bd = false;
    if (!w->eo) {
        // r_hat and e in the precision of the inner residual (FP32 with split fields)
        if ((st = h->cuda(blas_convert(P_F64, w->pa, nsc_of(h->op), h->g.vol, W, w->r64, w->scale, w->r, w->part,
                                       w->rr0, S), "solve: r_hat")))
            return st;
        if ((st = inner_cgls(h, w, diag_v, max_inner, inner_tol, S_, &bd))) return st;
        // x += (|r| / sqrt(n)) e in FP64 (the update is kept even after a breakdown:
        // the next FP64 residual decides)
        return h->cuda(blas_axpy_to64(w->pa, nsc_of(h->op), h->g.vol, W, w->coef, w->e, w->x64, S),
                       "solve: x update");
    }
    // even-odd: r_hat -> (r_e, r_o); the Schur right-hand side r = r_o - H_oe r_e / a
    if ((st = upload_eo_coef(h, w))) return st;
    if ((st = h->cuda(eo_split(w->pa, nsc_of(h->op), h->g, W, w->r64, w->scale, w->re, w->ro, S), "solve: r_hat")))
        return st;
    if ((st = eo_sweep(h, w, false, 1, w->r, w->re, w->ro, EO_RHS))) return st;
    if ((st = h->cuda(blas_norm2(w->pa, w->n, W, w->r, w->part, w->rr0, S), "solve: |r|"))) return st;
    if ((st = inner_cgls(h, w, diag_v, max_inner, inner_tol, S_, &bd))) return st;
    // e_e = (r_e - H_eo e_o) / a, then x += (|r| / sqrt(n)) (e_e, e_o)
    if ((st = eo_sweep(h, w, false, 0, w->tmp, w->e, w->re, EO_REC))) return st;
    S_->sweeps++;   // the two half sweeps around the inner solve
    return h->cuda(eo_axpy_to64(w->pa, nsc_of(h->op), h->g, W, w->coef, w->tmp, w->e, w->x64, S), "solve: x update");
}

// r64 = b64 - D x64 with FP64 links and FP64 data, rr64 (host) = |r|^2 per
// slot.  With df the sweep runs in double-float arithmetic (dirac_df.cuh) on
// a double-float copy of x and writes D x (double-float) into r64, which the
// residual kernel then overwrites with b - D x in FP64.
static dirac_status fp64_residual(dirac_handle* h, SolverWS* w, const double* diag_v, std::vector<double>& rr64,
                                  dirac_solve_stats* S_, bool df)
{
    const int W = w->W;
    const size_t n = (size_t)nsc_of(h->op) * nblk_of((size_t)h->g.vol) * 32;
    cudaStream_t S = h->stream;
    dirac_status st;
    if (df) {
        const void* Ldf = nullptr;
        if ((st = h->ensure_links_df(&Ldf))) return st;
        if (!w->xdf && (st = h->alloc(&w->xdf, n * W * 16, "solver x (double-float)"))) return st;
        if ((st = h->cuda(df_from_f64(n * W, w->x64, w->xdf, S), "solve: x to double-float"))) return st;
        ApplyArgs a = h->args(w->r64, w->xdf, W, h->diag);
        a.links = Ldf;
        a.diag_v = diag_v;
        if ((st = h->cuda(launch_apply_df(h->op, a, S), "solve: double-float residual sweep"))) return st;
        if ((st = h->cuda(blas_residual_df(n, W, w->b64, w->r64, w->r64, w->part, w->rr64, S), "solve: residual")))
            return st;
    } else {
        const void* L64 = nullptr;
        if ((st = h->ensure_links64b(&L64))) return st;
        LaunchCfg cfg64 = default_config(h->op, P_F64, W);
        cfg64.fmt = 0;
        if ((st = h->run_apply(false, w->r64, w->x64, W, h->diag, L64, P_F64, cfg64, diag_v))) return st;
        if ((st = h->cuda(blas_residual64(n, W, w->b64, w->r64, w->r64, w->part, w->rr64, S), "solve: residual")))
            return st;
    }
    S_->fp64_sweeps++;
    rr64.resize(W);
    if ((st = h->cuda(cudaMemcpyAsync(rr64.data(), w->rr64, W * sizeof(double), cudaMemcpyDeviceToHost, S), "copy")))
        return st;
    return h->cuda(cudaStreamSynchronize(S), "solve: sync");
}

// whether the outer residual may run in double-float: asked for, and every
// right-hand side's mean square |b|^2 / n well inside FP32's exponent range
// (the halves of a double-float value are FP32 numbers)
static bool use_df(const dirac_handle* h, const std::vector<double>& bb, size_t n)
{
    if (!h->outer_df) return false;
    for (double v : bb) {
        const double ms = v / (double)n;
        if (v > 0.0 && !(ms > 1e-36 && ms < 1e36)) return false;
    }
    return true;
}

// Runs a solve on the workspace's private stream, ordered after the work
// already enqueued on the handle's stream; the handle's stream is restored on
// every return path.  The solvers block until done, so later work on the
// caller's stream is ordered after them as well.
struct OnPrivateStream {
    dirac_handle* h;
    cudaStream_t saved;
    OnPrivateStream(dirac_handle* h_, SolverWS* w) : h(h_), saved(h_->stream)
    {
        cudaEventRecord(w->ev, saved);
        cudaStreamWaitEvent(w->cs, w->ev, 0);
        h->stream = w->cs;
    }
    ~OnPrivateStream()
    {
        cudaStreamSynchronize(h->stream);
        h->stream = saved;
    }
};

// whether the inner solves take the even-odd Schur complement: Wilson or
// staggered, every extent even (so that the hopping term only links opposite
// parities), a nonzero diagonal for every system, and not switched off
static bool use_even_odd(const dirac_handle* h, const double* diag, int ndiag)
{
    if (h->precond == 0 || (h->op != OP_WILSON && h->op != OP_STAGGERED)) return false;
    for (int mu = 0; mu < 4; ++mu)
        if (h->g.L[mu] % 2 != 0) return false;
    for (int i = 0; i < ndiag; ++i)
        if (!(diag[i] != 0.0) || !std::isfinite(diag[i])) return false;
    return true;
}

// inner_tol = 0: the reduction an inner solve can reach with the fields it
// keeps -- FP64 1e-10; FP32 (or split fields, whose residual is FP32) 1e-5;
// FP16 2e-3; BF16 1e-2
static double default_inner_tol(const SolverWS* w)
{
    if (w->pa == P_F64) return 1e-10;
    if (w->pa == P_F32) return 1e-5;
    return w->pd == P_F16 ? 2e-3 : 1e-2;
}

// whether the inner solve keeps split fields: asked for, 16-bit storage, and
// the Wilson even-odd (CGLS) or the Brillouin whole-lattice inner solve
static bool use_split(const dirac_handle* h, bool eo)
{
    return h->inner_fields == 1 && (h->prec == P_BF16 || h->prec == P_F16) &&
           ((eo && h->op == OP_WILSON) || (!eo && h->op == OP_BRILLOUIN));
}

static dirac_status check_solver_args(dirac_handle* h, double tol, int max_outer, int max_inner, double inner_tol,
                                      const char* name)
{
    if (!h->have_links) return h->fail(DIRAC_ERR_INVALID_ARG, "%s: call dirac_set_links first", name);
    if (!(tol > 0.0) || max_outer < 1 || max_inner < 1 || !(inner_tol >= 0.0) || !(inner_tol < 1.0))
        return h->fail(DIRAC_ERR_INVALID_ARG,
                       "%s: need tol > 0, max_outer >= 1, max_inner >= 1, 0 <= inner_tol < 1", name);
    return DIRAC_OK;
}

extern "C" DIRAC_API dirac_status dirac_solve(dirac_handle* h, void* x, const void* b, double tol,
                                              int max_outer, int max_inner, double inner_tol,
                                              double* rel_residual, dirac_solve_stats* stats)
{
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!x || !b || x == b) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve: NULL or aliased x, b");
    dirac_status st;
    if ((st = check_solver_args(h, tol, max_outer, max_inner, inner_tol, "dirac_solve"))) return st;
    if (!dirac_check_device_ptr(x) || !dirac_check_device_ptr(b))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve: x and b must be device pointers");
    if (h->op == OP_BRILLOUIN && (st = h->build_W64())) return st;
    SolverWS* w;
    const bool eo = use_even_odd(h, &h->diag, 1);
    if ((st = ensure_solver_ws(h, eo, use_split(h, eo), &w))) return st;
    w->dh.assign(h->Nv, h->diag);
    if (inner_tol == 0.0) inner_tol = default_inner_tol(w);
    OnPrivateStream guard(h, w);
    const int Nv = h->Nv, nsc = nsc_of(h->op);
    const size_t n = (size_t)nsc * nblk_of((size_t)h->g.vol) * 32;
    cudaStream_t S = h->stream;

#define CK(call, what)                               \
    do {                                             \
        if ((st = h->cuda((call), what))) return st; \
    } while (0)

    dirac_solve_stats S_ = {};
    std::vector<double> bb(Nv), rr64, res(Nv);
    std::vector<int> act(Nv);
    CK(launch_pack_spinor(P_F64, nsc, h->g, Nv, b, true, w->b64, S), "solve: pack b");
    CK(launch_pack_spinor(P_F64, nsc, h->g, Nv, x, true, w->x64, S), "solve: pack x");
    CK(blas_norm2(P_F64, n, Nv, w->b64, w->part, w->bb, S), "solve: |b|");
    CK(cudaMemcpyAsync(bb.data(), w->bb, Nv * sizeof(double), cudaMemcpyDeviceToHost, S), "solve: copy");
    dirac_status result = DIRAC_NOT_CONVERGED;
    int outer = 0;
    CK(cudaStreamSynchronize(S), "solve: sync");   // bb on the host
    const bool df = use_df(h, bb, n);
    for (;; ++outer) {
        if ((st = fp64_residual(h, w, nullptr, rr64, &S_, df))) return st;
        bool all = true, finite = true;
        for (int v = 0; v < Nv; ++v) {
            res[v] = bb[v] > 0.0 ? std::sqrt(rr64[v] / bb[v]) : std::sqrt(rr64[v]);
            if (trace_on()) fprintf(stderr, "[dirac] outer %d rhs %d: |r|/|b| %.3e\n", outer, v, res[v]);
            if (!std::isfinite(res[v])) finite = false;
            act[v] = res[v] > tol;
            all = all && !act[v];
        }
        if (!finite) {
            result = DIRAC_BREAKDOWN;
            break;
        }
        if (all) {
            result = DIRAC_OK;
            break;
        }
        if (outer >= max_outer) break;
        if ((st = refine_step(h, w, nullptr, act, rr64, max_inner, inner_tol, &S_))) return st;
    }
    S_.outer_iterations = outer;
    S_.even_odd = w->eo ? 1 : 0;
    S_.df_residual = df ? 1 : 0;
    S_.split_fields = w->split ? 1 : 0;
    CK(launch_unpack_spinor(P_F64, nsc, h->g, Nv, w->x64, x, true, S), "solve: unpack x");
    CK(cudaStreamSynchronize(S), "solve: sync");
#undef CK
    double rmax = 0.0;
    for (int v = 0; v < Nv; ++v) rmax = std::max(rmax, res[v]);
    S_.residual_max = rmax;
    S_.seconds = std::chrono::duration<double>(clk::now() - t0).count();
    if (rel_residual)
        for (int v = 0; v < Nv; ++v) rel_residual[v] = res[v];
    if (stats) *stats = S_;
    if (result == DIRAC_NOT_CONVERGED)
        h->fail(result, "dirac_solve: max relative residual %.3e > tol %.3e after %d outer steps", rmax, tol, outer);
    else if (result == DIRAC_BREAKDOWN)
        h->fail(result, "dirac_solve: non-finite residual");
    return result;
}

extern "C" DIRAC_API dirac_status dirac_solve_batched(dirac_handle* h, int nsys, const int* Nv_i,
                                                      const double* mass_i, void* const* x_i,
                                                      const void* const* b_i, double tol, int max_outer,
                                                      int max_inner, double inner_tol, double* rel_residual,
                                                      dirac_system_stats* sys_stats, dirac_solve_stats* stats)
{
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (!h) return DIRAC_ERR_INVALID_ARG;
    dirac_status st;
    if (nsys < 1 || !Nv_i || !mass_i || !x_i || !b_i)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve_batched: need nsys >= 1 and non-NULL arrays");
    if ((st = check_solver_args(h, tol, max_outer, max_inner, inner_tol, "dirac_solve_batched"))) return st;
    for (int i = 0; i < nsys; ++i) {
        if (Nv_i[i] < 1) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve_batched: system %d has Nv < 1", i);
        if (h->op == OP_WILSON && !(mass_i[i] > 0.0))
            return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve_batched: system %d: Wilson takes kappa > 0", i);
        if (!x_i[i] || !b_i[i] || x_i[i] == b_i[i] || !dirac_check_device_ptr(x_i[i]) ||
            !dirac_check_device_ptr(b_i[i]))
            return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve_batched: system %d: x, b must be distinct device "
                                                  "pointers", i);
    }
    if (h->op == OP_BRILLOUIN && (st = h->build_W64())) return st;
    std::vector<double> sys_diag(nsys);
    for (int i = 0; i < nsys; ++i) sys_diag[i] = h->diag_of(mass_i[i]);
    SolverWS* w;
    const bool eo = use_even_odd(h, sys_diag.data(), nsys);
    if ((st = ensure_solver_ws(h, eo, use_split(h, eo), &w))) return st;
    if (inner_tol == 0.0) inner_tol = default_inner_tol(w);
    OnPrivateStream guard(h, w);
    const int W = w->W, nsc = nsc_of(h->op);
    const size_t n = (size_t)nsc * nblk_of((size_t)h->g.vol) * 32;
    cudaStream_t S = h->stream;

#define CK(call, what)                               \
    do {                                             \
        if ((st = h->cuda((call), what))) return st; \
    } while (0)

    // the queue of columns, in system order
    std::deque<std::pair<int, int>> queue;
    std::vector<size_t> col_base(nsys + 1, 0);
    for (int i = 0; i < nsys; ++i) {
        for (int c = 0; c < Nv_i[i]; ++c) queue.emplace_back(i, c);
        col_base[i + 1] = col_base[i] + Nv_i[i];
    }
    std::vector<int> slot_sys(W, -1), slot_col(W, -1), slot_outer(W, 0);
    std::vector<double> diag(W, h->diag), bb(W, 0.0), rr64, res_col(col_base[nsys], 0.0);
    std::vector<float> diagf(W);
    std::vector<int> outer_sys(nsys, 0), conv_col(col_base[nsys], 0);
    dirac_solve_stats S_ = {};
    CK(cudaMemsetAsync(w->b64, 0, n * W * 16, S), "batched: clear b");
    CK(cudaMemsetAsync(w->x64, 0, n * W * 16, S), "batched: clear x");
    bool any_breakdown = false;
    bool df = h->outer_df != 0;   // cleared for good once an admitted b is out of the double-float range

    auto retire = [&](int v, double res, bool conv) -> dirac_status {
        const int i = slot_sys[v], c = slot_col[v];
        dirac_status s2 = h->cuda(launch_unpack_column64(nsc, h->g, v, w->x64, Nv_i[i], c, x_i[i], S),
                                  "batched: write back x");
        if (s2) return s2;
        res_col[col_base[i] + c] = res;
        conv_col[col_base[i] + c] = conv;
        outer_sys[i] = std::max(outer_sys[i], slot_outer[v]);
        slot_sys[v] = slot_col[v] = -1;
        // clear the slot (b = x = 0 gives r = 0) so that it stays inert until reused
        s2 = h->cuda(cudaMemsetAsync((char*)w->b64 + (size_t)v * n * 16, 0, n * 16, S), "batched: clear b");
        if (s2) return s2;
        return h->cuda(cudaMemsetAsync((char*)w->x64 + (size_t)v * n * 16, 0, n * 16, S), "batched: clear x");
    };

    for (;;) {
        // admit queued columns into free slots
        bool admitted = false;
        for (int v = 0; v < W && !queue.empty(); ++v) {
            if (slot_sys[v] >= 0) continue;
            auto [i, c] = queue.front();
            queue.pop_front();
            slot_sys[v] = i;
            slot_col[v] = c;
            slot_outer[v] = 0;
            diag[v] = h->diag_of(mass_i[i]);
            CK(launch_pack_column64(nsc, h->g, Nv_i[i], c, b_i[i], v, w->b64, S), "batched: admit b");
            CK(launch_pack_column64(nsc, h->g, Nv_i[i], c, x_i[i], v, w->x64, S), "batched: admit x0");
            admitted = true;
        }
        bool occupied = false;
        for (int v = 0; v < W; ++v) occupied = occupied || slot_sys[v] >= 0;
        if (!occupied) break;
        if (admitted) {
            w->dh = diag;
            CK(cudaMemcpyAsync(w->diag_v, diag.data(), W * sizeof(double), cudaMemcpyHostToDevice, S), "copy");
            diagf.assign(diag.begin(), diag.end());
            CK(cudaMemcpyAsync(w->diag_vf, diagf.data(), W * sizeof(float), cudaMemcpyHostToDevice, S), "copy");
            CK(blas_norm2(P_F64, n, W, w->b64, w->part, w->bb, S), "batched: |b|");
            CK(cudaMemcpyAsync(bb.data(), w->bb, W * sizeof(double), cudaMemcpyDeviceToHost, S), "copy");
        }
        if (admitted) {
            CK(cudaStreamSynchronize(S), "batched: sync");   // bb on the host
            df = df && use_df(h, bb, n);
        }
        if ((st = fp64_residual(h, w, w->diag_v, rr64, &S_, df))) return st;
        std::vector<int> act(W, 0);
        bool freed = false, any_active = false;
        for (int v = 0; v < W; ++v) {
            if (slot_sys[v] < 0) continue;
            const double res = bb[v] > 0.0 ? std::sqrt(rr64[v] / bb[v]) : std::sqrt(rr64[v]);
            if (!std::isfinite(res)) {
                any_breakdown = true;
                if ((st = retire(v, res, false))) return st;
                freed = true;
            } else if (res <= tol) {
                if ((st = retire(v, res, true))) return st;
                freed = true;
            } else if (slot_outer[v] >= max_outer) {
                if ((st = retire(v, res, false))) return st;
                freed = true;
            } else {
                act[v] = 1;
                any_active = true;
            }
        }
        if (freed && !queue.empty()) continue;   // refill the freed slots before the next refinement step
        if (!any_active) continue;
        if ((st = refine_step(h, w, w->diag_v, act, rr64, max_inner, inner_tol, &S_))) return st;
        for (int v = 0; v < W; ++v)
            if (act[v]) slot_outer[v]++;
        S_.outer_iterations++;
    }
    CK(cudaStreamSynchronize(S), "batched: sync");
#undef CK
    bool all_conv = true;
    double rmax = 0.0;
    for (int i = 0; i < nsys; ++i) {
        bool ci = true;
        double ri = 0.0;
        for (int c = 0; c < Nv_i[i]; ++c) {
            ci = ci && conv_col[col_base[i] + c];
            ri = std::max(ri, res_col[col_base[i] + c]);
        }
        all_conv = all_conv && ci;
        rmax = std::max(rmax, ri);
        if (sys_stats) {
            sys_stats[i].converged = ci;
            sys_stats[i].outer_iterations = outer_sys[i];
            sys_stats[i].residual_max = ri;
        }
    }
    if (rel_residual)
        for (size_t k = 0; k < col_base[nsys]; ++k) rel_residual[k] = res_col[k];
    S_.residual_max = rmax;
    S_.even_odd = w->eo ? 1 : 0;
    S_.df_residual = df ? 1 : 0;
    S_.split_fields = w->split ? 1 : 0;
    S_.seconds = std::chrono::duration<double>(clk::now() - t0).count();
    if (stats) *stats = S_;
    if (any_breakdown) return h->fail(DIRAC_BREAKDOWN, "dirac_solve_batched: non-finite residual");
    if (!all_conv)
        return h->fail(DIRAC_NOT_CONVERGED, "dirac_solve_batched: max relative residual %.3e > tol %.3e", rmax, tol);
    return DIRAC_OK;
}
