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
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <vector>

#include "dirac_blas.h"
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

struct SolverWS {
    int W = 0;
    int prec = 0;
    void *b64 = nullptr, *x64 = nullptr, *r64 = nullptr;     // FP64 internal fields
    void *e = nullptr, *r = nullptr, *s = nullptr, *p = nullptr, *t = nullptr;   // storage precision
    double* part = nullptr;                                   // reduction partials
    double* scal = nullptr;                                   // per-rhs scalar slots
    int* iflags = nullptr;                                    // active[W], breakdown, nactive
    double *bb, *rr64, *scale, *coef, *rr0, *rr, *gamma, *gnew, *delta, *alpha, *beta, *diag_v, *itol2;
    float* diag_vf;                                           // diag_v in FP32 for the FP32-arithmetic sweeps
    cudaStream_t cs = nullptr;          // private stream: graphs cannot be captured on the legacy stream
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // what the graph was captured with
    LaunchCfg g_cfg{0, 0, 0};
    const void* g_links = nullptr;
    const double* g_diag = nullptr;
};

}  // namespace dirac

void dirac_handle::free_solver_workspace()
{
    SolverWS* w = (SolverWS*)sw;
    if (!w) return;
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->cs) cudaStreamDestroy(w->cs);
    void** ptrs[] = {&w->b64, &w->x64, &w->r64, &w->e, &w->r, &w->s, &w->p, &w->t};
    for (void** q : ptrs) release(*q);
    void* pp = w->part;
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

static dirac_status ensure_solver_ws(dirac_handle* h, SolverWS** out)
{
    SolverWS* w = (SolverWS*)h->sw;
    if (w && w->W == h->Nv && w->prec == h->prec) {
        *out = w;
        return DIRAC_OK;
    }
    h->free_solver_workspace();
    w = new SolverWS();
    h->sw = w;
    w->W = h->Nv;
    w->prec = h->prec;
    const size_t n = (size_t)nsc_of(h->op) * nblk_of((size_t)h->g.vol) * 32;
    const size_t f64 = n * h->Nv * 16, fp = n * h->Nv * cbytes(h->prec);
    dirac_status st;
    if ((st = h->alloc(&w->b64, f64, "solver b"))) return st;
    if ((st = h->alloc(&w->x64, f64, "solver x"))) return st;
    if ((st = h->alloc(&w->r64, f64, "solver r"))) return st;
    void** inner[] = {&w->e, &w->r, &w->s, &w->p, &w->t};
    for (void** q : inner)
        if ((st = h->alloc(q, fp, "solver inner field"))) return st;
    // the padding sites of the last block of 32 stay zero (the vector kernels
    // run over whole blocks; the sweeps and packs write only real sites)
    void** fields64[] = {&w->b64, &w->x64, &w->r64};
    for (void** q : fields64)
        if ((st = h->cuda(cudaMemset(*q, 0, f64), "solver field clear"))) return st;
    for (void** q : inner)
        if ((st = h->cuda(cudaMemset(*q, 0, fp), "solver field clear"))) return st;
    void* pp = nullptr;
    if ((st = h->alloc(&pp, 2 * blas_partials(n, h->Nv) * sizeof(double), "solver partials"))) return st;
    w->part = (double*)pp;
    const int nslots = 12;
    if ((st = h->alloc(&pp, ((size_t)nslots * h->Nv + 1 + ((size_t)h->Nv + 1) / 2) * sizeof(double), "solver scalars")))
        return st;
    w->scal = (double*)pp;
    double** slots[] = {&w->bb, &w->rr64, &w->scale, &w->coef, &w->rr0, &w->rr,
                        &w->gamma, &w->gnew, &w->delta, &w->alpha, &w->beta, &w->diag_v};
    for (int i = 0; i < nslots; ++i) *slots[i] = w->scal + (size_t)i * h->Nv;
    w->itol2 = w->scal + (size_t)nslots * h->Nv;
    w->diag_vf = reinterpret_cast<float*>(w->scal + (size_t)nslots * h->Nv + 1);
    if ((st = h->alloc(&pp, ((size_t)h->Nv + 2) * sizeof(int), "solver flags"))) return st;
    w->iflags = (int*)pp;
    if ((st = h->cuda(cudaStreamCreateWithFlags(&w->cs, cudaStreamNonBlocking), "solver stream"))) return st;
    if ((st = h->cuda(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming), "solver event"))) return st;
    h->sw_bytes = 3 * f64 + 5 * fp;
    h->sw_nv = h->Nv;
    *out = w;
    return DIRAC_OK;
}

// one CGLS iteration over all W right-hand sides (kernel launches only, so it
// can be captured)
static dirac_status enqueue_iteration(dirac_handle* h, SolverWS* w, const double* diag_v)
{
    const int W = w->W, P = w->prec;
    const size_t n = (size_t)nsc_of(h->op) * nblk_of((size_t)h->g.vol) * 32;
    cudaStream_t S = h->stream;
    int* active = w->iflags;
    int* breakdown = w->iflags + W;
    int* nactive = w->iflags + W + 1;
    const unsigned sb = (unsigned)((W + 127) / 128);
    dirac_status st;
    const float* dvf = diag_v ? w->diag_vf : nullptr;
    if ((st = h->run_apply(false, w->t, w->p, W, h->diag, h->links, P, h->cfg, diag_v, 0, 0, dvf))) return st;
    if ((st = h->cuda(blas_norm2(P, n, W, w->t, w->part, w->delta, S), "solve: |t|"))) return st;
    k_cgls_alpha<<<sb, 128, 0, S>>>(W, w->gamma, w->delta, active, w->alpha, breakdown);
    if ((st = h->cuda(blas_cgls_step(P, n, W, w->alpha, w->e, w->p, w->r, w->t, w->part, w->rr, S), "solve: step")))
        return st;
    if ((st = h->run_apply(true, w->s, w->r, W, h->diag, h->links, P, h->cfg, diag_v, 0, 0, dvf))) return st;
    if ((st = h->cuda(blas_norm2(P, n, W, w->s, w->part, w->gnew, S), "solve: |s|"))) return st;
    k_cgls_beta<<<sb, 128, 0, S>>>(W, w->gnew, w->gamma, active, w->beta);
    if ((st = h->cuda(blas_xpay(P, n, W, w->s, w->beta, w->p, S), "solve: p = s + beta p"))) return st;
    k_cgls_mask<<<1, 256, 0, S>>>(W, w->rr, w->rr0, w->itol2, active, nactive);
    return h->cuda(cudaGetLastError(), "solve: scalar kernels");
}

static dirac_status ensure_graph(dirac_handle* h, SolverWS* w, const double* diag_v)
{
    if (w->gexec && w->g_cfg.R == h->cfg.R && w->g_cfg.block == h->cfg.block && w->g_cfg.variant == h->cfg.variant &&
        w->g_cfg.order == h->cfg.order && w->g_links == h->links && w->g_diag == diag_v)
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
    w->g_links = h->links;
    w->g_diag = diag_v;
    return DIRAC_OK;
}

// Inner CGLS on the active right-hand sides.  On entry: r holds r_hat, rr0 =
// |r_hat|^2, active[] is set on the device.  e is zeroed here.
static dirac_status inner_cgls(dirac_handle* h, SolverWS* w, const double* diag_v, int max_inner, double inner_tol,
                               dirac_solve_stats* S_, bool* breakdown_out)
{
    const int W = w->W, P = w->prec;
    const size_t n = (size_t)nsc_of(h->op) * nblk_of((size_t)h->g.vol) * 32;
    cudaStream_t S = h->stream;
    dirac_status st;
    *breakdown_out = false;
    const double itol2 = inner_tol * inner_tol;
    if ((st = h->cuda(cudaMemcpyAsync(w->itol2, &itol2, sizeof(double), cudaMemcpyHostToDevice, S), "solve: copy")))
        return st;
    if ((st = h->cuda(cudaMemsetAsync(w->iflags + W, 0, 2 * sizeof(int), S), "solve: memset"))) return st;
    if ((st = h->cuda(cudaMemsetAsync(w->e, 0, n * W * cbytes(P), S), "solve: e = 0"))) return st;
    // s = D^+ r, p = s, gamma = |s|^2
    if ((st = h->run_apply(true, w->s, w->r, W, h->diag, h->links, P, h->cfg, diag_v, 0, 0,
                           diag_v ? w->diag_vf : nullptr)))
        return st;
    S_->sweeps++;
    if ((st = h->cuda(blas_scale_copy(P, n, W, w->s, nullptr, w->p, w->part, w->gamma, S), "solve: p = s")))
        return st;
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
        S_->sweeps += 2 * chunk;
        int flags[2] = {0, 0};   // breakdown, nactive
        if ((st = h->cuda(cudaMemcpyAsync(flags, w->iflags + W, 2 * sizeof(int), cudaMemcpyDeviceToHost, S),
                          "solve: copy")))
            return st;
        if ((st = h->cuda(cudaStreamSynchronize(S), "solve: sync"))) return st;
        if (flags[0]) {
            // a zero or non-finite curvature on an active right-hand side: stop the
            // inner solve and let the FP64 outer residual judge the update
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
    const int W = w->W, P = w->prec;
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
    if ((st = h->cuda(blas_convert(P_F64, P, nsc_of(h->op), h->g.vol, W, w->r64, w->scale, w->r, w->part, w->rr0, S),
                      "solve: r_hat")))
        return st;
    bool bd = false;
    if ((st = inner_cgls(h, w, diag_v, max_inner, inner_tol, S_, &bd))) return st;
    // x += (|r| / sqrt(n)) e in FP64 (the update is kept even after a breakdown:
    // the next FP64 residual decides)
    return h->cuda(blas_axpy_to64(P, nsc_of(h->op), h->g.vol, W, w->coef, w->e, w->x64, S), "solve: x update");
}

// r64 = b64 - D x64 in FP64; rr64 (host) = |r|^2 per slot
static dirac_status fp64_residual(dirac_handle* h, SolverWS* w, const double* diag_v, std::vector<double>& rr64,
                                  dirac_solve_stats* S_)
{
    const int W = w->W;
    const size_t n = (size_t)nsc_of(h->op) * nblk_of((size_t)h->g.vol) * 32;
    cudaStream_t S = h->stream;
    const void* L64 = nullptr;
    dirac_status st;
    if ((st = h->ensure_links64b(&L64))) return st;
    const LaunchCfg cfg64 = default_config(h->op, P_F64, W);
    if ((st = h->run_apply(false, w->r64, w->x64, W, h->diag, L64, P_F64, cfg64, diag_v))) return st;
    S_->fp64_sweeps++;
    if ((st = h->cuda(blas_residual64(n, W, w->b64, w->r64, w->r64, w->part, w->rr64, S), "solve: residual")))
        return st;
    rr64.resize(W);
    if ((st = h->cuda(cudaMemcpyAsync(rr64.data(), w->rr64, W * sizeof(double), cudaMemcpyDeviceToHost, S), "copy")))
        return st;
    return h->cuda(cudaStreamSynchronize(S), "solve: sync");
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

static dirac_status check_solver_args(dirac_handle* h, double tol, int max_outer, int max_inner, double inner_tol,
                                      const char* name)
{
    if (!h->have_links) return h->fail(DIRAC_ERR_INVALID_ARG, "%s: call dirac_set_links first", name);
    if (!(tol > 0.0) || max_outer < 1 || max_inner < 1 || !(inner_tol > 0.0) || !(inner_tol < 1.0))
        return h->fail(DIRAC_ERR_INVALID_ARG,
                       "%s: need tol > 0, max_outer >= 1, max_inner >= 1, 0 < inner_tol < 1", name);
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
    if ((st = ensure_solver_ws(h, &w))) return st;
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
    for (;; ++outer) {
        if ((st = fp64_residual(h, w, nullptr, rr64, &S_))) return st;
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
    SolverWS* w;
    if ((st = ensure_solver_ws(h, &w))) return st;
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
            CK(cudaMemcpyAsync(w->diag_v, diag.data(), W * sizeof(double), cudaMemcpyHostToDevice, S), "copy");
            diagf.assign(diag.begin(), diag.end());
            CK(cudaMemcpyAsync(w->diag_vf, diagf.data(), W * sizeof(float), cudaMemcpyHostToDevice, S), "copy");
            CK(blas_norm2(P_F64, n, W, w->b64, w->part, w->bb, S), "batched: |b|");
            CK(cudaMemcpyAsync(bb.data(), w->bb, W * sizeof(double), cudaMemcpyDeviceToHost, S), "copy");
        }
        if ((st = fp64_residual(h, w, w->diag_v, rr64, &S_))) return st;
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
    S_.seconds = std::chrono::duration<double>(clk::now() - t0).count();
    if (stats) *stats = S_;
    if (any_breakdown) return h->fail(DIRAC_BREAKDOWN, "dirac_solve_batched: non-finite residual");
    if (!all_conv)
        return h->fail(DIRAC_NOT_CONVERGED, "dirac_solve_batched: max relative residual %.3e > tol %.3e", rmax, tol);
    return DIRAC_OK;
}
