// Defect-correction (iterative-refinement) solver for D x = b, all Nv
// right-hand sides at once, each with its own scalars and convergence.
//
// Outer loop, FP64 on the GPU (the only FP64 steps): r = b - D x with FP64
// links and an FP64 sweep, per-right-hand-side |r|^2 and |b|^2, stop when
// |r| / |b| <= tol for every right-hand side; otherwise normalise
// r_hat = r * sqrt(n) / |r| (unit RMS, safe for 16-bit storage), solve
// D e = r_hat approximately in the storage precision, and update
// x += (|r| / sqrt(n)) e in FP64.
// Inner solver: CGLS, i.e. conjugate gradients on the normal equations
// D^+ D e = D^+ r_hat, written so that it carries the true residual
// r = r_hat - D e of the unsymmetric system:
//     r = r_hat, s = D^+ r, p = s, gamma = |s|^2
//     loop: t = D p, delta = |t|^2, alpha = gamma / delta,
//           e += alpha p, r -= alpha t, s = D^+ r, gamma' = |s|^2,
//           beta = gamma' / gamma, p = s + beta p
// until |r| <= inner_tol |r_hat|.  Fields are stored in the handle's
// precision; arithmetic is FP32 (FP64 for FP64 handles); norms are FP64.
#include <chrono>
#include <cmath>
#include <vector>

#include "dirac_blas.h"
#include "dirac_handle.h"

using namespace dirac;

namespace dirac {

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

struct SolverWS {
    int Nv = 0;
    int prec = 0;
    void *b64 = nullptr, *x64 = nullptr, *r64 = nullptr;     // FP64 internal fields
    void *e = nullptr, *r = nullptr, *s = nullptr, *p = nullptr, *t = nullptr;   // storage precision
    double* part = nullptr;                                   // reduction partials
    double* scal = nullptr;                                   // per-rhs scalars, see below
    int* iflags = nullptr;                                    // active[Nv], breakdown
    // scalar slots, each Nv doubles
    double *bb, *rr64, *scale, *coef, *rr0, *rr, *gamma, *gnew, *delta, *alpha, *beta;
};

}  // namespace dirac

void dirac_handle::free_solver_workspace()
{
    SolverWS* w = (SolverWS*)sw;
    if (!w) return;
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
    if (w && w->Nv == h->Nv && w->prec == h->prec) {
        *out = w;
        return DIRAC_OK;
    }
    h->free_solver_workspace();
    w = new SolverWS();
    h->sw = w;
    w->Nv = h->Nv;
    w->prec = h->prec;
    const size_t n = (size_t)nsc_of(h->op) * h->g.vol;
    const size_t f64 = n * h->Nv * 16, fp = n * h->Nv * cbytes(h->prec);
    dirac_status st;
    if ((st = h->alloc(&w->b64, f64, "solver b"))) return st;
    if ((st = h->alloc(&w->x64, f64, "solver x"))) return st;
    if ((st = h->alloc(&w->r64, f64, "solver r"))) return st;
    void** inner[] = {&w->e, &w->r, &w->s, &w->p, &w->t};
    for (void** q : inner)
        if ((st = h->alloc(q, fp, "solver inner field"))) return st;
    void* pp = nullptr;
    if ((st = h->alloc(&pp, 2 * blas_partials(n, h->Nv) * sizeof(double), "solver partials"))) return st;
    w->part = (double*)pp;
    if ((st = h->alloc(&pp, 11 * (size_t)h->Nv * sizeof(double), "solver scalars"))) return st;
    w->scal = (double*)pp;
    double** slots[] = {&w->bb, &w->rr64, &w->scale, &w->coef, &w->rr0, &w->rr,
                        &w->gamma, &w->gnew, &w->delta, &w->alpha, &w->beta};
    for (int i = 0; i < 11; ++i) *slots[i] = w->scal + (size_t)i * h->Nv;
    if ((st = h->alloc(&pp, ((size_t)h->Nv + 1) * sizeof(int), "solver flags"))) return st;
    w->iflags = (int*)pp;
    h->sw_bytes = 3 * f64 + 5 * fp;
    h->sw_nv = h->Nv;
    *out = w;
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
    if (!h->have_links) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve: call dirac_set_links first");
    if (!(tol > 0.0) || max_outer < 1 || max_inner < 1 || !(inner_tol > 0.0) || !(inner_tol < 1.0))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve: need tol > 0, max_outer >= 1, max_inner >= 1, "
                                              "0 < inner_tol < 1");
    if (!dirac_check_device_ptr(x) || !dirac_check_device_ptr(b))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_solve: x and b must be device pointers");
    dirac_status st;
    if (h->op == OP_BRILLOUIN && (st = h->build_W64())) return st;
    SolverWS* w;
    if ((st = ensure_solver_ws(h, &w))) return st;
    const int Nv = h->Nv, P = h->prec, nsc = nsc_of(h->op);
    const size_t n = (size_t)nsc * h->g.vol;
    cudaStream_t S = h->stream;
    const void* L64 = (h->op == OP_BRILLOUIN) ? h->W64 : h->links64;
    const LaunchCfg cfg64 = default_config(h->op, P_F64, Nv);
    int* active = w->iflags;
    int* breakdown = w->iflags + Nv;
    const unsigned sb = (unsigned)((Nv + 127) / 128);

    dirac_solve_stats S_ = {};
    std::vector<double> bb(Nv), rr64(Nv), res(Nv), scale(Nv), coef(Nv), rrv(Nv), rr0(Nv);
    std::vector<int> act(Nv);

#define CK(call, what)                               \
    do {                                             \
        if ((st = h->cuda((call), what))) return st; \
    } while (0)

    CK(launch_pack_spinor(P_F64, nsc, h->g, Nv, b, true, w->b64, S), "solve: pack b");
    CK(launch_pack_spinor(P_F64, nsc, h->g, Nv, x, true, w->x64, S), "solve: pack x");
    CK(blas_norm2(P_F64, n, Nv, w->b64, w->part, w->bb, S), "solve: |b|");
    CK(cudaMemcpyAsync(bb.data(), w->bb, Nv * sizeof(double), cudaMemcpyDeviceToHost, S), "solve: copy");
    dirac_status result = DIRAC_NOT_CONVERGED;
    int outer = 0;
    for (;; ++outer) {
        // r = b - D x in FP64
        if ((st = h->run_apply(false, w->r64, w->x64, Nv, h->diag, L64, P_F64, cfg64))) return st;
        S_.fp64_sweeps++;
        CK(blas_residual64(n, Nv, w->b64, w->r64, w->r64, w->part, w->rr64, S), "solve: residual");
        CK(cudaMemcpyAsync(rr64.data(), w->rr64, Nv * sizeof(double), cudaMemcpyDeviceToHost, S), "solve: copy");
        CK(cudaStreamSynchronize(S), "solve: sync");
        bool all = true, finite = true;
        for (int v = 0; v < Nv; ++v) {
            res[v] = bb[v] > 0.0 ? std::sqrt(rr64[v] / bb[v]) : std::sqrt(rr64[v]);
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
        // r_hat = r sqrt(n) / |r|  in the storage precision
        for (int v = 0; v < Nv; ++v) {
            scale[v] = act[v] ? std::sqrt((double)n / rr64[v]) : 0.0;
            coef[v] = act[v] ? 1.0 / scale[v] : 0.0;
        }
        CK(cudaMemcpyAsync(w->scale, scale.data(), Nv * sizeof(double), cudaMemcpyHostToDevice, S), "solve: copy");
        CK(cudaMemcpyAsync(w->coef, coef.data(), Nv * sizeof(double), cudaMemcpyHostToDevice, S), "solve: copy");
        CK(cudaMemcpyAsync(active, act.data(), Nv * sizeof(int), cudaMemcpyHostToDevice, S), "solve: copy");
        CK(cudaMemsetAsync(breakdown, 0, sizeof(int), S), "solve: memset");
        CK(blas_scale_copy(P_F64, P, n, Nv, w->r64, w->scale, w->r, w->part, w->rr0, S), "solve: r_hat");
        CK(cudaMemsetAsync(w->e, 0, n * Nv * cbytes(P), S), "solve: e = 0");
        // s = D^+ r, p = s, gamma = |s|^2
        if ((st = h->run_apply(true, w->s, w->r, Nv, h->diag, h->links, P, h->cfg))) return st;
        S_.sweeps++;
        CK(blas_scale_copy(P, P, n, Nv, w->s, nullptr, w->p, w->part, w->gamma, S), "solve: p = s");
        CK(cudaMemcpyAsync(rr0.data(), w->rr0, Nv * sizeof(double), cudaMemcpyDeviceToHost, S), "solve: copy");
        const double itol2 = inner_tol * inner_tol;
        const int check_every = 8;
        for (int it = 1; it <= max_inner; ++it) {
            if ((st = h->run_apply(false, w->t, w->p, Nv, h->diag, h->links, P, h->cfg))) return st;
            CK(blas_norm2(P, n, Nv, w->t, w->part, w->delta, S), "solve: |t|");
            k_cgls_alpha<<<sb, 128, 0, S>>>(Nv, w->gamma, w->delta, active, w->alpha, breakdown);
            CK(blas_cgls_step(P, n, Nv, w->alpha, w->e, w->p, w->r, w->t, w->part, w->rr, S), "solve: step");
            if ((st = h->run_apply(true, w->s, w->r, Nv, h->diag, h->links, P, h->cfg))) return st;
            CK(blas_norm2(P, n, Nv, w->s, w->part, w->gnew, S), "solve: |s|");
            k_cgls_beta<<<sb, 128, 0, S>>>(Nv, w->gnew, w->gamma, active, w->beta);
            CK(blas_xpay(P, n, Nv, w->s, w->beta, w->p, S), "solve: p = s + beta p");
            S_.sweeps += 2;
            S_.inner_iterations++;
            if (it % check_every == 0 || it == max_inner) {
                int bd = 0;
                CK(cudaMemcpyAsync(rrv.data(), w->rr, Nv * sizeof(double), cudaMemcpyDeviceToHost, S), "solve: copy");
                CK(cudaMemcpyAsync(&bd, breakdown, sizeof(int), cudaMemcpyDeviceToHost, S), "solve: copy");
                CK(cudaStreamSynchronize(S), "solve: sync");
                bool any = false, changed = false;
                for (int v = 0; v < Nv; ++v) {
                    if (act[v] && (rrv[v] <= itol2 * rr0[v] || !std::isfinite(rrv[v]))) {
                        act[v] = 0;
                        changed = true;
                    }
                    any = any || act[v];
                }
                if (bd && any) {
                    // a zero or non-finite curvature on an active right-hand side: stop the
                    // inner solve here and let the outer FP64 residual judge the update
                    break;
                }
                if (!any) break;
                if (changed)
                    CK(cudaMemcpyAsync(active, act.data(), Nv * sizeof(int), cudaMemcpyHostToDevice, S), "solve: copy");
            }
        }
        // x += (|r| / sqrt(n)) e in FP64
        CK(blas_axpy_to64(P, n, Nv, w->coef, w->e, w->x64, S), "solve: x update");
    }
    S_.outer_iterations = outer;
    CK(launch_unpack_spinor(P_F64, nsc, h->g, Nv, w->x64, x, true, S), "solve: unpack x");
    CK(cudaStreamSynchronize(S), "solve: sync");
    double rmax = 0.0;
    for (int v = 0; v < Nv; ++v) rmax = std::max(rmax, res[v]);
    S_.residual_max = rmax;
    S_.seconds = std::chrono::duration<double>(clk::now() - t0).count();
    if (rel_residual)
        for (int v = 0; v < Nv; ++v) rel_residual[v] = res[v];
    if (stats) *stats = S_;
#undef CK
    if (result == DIRAC_NOT_CONVERGED)
        h->fail(result, "dirac_solve: max relative residual %.3e > tol %.3e after %d outer steps", rmax, tol, outer);
    else if (result == DIRAC_BREAKDOWN)
        h->fail(result, "dirac_solve: non-finite residual");
    return result;
}
