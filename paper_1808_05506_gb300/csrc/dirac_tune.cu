// Autotuner: the "best of breed" selection of Sec. 4 and Sec. 6 (build every
// variant, time a few calls, keep the winner for this machine) applied to
// the launch shape of the sweeps: right-hand sides per thread R, threads
// per block, launch variant and (variants 0 and 1) the site order.  Results can be kept in a plain-text cache file named by the
// environment variable DIRAC_TUNE_CACHE, one line per
// (operator, precision, lattice, Nv, device name).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dirac_eo.cuh"
#include "dirac_handle.h"

using namespace dirac;

static std::mutex g_cache_mu;

static std::string tune_key(const dirac_handle* h)
{
    cudaDeviceProp p;
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&p, h->device) == cudaSuccess) dev = p.name;
    for (auto& c : dev)
        if (c == ' ') c = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "op%d prec%d %dx%dx%dx%d nv%d %s", h->op, h->prec, h->g.L[0], h->g.L[1],
             h->g.L[2], h->g.L[3], h->Nv, dev.c_str());
    return buf;
}

// an entry: "<key> R<R> B<block> P<variant> T<order> F<link format> <ms>"
// (lines written without F read as format 0)
static bool cache_lookup(const std::string& key, int* R, int* B, int* Pp, int* T, double* ms, int* F = nullptr)
{
    const char* path = getenv("DIRAC_TUNE_CACHE");
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        const size_t kl = key.size();
        if (strncmp(line, key.c_str(), kl) == 0 && line[kl] == ' ') {
            int r, b, tc, pp, fm = 0;
            double t;
            if (sscanf(line + kl, " R%d B%d P%d T%d F%d %lf", &r, &b, &pp, &tc, &fm, &t) == 6 ||
                (fm = 0, sscanf(line + kl, " R%d B%d P%d T%d %lf", &r, &b, &pp, &tc, &t) == 5)) {
                *R = r;
                *B = b;
                *Pp = pp;
                *T = tc;
                *ms = t;
                if (F) *F = fm;
                found = true;   // the last entry wins
            }
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const std::string& key, int R, int B, int Pp, int T, double ms, int F = 0)
{
    const char* path = getenv("DIRAC_TUNE_CACHE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s R%d B%d P%d T%d F%d %.6f\n", key.c_str(), R, B, Pp, T, F, ms);
    fclose(f);
}

static bool trace_tune()
{
    const char* tr = getenv("DIRAC_TRACE");
    return tr && *tr && *tr != '0';
}

// The even-odd sweep of the inner solves (dirac_eo.cuh), when the handle's
// operator and lattice allow it: R in {1, 2, 4} (those built for Nv), 32, 64
// or 128 half sites per block, lexicographic or t-chunked site order; timed
// as the second sweep of an application of the Schur complement (both input
// fields read).  Kept in h->eo_cfg and in the cache under "eo <key>".
static dirac_status tune_even_odd(dirac_handle* h, int force)
{
    if ((h->op != OP_WILSON && h->op != OP_STAGGERED) || h->g.L[0] % 2 || h->g.L[1] % 2 || h->g.L[2] % 2 ||
        h->g.L[3] % 2)
        return DIRAC_OK;
    const std::string key = "eo " + tune_key(h);
    int R = 0, B = 0, Pp = 0, Tc = 0;
    double best = 0.0;
    if (!force && cache_lookup(key, &R, &B, &Pp, &Tc, &best) && eo_rhs_supported(h->op, h->prec, h->Nv, R) &&
        (B == 32 || B == 64 || B == 128) && Tc >= 0 && Tc <= h->g.L[3]) {
        h->eo_cfg = LaunchCfg{R, B, 0, Tc};
        return DIRAC_OK;
    }
    dirac_status st;
    if ((st = h->ensure_workspace())) return st;
    // ws_in: both inputs (a half field fits a whole-lattice one); ws_out: the output
    if ((st = h->cuda(cudaMemsetAsync(h->ws_in, 0, h->field_bytes_internal(h->Nv), h->stream), "autotune")))
        return st;
    void* coef = nullptr;
    const size_t esz = h->prec == P_F64 ? sizeof(double) : sizeof(float);
    if ((st = h->alloc(&coef, 2 * (size_t)h->Nv * esz, "autotune coefficients"))) return st;
    if ((st = h->cuda(cudaMemsetAsync(coef, 0, 2 * (size_t)h->Nv * esz, h->stream), "autotune"))) {
        h->release(coef);
        return st;
    }
    cudaEvent_t e0, e1;
    if ((st = h->cuda(cudaEventCreate(&e0), "autotune"))) {
        h->release(coef);
        return st;
    }
    if ((st = h->cuda(cudaEventCreate(&e1), "autotune"))) {
        cudaEventDestroy(e0);
        h->release(coef);
        return st;
    }
    best = 1e30;
    LaunchCfg win = eo_default_config(h->op, h->prec, h->Nv, h->g.L[3]);
    const int Rs[] = {1, 2, 4}, blocks[] = {32, 64, 128};
    for (int r : Rs) {
        if (!eo_rhs_supported(h->op, h->prec, h->Nv, r)) continue;
        for (int b : blocks)
            for (int oi = 0; oi < 2 && st == DIRAC_OK; ++oi) {
                const LaunchCfg c{r, b, 0, oi == 0 ? 0 : std::min(8, h->g.L[3])};
                const EoArgs a = make_eo_args(h->g, h->Nv, 1, h->ws_in, h->ws_in, h->ws_out, h->links, coef, c.order);
                std::vector<float> t;
                for (int rep = 0; rep < 7 && st == DIRAC_OK; ++rep) {
                    cudaEventRecord(e0, h->stream);
                    st = h->cuda(launch_eo(h->op, h->prec, false, a, c, h->stream), "autotune: even-odd sweep");
                    cudaEventRecord(e1, h->stream);
                    if (!st) st = h->cuda(cudaEventSynchronize(e1), "autotune");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep >= 2) t.push_back(ms);
                }
                if (st) break;
                std::sort(t.begin(), t.end());
                const double med = t[t.size() / 2];
                if (trace_tune())
                    fprintf(stderr, "[dirac] autotune %s R=%d block=%d order=%d: %.4f ms\n", key.c_str(), r, b,
                            c.order, med);
                if (med < best) {
                    best = med;
                    win = c;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->release(coef);
    if (st) return st;
    h->eo_cfg = win;
    cache_store(key, win.R, win.block, 0, win.order, best);
    return DIRAC_OK;
}

extern "C" DIRAC_API dirac_status dirac_autotune(dirac_handle* h, int force, int* R_out, int* block_out,
                                                 int* variant_out, double* ms_out)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!h->have_links) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_autotune: call dirac_set_links first");
    const std::string key = tune_key(h);
    int R = 0, B = 0, Pp = 0, Tc = 0, Fm = 0;
    double best = 0.0;
    if (!force && cache_lookup(key, &R, &B, &Pp, &Tc, &best, &Fm) &&
        apply_config_supported(h->op, h->prec, R, B, Pp, h->g) && Tc >= 0 && Tc <= h->g.L[3]) {
        h->cfg = LaunchCfg{R, B, Pp, Tc};
        // the cached link format, if these links allow it
        if (dirac_set_link_format(h, Fm) != DIRAC_OK) dirac_set_link_format(h, 0);
    } else {
        dirac_status st;
        if ((st = h->ensure_workspace())) return st;
        if ((st = h->cuda(cudaMemsetAsync(h->ws_in, 0, h->field_bytes_internal(h->Nv), h->stream), "autotune")))
            return st;
        std::vector<int> Rs = (h->op == OP_STAGGERED) ? std::vector<int>{1, 2, 4, 6} : std::vector<int>{1, 2, 3, 4};
        const int blocks[] = {32, 64, 128, 256};
        cudaEvent_t e0, e1;
        if ((st = h->cuda(cudaEventCreate(&e0), "autotune"))) return st;
        if ((st = h->cuda(cudaEventCreate(&e1), "autotune"))) {
            cudaEventDestroy(e0);
            return st;
        }
        // median of 5 timed calls after 2 warm-up calls; false if the shape
        // cannot run here or a kernel recorded a failure (never picked)
        auto time_cfg = [&](const LaunchCfg& c, double* med) -> bool {
            std::vector<float> t;
            cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream);
            for (int rep = 0; rep < 7 && st == DIRAC_OK; ++rep) {
                cudaEventRecord(e0, h->stream);
                const dirac_status ls = h->run_apply(false, h->ws_out, h->ws_in, h->Nv, h->diag, h->links, h->prec, c);
                if (ls != DIRAC_OK) {
                    cudaGetLastError();
                    return false;
                }
                cudaEventRecord(e1, h->stream);
                st = h->cuda(cudaEventSynchronize(e1), "autotune");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep >= 2) t.push_back(ms);   // two warm-up calls
            }
            if (st) return false;
            int kerr = 0;
            cudaMemcpy(&kerr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
            if (kerr) {
                cudaMemset(h->dev_err, 0, sizeof(int));
                return false;
            }
            std::sort(t.begin(), t.end());
            *med = t[t.size() / 2];
            const char* tr = getenv("DIRAC_TRACE");
            if (tr && *tr && *tr != '0')
                fprintf(stderr, "[dirac] autotune %s R=%d block=%d variant=%d order=%d format=%d: %.4f ms\n",
                        key.c_str(), c.R, c.block, c.variant, c.order, c.fmt, *med);
            return true;
        };
        best = 1e30;
        LaunchCfg win = h->cfg;
        win.fmt = 0;
        const int variants[] = {V_DIRECT, V_GROUPS, V_TMARCH, V_PIPE3, V_XROW, V_XLAST, V_TC};
        // link format 0 (the plain links) over every built launch shape, then
        // link format 1 (two-row links / 80 stored W) over the shapes that read
        // it, where the links allow it
        const int saved_fmt = h->link_fmt;
        bool have_alt = h->links_alt != nullptr;
        if (!have_alt && (h->op == OP_BRILLOUIN || h->prec != P_F64)) {
            have_alt = h->build_link_alt() == DIRAC_OK;
            if (!have_alt) h->release_link_alt();
            h->err.clear();
        }
        for (int fm = 0; fm < (have_alt ? 2 : 1) && st == DIRAC_OK; ++fm)
            for (int r : Rs) {
                if (r > h->Nv && r != Rs.front()) continue;
                for (int b : blocks)
                for (int pp : variants)
                for (int oi = 0; oi < 2; ++oi) {
                    if (!apply_config_supported(h->op, h->prec, r, b, pp, h->g)) continue;
                    if (fm == 1 && !link_format_supported(h->op, h->prec, pp)) continue;
                    if (fm == 0 && pp == V_TC) continue;   // reads link format 1 only
                    // site order: lexicographic, or t-chunks of 8 slices (variants 0 and 1)
                    const int tc = oi == 0 ? 0 : std::min(8, h->g.L[3]);
                    if (oi == 1 && pp != V_DIRECT && pp != V_GROUPS && pp != V_XLAST && pp != V_TC) continue;
                    LaunchCfg c{r, b, pp, tc, fm};
                    double med = 0.0;
                    if (!time_cfg(c, &med)) {
                        if (st) break;
                        continue;
                    }
                    if (med < best) {
                        best = med;
                        win = c;
                    }
                }
                if (st) break;
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st) {
            h->link_fmt = saved_fmt;
            return st;
        }
        h->cfg = LaunchCfg{win.R, win.block, win.variant, win.order};
        h->link_fmt = win.fmt == 1 ? 1 : 0;
        if (h->link_fmt == 0) h->release_link_alt();
        cache_store(key, win.R, win.block, win.variant, win.order, best, h->link_fmt);
    }
    dirac_status est = tune_even_odd(h, force);
    if (est) return est;
    if (R_out) *R_out = h->cfg.R;
    if (block_out) *block_out = h->cfg.block;
    if (variant_out) *variant_out = h->cfg.variant;
    if (ms_out) *ms_out = best;
    return DIRAC_OK;
}
