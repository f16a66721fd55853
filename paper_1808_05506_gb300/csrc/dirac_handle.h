// The opaque handle behind dirac_handle* (include/dirac.h).
#pragma once

#include <string>

#include "../../include/dirac.h"
#include "dirac_internal.h"

namespace dirac {
LaunchCfg default_config(int op, int prec, int Nv);
}

struct dirac_handle {
    int op = 0, Nc = 3, Nv = 1, prec = 1;
    dirac::Geom g{};
    double mass = 0.0;        // as given: staggered m, Wilson kappa, Brillouin m0
    double diag = 0.0;        // the site-diagonal coefficient of the sweep
    cudaStream_t stream = nullptr;
    int device = 0;
    dirac::LaunchCfg cfg{1, 128, dirac::V_DIRECT};
    int precond = 1;          // inner solves: 1 even-odd where it applies, 0 whole lattice
    int outer_df = 1;         // outer residual: 1 double-float sweep (non-FP64 handles), 0 FP64
    int inner_fields = 1;     // 16-bit Wilson even-odd inner solves: 1 split fields, 0 all 16-bit
    dirac::LaunchCfg eo_cfg{0, 0, 0, 0};   // launch shape of the even-odd sweeps (R = 0: not tuned)

    void* links = nullptr;    // storage-precision links [m][9][site] (m = mu, or 40 stored W)
    void* links64 = nullptr;  // FP64 V_mu [4][9][site]
    void* W64 = nullptr;      // FP64 W [40][9][site] (Brillouin; kept for F64 handles, lazy otherwise)
    void* links_df = nullptr; // the same in double-float storage (dirac_df.cuh), for the residual (lazy)
    void* links32 = nullptr;  // FP32 links of the split inner solve, blocked layout (lazy):
                              // V_mu, or all 80 Brillouin W per site
    void* links64b = nullptr; // FP64 links of the operator (V or W) in the blocked layout of the
                              // sweeps, for the solver's FP64 residual (lazy; F64 handles use links)
    void* links_alt = nullptr;  // link format 1 (dirac_set_link_format): Wilson / staggered two-row
                                // links [4][6][site], Brillouin all 80 W [80][9][site] (blocked)
    void* links_tc = nullptr;   // with link format 1 for 16-bit Brillouin: the 80 W of each site
                                // contiguous [site][80][9], directions in the order of the
                                // tensor-core sweep (which reads this copy)
    int link_fmt = 0;           // the format the apply sweeps read where their variant supports it
    bool have_links = false;
    int* dev_err = nullptr;   // device error word written by kernels whose bounded waits run out

    void* ws_in = nullptr;    // internal-layout workspaces of the canonical apply
    void* ws_out = nullptr;
    size_t ws_bytes = 0;

    // solver workspace (dirac_solve.cu)
    void* sw = nullptr;
    size_t sw_bytes = 0;
    int sw_nv = 0;

    // streams, events and staging buffers of dirac_apply_host (dirac_host_apply.cu)
    void* hx = nullptr;

    std::string err;

    ~dirac_handle();
    dirac_status fail(dirac_status st, const char* fmt, ...);
    dirac_status cuda(cudaError_t e, const char* what);
    dirac_status alloc(void** p, size_t bytes, const char* what);
    void release(void*& p);
    void release_after_sync(void*& p);
    void release_link_alt();   // both copies of link format 1 (links_alt, links_tc)
    size_t field_bytes_internal(int nv) const;
    size_t field_bytes_canonical(int nv) const;
    double diag_of(double mass) const;
    dirac_status ensure_workspace();
    dirac_status build_W64();
    dirac_status ensure_links64b(const void** out);
    dirac_status ensure_links_df(const void** out);
    dirac_status ensure_links32(const void** out);
    dirac_status refresh_links32();
    dirac_status build_link_alt();
    dirac::ApplyArgs args(void* out, const void* in, int nv, double diag_value) const;
    dirac_status run_apply(bool dagger, void* out, const void* in, int nv, double diag_value,
                           const void* link_ptr, int p, dirac::LaunchCfg c, const double* diag_v = nullptr,
                           int t0 = 0, int nt = 0, const float* diag_vf = nullptr);
    void free_solver_workspace();
    void free_host_apply();
};

bool dirac_check_device_ptr(const void* p);
