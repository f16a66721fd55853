// C ABI of the library (include/dirac.h): handle management, argument
// validation and the dispatch onto the kernels.
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/dirac.h"
#include "dirac_df.cuh"
#include "dirac_handle.h"

using namespace dirac;

static thread_local std::string g_create_error;

const char* dirac_version(void) { return "dirac_gb300 1.0 (sm_103a)"; }

const char* dirac_status_string(dirac_status st)
{
    switch (st) {
    case DIRAC_OK: return "ok";
    case DIRAC_ERR_INVALID_ARG: return "invalid argument";
    case DIRAC_ERR_UNSUPPORTED: return "unsupported";
    case DIRAC_ERR_OOM: return "out of device memory";
    case DIRAC_ERR_CUDA: return "CUDA error";
    case DIRAC_NOT_CONVERGED: return "not converged";
    case DIRAC_BREAKDOWN: return "breakdown";
    case DIRAC_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

dirac_status dirac_handle::fail(dirac_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return st;
}

dirac_status dirac_handle::cuda(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return DIRAC_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(DIRAC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(DIRAC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

dirac_status dirac_handle::alloc(void** p, size_t bytes, const char* what)
{
    *p = nullptr;
    if (bytes == 0) return DIRAC_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? DIRAC_ERR_OOM : DIRAC_ERR_CUDA,
                    "allocating %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
    }
    return DIRAC_OK;
}

void dirac_handle::release(void*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

size_t dirac_handle::field_bytes_internal(int nv) const
{
    return nblk_of((size_t)g.vol) * 32 * nv * nsc_of(op) * cbytes(prec);   // whole blocks of 32 sites
}

size_t dirac_handle::field_bytes_canonical(int nv) const
{
    return (size_t)g.vol * nv * nsc_of(op) * (prec == P_F64 ? 16 : 8);
}

double dirac_handle::diag_of(double mass) const
{
    if (op == OP_WILSON) return 1.0 / (2.0 * mass);          // 4 + m0, m0 = 1/(2 kappa) - 4
    if (op == OP_BRILLOUIN) return mass + 15.0 / 8.0;        // m0 - lambda_0 / 2
    return mass;                                             // staggered m
}

dirac_status dirac_handle::ensure_workspace()
{
    const size_t need = field_bytes_internal(Nv);
    if (ws_bytes >= need && ws_in && ws_out) return DIRAC_OK;
    release(ws_in);
    release(ws_out);
    ws_bytes = 0;
    dirac_status st = alloc(&ws_in, need, "apply workspace");
    if (st) return st;
    st = alloc(&ws_out, need, "apply workspace");
    if (st) return st;
    ws_bytes = need;
    return DIRAC_OK;
}

ApplyArgs dirac_handle::args(void* out, const void* in, int nv, double diag_value) const
{
    ApplyArgs a;
    a.g = g;
    a.Nv = nv;
    a.in = in;
    a.out = out;
    a.links = links;
    a.diag = diag_value;
    a.diag_v = nullptr;
    a.diagf = (float)diag_value;
    a.diag_vf = nullptr;
    a.err = dev_err;
    a.tc = 0;
    a.t0 = 0;
    a.nt = g.L[3];
    a.nsites = g.vol;
    return a;
}

dirac_status dirac_handle::run_apply(bool dagger, void* out, const void* in, int nv,
                                     double diag_value, const void* link_ptr, int p, LaunchCfg c,
                                     const double* diag_v, int t0, int nt, const float* diag_vf)
{
    // link format 1 (dirac_set_link_format) for the storage links, where the
    // launch variant reads it; every other call reads the plain links
    const int f = c.fmt < 0 ? link_fmt : c.fmt;
    if (f == 1 && link_ptr == links && p == prec && links_alt && link_format_supported(op, p, c.variant) &&
        (c.variant != V_TC || links_tc)) {
        link_ptr = c.variant == V_TC ? links_tc : links_alt;
        c.fmt = 1;
    } else {
        c.fmt = 0;
        // the tensor-core sweep reads only link format 1: without it, the CUDA-core sweep
        if (c.variant == V_TC) c = LaunchCfg{2, 128, V_DIRECT, c.order, 0};
    }
    ApplyArgs a = args(out, in, nv, diag_value);
    a.links = link_ptr;
    a.diag_v = diag_v;
    a.diag_vf = diag_vf;
    a.err = dev_err;
    if (nt > 0) {   // the slab of nt t-slices from t0 (variants 0, 1, 2 and 5)
        a.t0 = t0;
        a.nt = nt;
        a.nsites = (long)nt * g.stride[3];
    }
    a.tc = (c.variant == V_DIRECT || c.variant == V_GROUPS || c.variant == V_XLAST || c.variant == V_TC) ? c.order : 0;
    if (a.tc > 0) {
        a.fdc = make_fdiv((uint32_t)(g.L[2] * a.tc));
        a.fdt = make_fdiv((uint32_t)a.tc);
    }
    return cuda(launch_apply(op, p, dagger, a, c, stream), "apply kernel launch");
}

static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool dirac_check_device_ptr(const void* p) { return is_device_ptr(p) && ((uintptr_t)p % 16) == 0; }

// ------------------------------------------------------------------ lifecycle
dirac_status dirac_create(dirac_handle** h, dirac_op op, int Nc, int Nx, int Ny, int Nz, int Nt,
                          int Nv, double mass, dirac_prec prec, void* stream)
{
    if (!h) {
        g_create_error = "dirac_create: NULL handle pointer";
        return DIRAC_ERR_INVALID_ARG;
    }
    *h = nullptr;
    if (op < DIRAC_STAGGERED || op > DIRAC_BRILLOUIN) {
        g_create_error = "dirac_create: unknown operator";
        return DIRAC_ERR_INVALID_ARG;
    }
    if (prec < DIRAC_F64 || prec > DIRAC_F16) {
        g_create_error = "dirac_create: unknown precision";
        return DIRAC_ERR_INVALID_ARG;
    }
    if (Nc != 3) {
        g_create_error = "dirac_create: only Nc = 3 is built";
        return DIRAC_ERR_UNSUPPORTED;
    }
    if (Nx < 2 || Ny < 2 || Nz < 2 || Nt < 2) {
        g_create_error = "dirac_create: every lattice extent must be >= 2";
        return DIRAC_ERR_INVALID_ARG;
    }
    if (Nv < 1) {
        g_create_error = "dirac_create: Nv must be >= 1";
        return DIRAC_ERR_INVALID_ARG;
    }
    if (op == DIRAC_WILSON && !(mass > 0.0)) {
        g_create_error = "dirac_create: Wilson takes the hopping parameter kappa > 0";
        return DIRAC_ERR_INVALID_ARG;
    }
    const long vol = (long)Nx * Ny * Nz * Nt;
    if (vol > (1L << 31) / 2 || (double)vol * Nv * 12 * 16 > 2.0e11) {
        g_create_error = "dirac_create: lattice x Nv too large for one GPU";
        return DIRAC_ERR_INVALID_ARG;
    }
    dirac_handle* H = new (std::nothrow) dirac_handle();
    if (!H) {
        g_create_error = "dirac_create: host allocation failed";
        return DIRAC_ERR_OOM;
    }
    H->op = (int)op;
    H->Nc = Nc;
    H->Nv = Nv;
    H->prec = (int)prec;
    H->outer_df = prec == DIRAC_F64 ? 0 : 1;   // FP64 handles keep an FP64 outer residual
    H->g = make_geom(Nx, Ny, Nz, Nt);
    H->mass = mass;
    H->diag = H->diag_of(mass);
    H->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&H->device) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "dirac_create: no CUDA device";
        delete H;
        return DIRAC_ERR_CUDA;
    }
    H->cfg = default_config(H->op, H->prec, Nv);
    if (cudaMalloc((void**)&H->dev_err, sizeof(int)) != cudaSuccess || cudaMemset(H->dev_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "dirac_create: cannot allocate the device error word";
        delete H;
        return DIRAC_ERR_OOM;
    }
    if (H->op == OP_BRILLOUIN) {
        cudaError_t e = upload_brillouin_table(H->stream);
        if (e == cudaSuccess && (prec == DIRAC_BF16 || prec == DIRAC_F16)) e = brillouin_tc_prepare(H->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g_create_error = std::string("dirac_create: direction table upload: ") + cudaGetErrorString(e);
            delete H;
            return DIRAC_ERR_CUDA;
        }
    }
    *h = H;
    return DIRAC_OK;
}

dirac_handle::~dirac_handle()
{
    void* e = dev_err;
    release(e);
    release(links);
    release(links64);
    release(W64);
    release(links64b);
    release(links_df);
    release(links32);
    release(links_alt);
    release(links_tc);
    release(ws_in);
    release(ws_out);
    free_solver_workspace();
    free_host_apply();
}

dirac_status dirac_destroy(dirac_handle* h)
{
    if (!h) return DIRAC_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    const int dev = h->device;
    if (cur != dev) cudaSetDevice(dev);
    delete h;
    if (cur != dev) cudaSetDevice(cur);
    return DIRAC_OK;
}

dirac_status dirac_set_mass(dirac_handle* h, double mass)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (h->op == OP_WILSON && !(mass > 0.0))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_mass: Wilson takes kappa > 0");
    h->mass = mass;
    h->diag = h->diag_of(mass);
    return DIRAC_OK;
}

dirac_status dirac_set_stream(dirac_handle* h, void* stream)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    return DIRAC_OK;
}

// ------------------------------------------------------------------ links
dirac_status dirac_set_links(dirac_handle* h, const void* V, dirac_prec V_prec, int on_device)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!V) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_links: NULL links");
    if (V_prec != DIRAC_F64 && V_prec != DIRAC_F32)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_links: links must be complex double or float");
    if (on_device && !is_device_ptr(V))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_links: on_device = 1 but V is not a device pointer");
    if ((uintptr_t)V % 16)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_links: V must be 16-byte aligned");
    const bool f64 = V_prec == DIRAC_F64;
    const size_t canon_bytes = (size_t)h->g.vol * 4 * 9 * (f64 ? 16 : 8);
    dirac_status st;
    void* dV = nullptr;
    const void* src = V;
    if (!on_device) {
        if ((st = h->alloc(&dV, canon_bytes, "staging links"))) return st;
        if ((st = h->cuda(cudaMemcpyAsync(dV, V, canon_bytes, cudaMemcpyHostToDevice, h->stream),
                          "copying links to the device"))) {
            h->release(dV);
            return st;
        }
        src = dV;
    }
    if (!h->links64 && (st = h->alloc(&h->links64, (size_t)h->g.vol * 4 * 9 * 16, "FP64 links"))) {
        h->release(dV);
        return st;
    }
    st = h->cuda(launch_links_to_f64(h->g, src, f64, h->links64, h->stream), "links conversion");
    h->release_after_sync(dV);
    if (st) return st;
    h->release(h->W64);
    h->release(h->links64b);
    h->release(h->links_df);
    const int nmat = (h->op == OP_BRILLOUIN) ? 40 : 4;
    if (!h->links && (st = h->alloc(&h->links, nblk_of((size_t)h->g.vol) * 32 * 9 * nmat * cbytes(h->prec), "links")))
        return st;
    if (h->op == OP_BRILLOUIN) {
        if ((st = h->build_W64())) return st;
        st = h->cuda(launch_convert_links(h->prec, h->g, 40, h->W64, h->links, h->stream), "W conversion");
        if (st) return st;
        // the FP32 copy of the split inner solve is refreshed in place (a
        // captured solver graph holds its address)
        if (h->links32 && h->links32 != h->links && (st = h->refresh_links32())) return st;
        if (h->prec != P_F64) h->release_after_sync(h->W64);   // rebuilt on demand by the solver
    } else {
        st = h->cuda(launch_convert_links(h->prec, h->g, 4, h->links64, h->links, h->stream), "links conversion");
        if (st) return st;
        // the FP32 copy of the split inner solve is refreshed in place, like the
        // storage links: a captured solver graph holds both addresses
        if (h->links32 && h->links32 != h->links) {
            st = h->cuda(launch_convert_links(P_F32, h->g, 4, h->links64, h->links32, h->stream), "FP32 links");
            if (st) return st;
        }
    }
    if (h->link_fmt == 1) {
        // rebuilt in place (same address); links that do not allow format 1
        // (two-row links of links that are not special unitary) fall back to
        // format 0, which gives the same operator
        if (h->build_link_alt() != DIRAC_OK) {
            h->release_link_alt();
            h->link_fmt = 0;
        }
    }
    st = h->cuda(cudaStreamSynchronize(h->stream), "dirac_set_links");
    if (st) return st;
    h->have_links = true;
    return DIRAC_OK;
}

// format 1 of the storage links (links_alt) from the current links: Brillouin,
// all 80 directions per site; Wilson and staggered, the first two rows of each
// link, after checking in FP64 that the links are special unitary to the
// precision of the storage (the third row is rebuilt from the first two)
dirac_status dirac_handle::build_link_alt()
{
    dirac_status st;
    const size_t nsite = nblk_of((size_t)g.vol) * 32;
    if (op == OP_BRILLOUIN) {
        if (!links_alt && (st = alloc(&links_alt, nsite * 80 * 9 * cbytes(prec), "80-direction W"))) return st;
        if ((st = cuda(launch_brillouin_w80(prec, g, links, links_alt, stream), "80-direction W"))) return st;
        if (prec != P_BF16 && prec != P_F16) return DIRAC_OK;
        // the copy the tensor-core sweep reads: the 80 W of a site in one piece
        if (!links_tc && (st = alloc(&links_tc, nsite * 80 * 9 * cbytes(prec), "80-direction W, site-major"))) return st;
        return cuda(launch_brillouin_tc_links(g, links_alt, links_tc, stream), "80-direction W, site-major");
    }
    if (prec == P_F64)
        return fail(DIRAC_ERR_UNSUPPORTED, "dirac_set_link_format: two-row links are built for FP32 and 16-bit storage");
    void* d = nullptr;
    if ((st = alloc(&d, sizeof(double), "SU(3) check"))) return st;
    double dev = 0.0;
    st = cuda(launch_su3_deviation(g, links64, static_cast<double*>(d), stream), "SU(3) check");
    if (!st) st = cuda(cudaMemcpyAsync(&dev, d, sizeof(double), cudaMemcpyDeviceToHost, stream), "SU(3) check");
    if (!st) st = cuda(cudaStreamSynchronize(stream), "SU(3) check");
    release(d);
    if (st) return st;
    const double tol = prec == P_F32 ? 1e-6 : 1e-2;
    if (!(dev <= tol))
        return fail(DIRAC_ERR_INVALID_ARG,
                    "dirac_set_link_format: two-row links need special unitary links; max |U_2c - conj(U_0 x U_1)_c| "
                    "= %.3g > %.0e",
                    dev, tol);
    if (!links_alt && (st = alloc(&links_alt, nsite * 4 * 6 * cbytes(prec), "two-row links"))) return st;
    return cuda(launch_links_2row(prec, g, links, links_alt, stream), "two-row links");
}

// the operator's links in FP64 and in the sweeps' blocked layout (the FP64 copies
// links64 / W64 are [m][9][site], the layout the W build and the force read)
dirac_status dirac_handle::ensure_links64b(const void** out)
{
    if (prec == P_F64) {
        *out = links;
        return DIRAC_OK;
    }
    if (!links64b) {
        dirac_status st;
        const int nmat = (op == OP_BRILLOUIN) ? 40 : 4;
        if (op == OP_BRILLOUIN && (st = build_W64())) return st;
        if ((st = alloc(&links64b, nblk_of((size_t)g.vol) * 32 * 9 * nmat * 16, "FP64 links (blocked)"))) return st;
        if ((st = cuda(launch_convert_links(P_F64, g, nmat, op == OP_BRILLOUIN ? W64 : links64, links64b, stream),
                       "FP64 links (blocked)"))) {
            release(links64b);
            return st;
        }
    }
    *out = links64b;
    return DIRAC_OK;
}

dirac_status dirac_handle::ensure_links_df(const void** out)
{
    if (!links_df) {
        const void* L64 = nullptr;
        dirac_status st;
        if ((st = ensure_links64b(&L64))) return st;
        const int nmat = (op == OP_BRILLOUIN) ? 40 : 4;
        const size_t n16 = nblk_of((size_t)g.vol) * 32 * 9 * nmat;
        if ((st = alloc(&links_df, n16 * 16, "double-float links"))) return st;
        if ((st = cuda(df_from_f64(n16, L64, links_df, stream), "double-float links"))) {
            release(links_df);
            return st;
        }
    }
    *out = links_df;
    return DIRAC_OK;
}

dirac_status dirac_handle::ensure_links32(const void** out)
{
    if (prec == P_F32) {
        *out = links;
        return DIRAC_OK;
    }
    if (!links32) {
        // Brillouin: all 80 W per site in FP32 (link format 1), from the FP64 W,
        // which the solver builds first
        const void* src = op == OP_BRILLOUIN ? W64 : links64;
        if (!src) return fail(DIRAC_ERR_INVALID_ARG, "FP32 link copy: no FP64 links");
        dirac_status st;
        const size_t nmat = op == OP_BRILLOUIN ? 80 : 4;
        if ((st = alloc(&links32, nblk_of((size_t)g.vol) * 32 * 9 * nmat * 8, "FP32 links (blocked)"))) return st;
        if ((st = refresh_links32())) {
            release(links32);
            return st;
        }
    }
    *out = links32;
    return DIRAC_OK;
}

// the FP32 link copy of the split inner solve from the FP64 links (Brillouin:
// W64 into planes 0..39, then planes 40..79 = W_{-d}(x) in place)
dirac_status dirac_handle::refresh_links32()
{
    if (op != OP_BRILLOUIN)
        return cuda(launch_convert_links(P_F32, g, 4, links64, links32, stream), "FP32 links (blocked)");
    dirac_status st;
    if ((st = cuda(launch_convert_links(P_F32, g, 40, W64, links32, stream), "FP32 W (blocked)"))) return st;
    return cuda(launch_brillouin_w80(P_F32, g, links32, links32, stream), "FP32 W, 80 directions");
}

dirac_status dirac_handle::build_W64()
{
    if (W64) return DIRAC_OK;
    dirac_status st;
    void* tmp = nullptr;
    if ((st = alloc(&tmp, (size_t)g.vol * 81 * 9 * 16, "W build scratch"))) return st;
    if ((st = alloc(&W64, (size_t)g.vol * 40 * 9 * 16, "FP64 W"))) {
        release(tmp);
        return st;
    }
    st = cuda(launch_build_W(g, links64, tmp, W64, stream), "W build");
    release_after_sync(tmp);
    return st;
}

void dirac_handle::release_after_sync(void*& p)
{
    if (!p) return;
    cudaStreamSynchronize(stream);
    release(p);
}

void dirac_handle::release_link_alt()
{
    release_after_sync(links_alt);
    release_after_sync(links_tc);
}

// ------------------------------------------------------------------ fields
dirac_status dirac_field_bytes(const dirac_handle* h, dirac_layout layout, size_t* bytes)
{
    if (!h || !bytes) return DIRAC_ERR_INVALID_ARG;
    *bytes = layout == DIRAC_INTERNAL ? h->field_bytes_internal(h->Nv) : h->field_bytes_canonical(h->Nv);
    return DIRAC_OK;
}

dirac_status dirac_pack(dirac_handle* h, void* internal_out, const void* canonical_in)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!internal_out || !canonical_in || internal_out == canonical_in)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_pack: NULL or aliased pointers");
    if (!dirac_check_device_ptr(internal_out) || !dirac_check_device_ptr(canonical_in))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_pack: need 16-byte aligned device pointers");
    return h->cuda(launch_pack_spinor(h->prec, nsc_of(h->op), h->g, h->Nv, canonical_in,
                                      h->prec == P_F64, internal_out, h->stream), "pack");
}

dirac_status dirac_unpack(dirac_handle* h, void* canonical_out, const void* internal_in)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!canonical_out || !internal_in || canonical_out == internal_in)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_unpack: NULL or aliased pointers");
    if (!dirac_check_device_ptr(canonical_out) || !dirac_check_device_ptr(internal_in))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_unpack: need 16-byte aligned device pointers");
    return h->cuda(launch_unpack_spinor(h->prec, nsc_of(h->op), h->g, h->Nv, internal_in,
                                        canonical_out, h->prec == P_F64, h->stream), "unpack");
}

// ------------------------------------------------------------------ apply
static dirac_status apply_common(dirac_handle* h, bool dagger, void* out, const void* in,
                                 dirac_layout layout, const char* name)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!out || !in) return h->fail(DIRAC_ERR_INVALID_ARG, "%s: NULL pointer", name);
    if (out == in) return h->fail(DIRAC_ERR_INVALID_ARG, "%s: out must not alias in", name);
    if (layout != DIRAC_CANONICAL && layout != DIRAC_INTERNAL)
        return h->fail(DIRAC_ERR_INVALID_ARG, "%s: unknown layout", name);
    if (!h->have_links) return h->fail(DIRAC_ERR_INVALID_ARG, "%s: call dirac_set_links first", name);
    if (!dirac_check_device_ptr(out) || !dirac_check_device_ptr(in))
        return h->fail(DIRAC_ERR_INVALID_ARG, "%s: in and out must be 16-byte aligned device pointers", name);
    dirac_status st;
    if (layout == DIRAC_INTERNAL)
        return h->run_apply(dagger, out, in, h->Nv, h->diag, h->links, h->prec, h->cfg);
    if ((st = h->ensure_workspace())) return st;
    if ((st = dirac_pack(h, h->ws_in, in))) return st;
    if ((st = h->run_apply(dagger, h->ws_out, h->ws_in, h->Nv, h->diag, h->links, h->prec, h->cfg)))
        return st;
    return dirac_unpack(h, out, h->ws_out);
}

dirac_status dirac_apply(dirac_handle* h, void* out, const void* in, dirac_layout layout)
{
    return apply_common(h, false, out, in, layout, "dirac_apply");
}

dirac_status dirac_apply_dagger(dirac_handle* h, void* out, const void* in, dirac_layout layout)
{
    return apply_common(h, true, out, in, layout, "dirac_apply_dagger");
}

// ------------------------------------------------------------------ config
dirac_status dirac_set_kernel_config(dirac_handle* h, int R, int block, int variant)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!apply_config_supported(h->op, h->prec, R, block, variant, h->g))
        return h->fail(DIRAC_ERR_UNSUPPORTED, "dirac_set_kernel_config: R = %d, block = %d, variant = %d not built",
                       R, block, variant);
    if (variant == V_TC && h->link_fmt != 1) {
        // the tensor-core sweep reads all 80 W per site (link format 1)
        const dirac_status st = dirac_set_link_format(h, 1);
        if (st) return st;
    }
    h->cfg = LaunchCfg{R, block, variant, h->cfg.order};
    return DIRAC_OK;
}

dirac_status dirac_set_link_format(dirac_handle* h, int fmt)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (fmt != 0 && fmt != 1)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_link_format: format %d is not 0 or 1", fmt);
    if (fmt == 0) {
        h->link_fmt = 0;
        h->release_link_alt();
        return DIRAC_OK;
    }
    if (h->op != OP_BRILLOUIN && h->prec == P_F64)
        return h->fail(DIRAC_ERR_UNSUPPORTED, "dirac_set_link_format: two-row links are built for FP32 and 16-bit storage");
    if (h->have_links) {
        dirac_status st = h->build_link_alt();
        if (!st) st = h->cuda(cudaStreamSynchronize(h->stream), "dirac_set_link_format");
        if (st) {
            h->release_link_alt();
            h->link_fmt = 0;
            return st;
        }
    }
    h->link_fmt = 1;
    return DIRAC_OK;
}

dirac_status dirac_get_link_format(const dirac_handle* h, int* fmt)
{
    if (!h || !fmt) return DIRAC_ERR_INVALID_ARG;
    *fmt = h->link_fmt;
    return DIRAC_OK;
}

dirac_status dirac_set_site_order(dirac_handle* h, int tchunk)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (tchunk < 0 || tchunk > h->g.L[3])
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_site_order: tchunk = %d not in 0..Nt = %d", tchunk,
                       h->g.L[3]);
    h->cfg.order = tchunk;
    return DIRAC_OK;
}

dirac_status dirac_get_site_order(const dirac_handle* h, int* tchunk)
{
    if (!h || !tchunk) return DIRAC_ERR_INVALID_ARG;
    *tchunk = h->cfg.order;
    return DIRAC_OK;
}

dirac_status dirac_set_preconditioner(dirac_handle* h, int mode)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (mode != 0 && mode != 1)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_preconditioner: mode %d is not 0 or 1", mode);
    h->precond = mode;
    return DIRAC_OK;
}

dirac_status dirac_set_residual_arithmetic(dirac_handle* h, int mode)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (mode != 0 && mode != 1)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_residual_arithmetic: mode %d is not 0 or 1", mode);
    h->outer_df = mode;
    return DIRAC_OK;
}

dirac_status dirac_get_residual_arithmetic(const dirac_handle* h, int* mode)
{
    if (!h || !mode) return DIRAC_ERR_INVALID_ARG;
    *mode = h->outer_df;
    return DIRAC_OK;
}

dirac_status dirac_set_inner_fields(dirac_handle* h, int mode)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (mode != 0 && mode != 1)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_set_inner_fields: mode %d is not 0 or 1", mode);
    h->inner_fields = mode;
    return DIRAC_OK;
}

dirac_status dirac_get_inner_fields(const dirac_handle* h, int* mode)
{
    if (!h || !mode) return DIRAC_ERR_INVALID_ARG;
    *mode = h->inner_fields;
    return DIRAC_OK;
}

dirac_status dirac_get_preconditioner(const dirac_handle* h, int* mode)
{
    if (!h || !mode) return DIRAC_ERR_INVALID_ARG;
    *mode = h->precond;
    return DIRAC_OK;
}

dirac_status dirac_get_kernel_config(const dirac_handle* h, int* R, int* block, int* variant)
{
    if (!h || !R || !block || !variant) return DIRAC_ERR_INVALID_ARG;
    *R = h->cfg.R;
    *block = h->cfg.block;
    *variant = h->cfg.variant;
    return DIRAC_OK;
}

dirac_status dirac_sync(dirac_handle* h)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    dirac_status st = h->cuda(cudaStreamSynchronize(h->stream), "dirac_sync");
    if (st) return st;
    int e = 0;
    if ((st = h->cuda(cudaMemcpy(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "dirac_sync"))) return st;
    if (e) {
        cudaMemset(h->dev_err, 0, sizeof(int));
        return h->fail(DIRAC_TIMEOUT, "dirac_sync: a kernel's bounded wait ran out (status %d)", e);
    }
    return DIRAC_OK;
}

const char* dirac_last_error(const dirac_handle* h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

// ------------------------------------------------------------------ dispatch
namespace dirac {

bool apply_config_supported(int op, int prec, int R, int block, int variant, const Geom& g)
{
    if (block < 32 || block > 256 || block % 32) return false;
    if (variant == V_XROW)
        return op == OP_WILSON && prec != P_F64 && R >= 1 && R <= 2 && block <= 192 && 32 % g.L[0] == 0 &&
               g.stride[3] % 32 == 0;
    if (variant == V_TC) return op == OP_BRILLOUIN && (prec == P_BF16 || prec == P_F16) && R == 1 && block == 128;
    if (variant == V_XLAST)
        return prec != P_F64 && block <= 64 && 32 % g.L[0] == 0 && g.stride[3] % 32 == 0 &&
               ((op == OP_WILSON && R >= 1 && R <= 2) || (op == OP_STAGGERED && (R == 1 || R == 2 || R == 4 || R == 6)));
    const bool Rok = (op == OP_STAGGERED) ? (R == 1 || R == 2 || R == 4 || R == 6) : (R >= 1 && R <= 4);
    if (!Rok) return false;
    if (variant == V_DIRECT) return true;
    if (op == OP_WILSON && prec == P_F64) return false;   // FP64 Wilson: direct variant only
    if (variant == V_GROUPS) return block <= 64;
    if (variant == V_TMARCH) return op == OP_WILSON && R <= 2 && block <= 128;
    return op == OP_WILSON && variant == V_PIPE3 && wilson_pipe_smem(prec, R, block, 3) <= 227 * 1024;
}

LaunchCfg default_config(int op, int prec, int Nv)
{
    // the largest right-hand-side group that divides Nv and fits the
    // registers without spilling (FP64 sweeps use at most 2 / 4)
    if (op == OP_STAGGERED) {
        int R = (Nv % 6 == 0) ? 6 : (Nv % 4 == 0 ? 4 : (Nv % 2 == 0 ? 2 : 1));
        if (prec == P_F64 && R > 4) R = 4;
        return LaunchCfg{R, 128, V_DIRECT};
    }
    if (prec == P_F64) return LaunchCfg{(Nv % 2 == 0) ? 2 : 1, 128, V_DIRECT};
    int R = (Nv % 2 == 0) ? 2 : 1;
    return LaunchCfg{R, 128, V_DIRECT};
}

cudaError_t launch_apply(int op, int prec, bool dagger, const ApplyArgs& a, LaunchCfg cfg, cudaStream_t st)
{
    if (a.g.vol == 0 || a.Nv == 0) return cudaSuccess;
    switch (op) {
    case OP_STAGGERED: return launch_apply_staggered(prec, dagger, a, cfg, st);
    case OP_WILSON: return launch_apply_wilson(prec, dagger, a, cfg, st);
    case OP_BRILLOUIN: return launch_apply_brillouin(prec, dagger, a, cfg, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dirac
