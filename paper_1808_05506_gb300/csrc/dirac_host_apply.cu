// dirac_apply_host: out = D in with both fields in host memory, the copies
// overlapped with the sweep (no counterpart in the paper, whose fields live
// in the memory of the node that sweeps them).
//
// The lattice is cut into S slabs of consecutive t-slices.  Three streams:
//   copy-in   H2D of slab k into one of two canonical staging buffers;
//   compute   (the handle's stream) pack slab k into the internal field, then
//             sweep every slice whose t-neighbours are packed by now (up to
//             the second-to-last slice of slab k; slice 0 needs slice Nt - 1
//             and is swept last) and unpack them into an output staging
//             buffer;
//   copy-out  D2H of each finished range of slices.
// Events order the buffer reuse (two input and two output staging buffers),
// so the H2D of slab k + 1, the sweep of the slices of slab k and the D2H of
// the previous range run at the same time; only one slice's sweep and copy
// remain after the last slab has arrived.  The sweep of a range computes
// exactly what the whole-lattice sweep computes at those sites.
#include <cstdint>
#include <cstring>

#include "dirac_handle.h"

using namespace dirac;

namespace {

struct HostApply {
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t in_full[2] = {}, in_free[2] = {}, out_full[2] = {}, out_free[2] = {};
    cudaEvent_t start = nullptr, done = nullptr;
    void* stage_in[2] = {};
    void* stage_out[2] = {};
    size_t stage_bytes = 0;
    int device = 0;
};

// slab thickness: about 16 slabs
int slab_slices(int Lt) { return Lt >= 16 ? (Lt + 15) / 16 : 1; }

bool is_host_ptr(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;   // memory CUDA does not know: plain (pageable) host memory
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}   // namespace

void dirac_handle::free_host_apply()
{
    if (!hx) return;
    HostApply* x = static_cast<HostApply*>(hx);
    if (x->cin) cudaStreamSynchronize(x->cin);
    if (x->cout) cudaStreamSynchronize(x->cout);
    for (int b = 0; b < 2; ++b) {
        release(x->stage_in[b]);
        release(x->stage_out[b]);
        if (x->in_full[b]) cudaEventDestroy(x->in_full[b]);
        if (x->in_free[b]) cudaEventDestroy(x->in_free[b]);
        if (x->out_full[b]) cudaEventDestroy(x->out_full[b]);
        if (x->out_free[b]) cudaEventDestroy(x->out_free[b]);
    }
    if (x->start) cudaEventDestroy(x->start);
    if (x->done) cudaEventDestroy(x->done);
    if (x->cin) cudaStreamDestroy(x->cin);
    if (x->cout) cudaStreamDestroy(x->cout);
    delete x;
    hx = nullptr;
}

static dirac_status ensure_host_apply(dirac_handle* h, size_t stage_bytes)
{
    HostApply* x = static_cast<HostApply*>(h->hx);
    if (x && x->stage_bytes >= stage_bytes) return DIRAC_OK;
    h->free_host_apply();
    x = new HostApply();
    h->hx = x;
    dirac_status st;
    const unsigned fl = cudaEventDisableTiming;
    if ((st = h->cuda(cudaStreamCreateWithFlags(&x->cin, cudaStreamNonBlocking), "dirac_apply_host: streams")) ||
        (st = h->cuda(cudaStreamCreateWithFlags(&x->cout, cudaStreamNonBlocking), "dirac_apply_host: streams")) ||
        (st = h->cuda(cudaEventCreateWithFlags(&x->start, fl), "dirac_apply_host: events")) ||
        (st = h->cuda(cudaEventCreateWithFlags(&x->done, fl), "dirac_apply_host: events"))) {
        h->free_host_apply();
        return st;
    }
    for (int b = 0; b < 2; ++b) {
        if ((st = h->cuda(cudaEventCreateWithFlags(&x->in_full[b], fl), "dirac_apply_host: events")) ||
            (st = h->cuda(cudaEventCreateWithFlags(&x->in_free[b], fl), "dirac_apply_host: events")) ||
            (st = h->cuda(cudaEventCreateWithFlags(&x->out_full[b], fl), "dirac_apply_host: events")) ||
            (st = h->cuda(cudaEventCreateWithFlags(&x->out_free[b], fl), "dirac_apply_host: events")) ||
            (st = h->alloc(&x->stage_in[b], stage_bytes, "dirac_apply_host staging")) ||
            (st = h->alloc(&x->stage_out[b], stage_bytes, "dirac_apply_host staging"))) {
            h->free_host_apply();
            return st;
        }
    }
    x->stage_bytes = stage_bytes;
    return DIRAC_OK;
}

#define HCK(call, what)                                    \
    do {                                                   \
        dirac_status s_ = h->cuda((call), what);           \
        if (s_ != DIRAC_OK) return s_;                     \
    } while (0)

extern "C" DIRAC_API dirac_status dirac_apply_host(dirac_handle* h, void* out, const void* in, int dagger)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!h->have_links) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_host: call dirac_set_links first");
    if (!out || !in) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_host: NULL field");
    if (!is_host_ptr(out) || !is_host_ptr(in))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_host: in and out must be host memory");
    const size_t field = h->field_bytes_canonical(h->Nv);
    const char* ib = static_cast<const char*>(in);
    char* ob = static_cast<char*>(out);
    if (ob < ib + field && ib < ob + field)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_host: out overlaps in");
    dirac_status st;
    if ((st = h->ensure_workspace())) return st;

    const int Lt = h->g.L[3];
    const int ts = slab_slices(Lt);
    const int S = (Lt + ts - 1) / ts;
    const long vol3 = h->g.stride[3];
    const size_t site_bytes = field / (size_t)h->g.vol;   // canonical bytes per site (all Nv)
    // a staging buffer holds one slab in and up to ts + 1 finished slices out
    if ((st = ensure_host_apply(h, (size_t)(ts + 1) * vol3 * site_bytes))) return st;
    HostApply* x = static_cast<HostApply*>(h->hx);
    const bool f64 = h->prec == P_F64;
    const int nsc = nsc_of(h->op);
    // the slab sweeps need a launch shape that can cover a t-slab
    LaunchCfg c = h->cfg;
    if (c.variant != V_DIRECT && c.variant != V_GROUPS && c.variant != V_TMARCH && c.variant != V_XROW &&
        c.variant != V_XLAST && c.variant != V_TC)
        c = LaunchCfg{c.R, 64, V_GROUPS, c.order};
    if (!apply_config_supported(h->op, h->prec, c.R, c.block, c.variant, h->g)) c = default_config(h->op, h->prec, h->Nv);
    auto slab_t0 = [&](int k) { return k * ts; };
    auto slab_nt = [&](int k) { return (k + 1) * ts <= Lt ? ts : Lt - k * ts; };

    // everything of this call starts after the work already on the handle's stream
    HCK(cudaEventRecord(x->start, h->stream), "dirac_apply_host");
    HCK(cudaStreamWaitEvent(x->cin, x->start, 0), "dirac_apply_host");
    HCK(cudaStreamWaitEvent(x->cout, x->start, 0), "dirac_apply_host");
    bool out_used[2] = {false, false};
    int nout = 0;
    int done_to = 1;   // slices 1 .. done_to - 1 are swept
    // sweep, unpack and copy out the slices t0 .. t1 - 1
    auto emit = [&](int t0, int t1) -> dirac_status {
        if (t1 <= t0) return DIRAC_OK;
        const int bo = nout & 1;
        if (out_used[bo]) HCK(cudaStreamWaitEvent(h->stream, x->out_free[bo], 0), "dirac_apply_host");
        const int nt = t1 - t0;
        dirac_status s2 = h->run_apply(dagger != 0, h->ws_out, h->ws_in, h->Nv, h->diag, h->links, h->prec, c,
                                       nullptr, t0, nt);
        if (s2) return s2;
        HCK(launch_unpack_spinor(h->prec, nsc, h->g, h->Nv, h->ws_out, x->stage_out[bo], f64, h->stream,
                                 (long)t0 * vol3, (long)nt * vol3),
            "dirac_apply_host: unpack");
        HCK(cudaEventRecord(x->out_full[bo], h->stream), "dirac_apply_host");
        HCK(cudaStreamWaitEvent(x->cout, x->out_full[bo], 0), "dirac_apply_host");
        HCK(cudaMemcpyAsync(ob + (size_t)t0 * vol3 * site_bytes, x->stage_out[bo], (size_t)nt * vol3 * site_bytes,
                            cudaMemcpyDeviceToHost, x->cout),
            "dirac_apply_host: device to host");
        HCK(cudaEventRecord(x->out_free[bo], x->cout), "dirac_apply_host");
        out_used[bo] = true;
        ++nout;
        return DIRAC_OK;
    };
    for (int k = 0; k < S; ++k) {
        const int b = k & 1;
        if (k >= 2) HCK(cudaStreamWaitEvent(x->cin, x->in_free[b], 0), "dirac_apply_host");
        const int t0 = slab_t0(k), nt = slab_nt(k);
        HCK(cudaMemcpyAsync(x->stage_in[b], ib + (size_t)t0 * vol3 * site_bytes, (size_t)nt * vol3 * site_bytes,
                            cudaMemcpyHostToDevice, x->cin),
            "dirac_apply_host: host to device");
        HCK(cudaEventRecord(x->in_full[b], x->cin), "dirac_apply_host");
        HCK(cudaStreamWaitEvent(h->stream, x->in_full[b], 0), "dirac_apply_host");
        HCK(launch_pack_spinor(h->prec, nsc, h->g, h->Nv, x->stage_in[b], f64, h->ws_in, h->stream,
                               (long)t0 * vol3, (long)nt * vol3),
            "dirac_apply_host: pack");
        HCK(cudaEventRecord(x->in_free[b], h->stream), "dirac_apply_host");
        // slices up to the second-to-last one of slab k have their t-neighbours
        // (all of them once the last slab is in); slice 0 waits for slice Nt - 1
        const int hi = (k == S - 1) ? Lt : t0 + nt - 1;
        if ((st = emit(done_to, hi))) return st;
        if (hi > done_to) done_to = hi;
    }
    if ((st = emit(0, 1))) return st;
    // the handle's stream completes when the last copy to the host has landed
    HCK(cudaEventRecord(x->done, x->cout), "dirac_apply_host");
    HCK(cudaStreamWaitEvent(h->stream, x->done, 0), "dirac_apply_host");
    return DIRAC_OK;
}
