// dirac_apply_static: out = D in (or D^+ in) on canonical fields, like
// dirac_apply with DIRAC_CANONICAL, but without any device allocation.
//
// The canonical apply converts its input into the internal layout and back
// through two internal-layout work fields.  dirac_apply keeps them in memory
// the handle allocates on first use; this entry point keeps them instead in
// one fixed array in the library's own device memory, reserved when the
// library's device code is loaded on a GPU and kept until the process exits.
// It serves callers that must not allocate while they work: latency-critical
// loops that cannot afford cudaMalloc / cudaFree (which can synchronise the
// device), and hosts whose device memory is entirely reserved up front by
// their own allocator, so that a library allocation would fail or evict.
#include <cuda.h>
#include <mutex>

#include "dirac_handle.h"

using namespace dirac;

namespace {

// 64 MiB: room for two work fields of up to 32 MiB each.  An FP32 Wilson or
// Brillouin field takes 96 bytes per site and right-hand side (48 for BF16 /
// FP16, 192 for FP64; staggered a quarter of that), so FP32 Wilson fits
// while 2 x 96 B x Nv x sites <= 64 MiB: 16^4 with Nv <= 5, 8^4 with Nv <= 85.
constexpr size_t kScratchBytes = size_t(64) << 20;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;

// The device address of g_scratch, per device, with the unique id of the
// CUDA context it was looked up in.  In host code the name g_scratch is only a
// host-side stand-in, so the address is looked up with the device current.
// The device image (and the array with it) is loaded anew when a context is
// destroyed and recreated (cudaDeviceReset, or the primary context released
// and retained again), so the cached address is only reused while the
// current context is the one it was looked up in.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    void* p = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

using PFN_CtxGetCurrent = CUresult (*)(CUcontext*);
using PFN_CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// unique id of the current context (driver entry points resolved once through
// the runtime, so the library needs no link-time dependency on libcuda);
// false when the driver does not offer it
bool current_context_id(unsigned long long* id)
{
    static PFN_CtxGetCurrent get_current = nullptr;
    static PFN_CtxGetId get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<PFN_CtxGetCurrent>(f1);
            get_id = reinterpret_cast<PFN_CtxGetId>(f2);
        }
        cudaGetLastError();
        resolved = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

dirac_status scratch_address(dirac_handle* h, int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return h->fail(DIRAC_ERR_UNSUPPORTED, "dirac_apply_static: device %d beyond the %d supported", dev,
                       kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    ScratchAddr& c = g_scratch_addr[dev];
    // without a context id the address is looked up on every call
    if (!c.p || !have_id || c.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            c = ScratchAddr{};
            return h->fail(DIRAC_ERR_CUDA, "dirac_apply_static: cannot resolve the static scratch area: %s",
                           cudaGetErrorString(e));
        }
        c.p = p;
        c.ctx_id = have_id ? id : 0;
    }
    *out = c.p;
    return DIRAC_OK;
}

}  // namespace

extern "C" DIRAC_API dirac_status dirac_apply_static(dirac_handle* h, void* out, const void* in, int dagger)
{
    if (!h) return DIRAC_ERR_INVALID_ARG;
    if (!out || !in) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_static: NULL pointer");
    if (out == in) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_static: out must not alias in");
    if (!h->have_links) return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_static: call dirac_set_links first");
    const size_t field = h->field_bytes_internal(h->Nv);
    const size_t field_padded = (field + 255) / 256 * 256;
    if (2 * field_padded > kScratchBytes)
        return h->fail(DIRAC_ERR_INVALID_ARG,
                       "dirac_apply_static: needs %zu bytes of scratch (two internal fields of %zu bytes); "
                       "the static area holds %zu bytes: use dirac_apply",
                       2 * field_padded, field, kScratchBytes);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return h->fail(DIRAC_ERR_CUDA, "dirac_apply_static: no current device");
    }
    if (cur != h->device)
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_static: make the handle's device %d current (it is %d)",
                       h->device, cur);
    if (!dirac_check_device_ptr(out) || !dirac_check_device_ptr(in))
        return h->fail(DIRAC_ERR_INVALID_ARG, "dirac_apply_static: in and out must be device pointers");
    void* base = nullptr;
    dirac_status st;
    if ((st = scratch_address(h, cur, &base))) return st;
    void* a = base;
    void* b = static_cast<char*>(base) + field_padded;
    // the packing kernel writes every real site of a, which is all the sweep
    // reads, and the sweep writes every real site of b, which is all the
    // unpacking kernel reads; the padding sites of the last block of 32 keep
    // whatever an earlier call left there and are never read, so nothing
    // needs clearing
    if ((st = h->cuda(launch_pack_spinor(h->prec, nsc_of(h->op), h->g, h->Nv, in, h->prec == P_F64, a, h->stream),
                      "dirac_apply_static: pack")))
        return st;
    if ((st = h->run_apply(dagger != 0, b, a, h->Nv, h->diag, h->links, h->prec, h->cfg))) return st;
    return h->cuda(launch_unpack_spinor(h->prec, nsc_of(h->op), h->g, h->Nv, b, out, h->prec == P_F64, h->stream),
                   "dirac_apply_static: unpack");
}
