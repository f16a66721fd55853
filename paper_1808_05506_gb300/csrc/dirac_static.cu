// dirac_apply_static: out = D in (or D^+ in) on canonical fields, like
// dirac_apply with DIRAC_CANONICAL, but without any device allocation.
//
// The canonical apply converts its input into the internal layout and back
// through two internal-layout work fields.  dirac_apply keeps them in memory
// the handle allocates on first use; this entry point keeps them instead in
// one fixed array in the library's own device memory, reserved when the
// library's device code is loaded on a GPU and kept until the process exits.
// It serves callers that must not allocate while they work: code enqueuing
// into a stream that is being captured into a CUDA graph (cudaMalloc is not
// allowed there), latency-critical loops that cannot afford cudaMalloc /
// cudaFree (which can synchronise the device), and hosts whose device memory
// is entirely reserved up front by their own allocator.
#include <mutex>

#include "dirac_handle.h"

using namespace dirac;

namespace {

// 64 MiB: room for the two work fields of lattices up to about 32 MiB per
// field (e.g. 8^4 x 12 right-hand sides, 16^4 x 2, FP32 Wilson).
constexpr size_t kScratchBytes = size_t(64) << 20;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// The device address of g_scratch on the current device.  In host code the
// name g_scratch is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
dirac_status scratch_address(dirac_handle* h, int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return h->fail(DIRAC_ERR_UNSUPPORTED, "dirac_apply_static: device %d beyond the %d supported", dev,
                       kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return h->fail(DIRAC_ERR_CUDA, "dirac_apply_static: cannot resolve the static scratch area: %s",
                           cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
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
    // the packing kernel overwrites every element of a that the sweep reads and
    // the sweep writes every element of b, so nothing needs clearing
    if ((st = h->cuda(launch_pack_spinor(h->prec, nsc_of(h->op), h->g, h->Nv, in, h->prec == P_F64, a, h->stream),
                      "dirac_apply_static: pack")))
        return st;
    if ((st = h->run_apply(dagger != 0, b, a, h->Nv, h->diag, h->links, h->prec, h->cfg))) return st;
    return h->cuda(launch_unpack_spinor(h->prec, nsc_of(h->op), h->g, h->Nv, b, out, h->prec == P_F64, h->stream),
                   "dirac_apply_static: unpack");
}
