// Wilson D_W and D_W^+ sweeps (Sec. 4, Eq. def_wils at c_SW = 0) on the
// internal site-fastest layout.  One thread owns one site and R right-hand
// sides: every link is loaded once per thread and applied to its R spinors
// from registers, and every output element is written once.  Consecutive
// blocks cover the right-hand-side groups of the same sites, so the other
// groups find the links in L2.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "dirac_internal.h"

namespace dirac {

template <typename T>
cudaError_t wilson_go_T(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st);

bool wilson_tma_geometry(const Geom& g, int S, int* ny)
{
    if (S % 32 || S > 128 || S % g.L[0]) return false;
    const int n = S / g.L[0];
    if (n < 1 || g.L[1] % n) return false;
    if (g.L[0] % 4) return false;   // 16-byte rows of 16-bit links
    *ny = n;
    return true;
}

// 5-D views, innermost first: 16-byte word (4 x 32 bit), x (or x-chunks for
// links), y, z + Lz t, plane (v * K + k for spinors, mu * 9 + e for links).
// The boxes cover ny rows of one (z, t) plane and P spinor planes / 9 link planes.
bool wilson_tma_maps(const ApplyArgs& a, int prec, int P, int ny, void* mspin, void* mlink)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        else
            cudaGetLastError();
    });
    if (!encode) return false;
    const Geom& g = a.g;
    const int K = prec == P_F32 ? 6 : 3;
    const int LB = prec == P_F32 ? 8 : 4;
    const cuuint64_t Lx = g.L[0], Ly = g.L[1], ZT = (cuuint64_t)g.L[2] * g.L[3];
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    {
        const cuuint64_t dims[5] = {4, Lx, Ly, ZT, (cuuint64_t)a.Nv * K};
        const cuuint64_t strides[4] = {16, Lx * 16, Lx * Ly * 16, (cuuint64_t)g.vol * 16};
        const cuuint32_t box[5] = {4, (cuuint32_t)Lx, (cuuint32_t)ny, 1, (cuuint32_t)P};
        if (encode((CUtensorMap*)mspin, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, const_cast<void*>(a.in), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    {
        const cuuint64_t xc = Lx * LB / 16;
        const cuuint64_t dims[5] = {4, xc, Ly, ZT, 36};
        const cuuint64_t strides[4] = {16, Lx * LB, Lx * Ly * LB, (cuuint64_t)g.vol * LB};
        const cuuint32_t box[5] = {4, (cuuint32_t)xc, (cuuint32_t)ny, 1, 9};
        if (encode((CUtensorMap*)mlink, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, const_cast<void*>(a.links), dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

size_t wilson_tma_smem(int prec, int R, int S)
{
    const int RB = 2 * R;
    const size_t K = prec == P_F32 ? 6 : 3;
    const size_t LB = prec == P_F32 ? 8 : 4;
    const int nst = prec == P_F32 ? 3 : 4;
    return 256 + 128 + (size_t)nst * ((size_t)RB * K * S * 16 + 9 * S * LB);
}

size_t wilson_pipe_smem(int prec, int R, int block, int stages)
{
    const size_t K = prec == P_F64 ? 12 : (prec == P_F32 ? 6 : 3);
    const size_t LB = prec == P_F64 ? 16 : (prec == P_F32 ? 8 : 4);
    return (R * K * 16 + 9 * LB) * stages * block;
}

cudaError_t launch_apply_wilson(int prec, bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    switch (prec) {
    case P_F64: return wilson_go_T<double>(dag, a, c, st);
    case P_F32: return wilson_go_T<float>(dag, a, c, st);
    case P_BF16: return wilson_go_T<__nv_bfloat16>(dag, a, c, st);
    case P_F16: return wilson_go_T<__half>(dag, a, c, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dirac
