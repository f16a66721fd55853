// Even-odd Wilson sweeps of the split inner solve (dirac_eo.cuh): FP32 links
// and FP32 solution, residual and operator products, with the search
// directions and the adjoint sweep's intermediate in 16 bits.
#include "dirac_eo.cuh"

namespace dirac {

template <typename H, int R>
static cudaError_t split_go(int kind, const EoArgs& a, int block, cudaStream_t st)
{
    switch (kind) {
    case EO_SPLIT_HP: return eo_go_typed<OP_WILSON, float, H, float, float, R, false>(a, block, st);
    case EO_SPLIT_SP: return eo_go_typed<OP_WILSON, float, float, H, float, R, false>(a, block, st);
    case EO_SPLIT_HR: return eo_go_typed<OP_WILSON, float, float, float, H, R, true>(a, block, st);
    case EO_SPLIT_SR: return eo_go_typed<OP_WILSON, float, H, float, H, R, true>(a, block, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_eo_wilson_split(int prec16, int kind, const EoArgs& a, LaunchCfg cfg, cudaStream_t st)
{
    if (a.vh == 0 || a.Nv == 0) return cudaSuccess;
    if (!eo_rhs_supported(OP_WILSON, P_F32, a.Nv, cfg.R)) return cudaErrorInvalidValue;
    if (prec16 == P_BF16)
        return cfg.R == 2 ? split_go<__nv_bfloat16, 2>(kind, a, cfg.block, st)
                          : split_go<__nv_bfloat16, 1>(kind, a, cfg.block, st);
    if (prec16 == P_F16)
        return cfg.R == 2 ? split_go<__half, 2>(kind, a, cfg.block, st) : split_go<__half, 1>(kind, a, cfg.block, st);
    return cudaErrorInvalidValue;
}

}  // namespace dirac
