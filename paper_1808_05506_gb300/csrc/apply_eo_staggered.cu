// Even-odd staggered sweeps (dirac_eo.cuh), one instantiation per storage
// type and right-hand sides per thread.
#include "dirac_eo.cuh"

namespace dirac {

cudaError_t launch_eo_staggered(int prec, bool dag, const EoArgs& a, int R, int block, cudaStream_t st)
{
#define GO(T)                                                          \
    return R == 4 ? eo_go<OP_STAGGERED, T, 4>(dag, a, block, st)       \
                  : (R == 2 ? eo_go<OP_STAGGERED, T, 2>(dag, a, block, st) \
                            : eo_go<OP_STAGGERED, T, 1>(dag, a, block, st))
    switch (prec) {
    case P_F64:   // R <= 2 (R = 4 spills)
        return R == 2 ? eo_go<OP_STAGGERED, double, 2>(dag, a, block, st)
                      : eo_go<OP_STAGGERED, double, 1>(dag, a, block, st);
    case P_F32: GO(float);
    case P_BF16: GO(__nv_bfloat16);
    case P_F16: GO(__half);
    default: return cudaErrorInvalidValue;
    }
#undef GO
}

}  // namespace dirac
