// Even-odd Wilson sweeps (dirac_eo.cuh), one instantiation per storage type
// and right-hand sides per thread.
#include "dirac_eo.cuh"

namespace dirac {

cudaError_t launch_eo_wilson(int prec, bool dag, const EoArgs& a, int R, int block, cudaStream_t st)
{
#define GO(T) \
    return R == 2 ? eo_go<OP_WILSON, T, 2>(dag, a, block, st) : eo_go<OP_WILSON, T, 1>(dag, a, block, st)
    switch (prec) {
    case P_F64: return eo_go<OP_WILSON, double, 1>(dag, a, block, st);   // R = 1 (R = 2 spills)
    case P_F32: GO(float);
    case P_BF16: GO(__nv_bfloat16);
    case P_F16: GO(__half);
    default: return cudaErrorInvalidValue;
    }
#undef GO
}

}  // namespace dirac
