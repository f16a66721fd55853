// Brillouin sweeps of the split inner solve, BF16 directions (apply_brillouin_split.cuh).
#include "apply_brillouin_split.cuh"

namespace dirac {

cudaError_t launch_brillouin_split_f16(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st);
cudaError_t brillouin_split_prepare_f16(cudaStream_t st);

cudaError_t brillouin_split_prepare(int prec16, cudaStream_t st)
{
    if (prec16 == P_BF16) return split_table(st);
    if (prec16 == P_F16) return brillouin_split_prepare_f16(st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_brillouin_split(int prec16, bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    if (prec16 == P_BF16) return split_launch<__nv_bfloat16>(dag, a, c, st);
    if (prec16 == P_F16) return launch_brillouin_split_f16(dag, a, c, st);
    return cudaErrorInvalidValue;
}

}  // namespace dirac
