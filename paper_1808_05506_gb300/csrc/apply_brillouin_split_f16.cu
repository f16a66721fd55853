// Brillouin sweeps of the split inner solve, FP16 directions (apply_brillouin_split.cuh).
#include "apply_brillouin_split.cuh"

namespace dirac {

cudaError_t brillouin_split_prepare_f16(cudaStream_t st) { return split_table(st); }

cudaError_t launch_brillouin_split_f16(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st)
{
    return split_launch<__half>(dag, a, c, st);
}

}  // namespace dirac
