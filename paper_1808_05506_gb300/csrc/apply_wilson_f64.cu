// Wilson sweeps with f64 storage (instantiation of apply_wilson_impl.cuh).
#include "apply_wilson_impl.cuh"

namespace dirac {
template cudaError_t wilson_go_T<double>(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st);
}  // namespace dirac
