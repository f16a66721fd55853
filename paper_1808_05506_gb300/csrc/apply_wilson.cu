// Wilson D_W and D_W^+ sweeps (Sec. 4, Eq. def_wils at c_SW = 0) on the
// internal blocked layout.  One thread owns one site and R right-hand
// sides: every link is loaded once per thread and applied to its R spinors
// from registers, and every output element is written once.  Consecutive
// blocks cover the right-hand-side groups of the same sites, so the other
// groups find the links in L2.
#include "dirac_internal.h"

namespace dirac {

template <typename T>
cudaError_t wilson_go_T(bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st);

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
