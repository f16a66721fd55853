// Host-side launchers shared between the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "dirac_common.cuh"
#include "dirac_kernels.cuh"

namespace dirac {

enum Op { OP_STAGGERED = 0, OP_WILSON = 1, OP_BRILLOUIN = 2 };

// complex numbers per site and right-hand side
inline int nsc_of(int op) { return op == OP_STAGGERED ? 3 : 12; }

// bytes of one storage-precision complex number
inline size_t cbytes(int prec)
{
    return prec == P_F64 ? 16 : (prec == P_F32 ? 8 : 4);
}

// Launch variants of a sweep
enum Variant {
    V_DIRECT = 0,   // one thread per (site, group of R right-hand sides); the groups of a
                    // site sit in consecutive blocks
    V_GROUPS = 1,   // the groups of the same sites share a block (blockDim.y), so each
                    // link is fetched from L2 once per block and reused through L1
    V_TMARCH = 2,   // Wilson: V_GROUPS over (x, y, z) site columns, each thread walking up to
                    // 8 consecutive t-slices with the t hops carried in registers
    V_PIPE3 = 3,    // Wilson: V_DIRECT with a 3-stage cp.async pipeline in shared memory
    // 4 is not used (a variant with bulk-copied tiles, retired with the blocked layout)
    V_XROW = 5,     // Wilson (FP32/BF16/FP16), Lx dividing 32: a warp holds 32 consecutive sites
                    // of the (x, y, z) volume (whole x-rows) and walks up to 8 t-slices; x hops
                    // by warp shuffles, t hops carried in registers; `block` = threads
                    // (block / 32 right-hand-side groups per block)
    V_XLAST = 6,    // Wilson (R <= 2) and staggered, FP32/BF16/FP16, Lx dividing 32 and 32
                    // dividing Lx Ly Lz: V_GROUPS with the x hops last, by lane exchange of the
                    // site's own spinor (wilson_site_xlast, staggered_site_xlast); `block` =
                    // sites per block (32 or 64)
    V_TC = 7        // Brillouin, BF16/FP16 storage, link format 1: the per-site contraction on
                    // the tensor cores (tcgen05.mma, apply_brillouin_tc.cu); R = 1, block = 128
};

struct LaunchCfg {
    int R;         // right-hand sides per thread
    int block;     // V_DIRECT, V_PIPE3: threads per block; V_GROUPS: sites per block
    int variant;   // Variant
    int order = 0; // V_DIRECT, V_GROUPS: site order of the grid (site_of t-chunk, 0 lexicographic)
    int fmt = -1;  // link format of the sweep (link_format_supported): 0 the plain links
                   // (Brillouin: 40 stored W); 1 Wilson / staggered two-row links,
                   // Brillouin all 80 W stored per site; -1 the handle's format
};

// whether a launch variant reads link format 1: Wilson and staggered
// V_GROUPS and V_XLAST with FP32 / 16-bit storage, Brillouin V_DIRECT and
// V_GROUPS
inline bool link_format_supported(int op, int prec, int variant)
{
    if (op == OP_BRILLOUIN) return variant == V_DIRECT || variant == V_GROUPS || variant == V_TC;
    return prec != P_F64 && (variant == V_GROUPS || variant == V_XLAST);
}

// threads per block of V_GROUPS: block sites x gy groups with block * gy <= 192
inline int groups_per_block(int block, int ngroups)
{
    int gy = 192 / block;
    return gy < ngroups ? gy : ngroups;
}

bool apply_config_supported(int op, int prec, int R, int block, int variant, const Geom& g);
size_t wilson_pipe_smem(int prec, int R, int block, int stages);

// two-row links [4][site/32][6][32] (rows 0, 1 of the storage links) and the
// largest deviation from special unitarity max |U_2c - conj(U_0 x U_1)_c|
// of the FP64 links V64 [4][9][site] (into *dev, a device double)
cudaError_t launch_links_2row(int prec, const Geom& g, const void* links, void* out, cudaStream_t st);
cudaError_t launch_su3_deviation(const Geom& g, const void* V64, double* dev, cudaStream_t st);
// Brillouin: all 80 directions per site [80][site/32][9][32] from the 40 stored
// ones: planes 0..39 copied, plane 40 + j holds W_{-d_j}(x) = W_{d_j}(x - d_j)^+
// (in place when out == links: an 80-plane array whose planes 0..39 are set)
cudaError_t launch_brillouin_w80(int prec, const Geom& g, const void* links, void* out, cudaStream_t st);

// out = D in (or D^+ in) on internal-layout fields
cudaError_t launch_apply(int op, int prec, bool dagger, const ApplyArgs& a, LaunchCfg cfg,
                         cudaStream_t st);
cudaError_t launch_apply_staggered(int prec, bool dagger, const ApplyArgs& a, LaunchCfg cfg,
                                   cudaStream_t st);
cudaError_t launch_apply_wilson(int prec, bool dagger, const ApplyArgs& a, LaunchCfg cfg,
                                cudaStream_t st);
cudaError_t launch_apply_brillouin(int prec, bool dagger, const ApplyArgs& a, LaunchCfg cfg,
                                   cudaStream_t st);

// Brillouin sweep on the tensor cores (V_TC; a.links = the 80 W per site in the
// 16-bit storage type); prepare uploads its direction table (once per device,
// before any stream capture)
cudaError_t brillouin_tc_prepare(cudaStream_t st);
cudaError_t launch_brillouin_tc(int prec, bool dag, const ApplyArgs& a, cudaStream_t st);
// the site-major copy of the 80 W (16-bit storage) the tensor-core sweep reads,
// from link format 1 ([80][9][site], blocked); needs brillouin_tc_prepare
cudaError_t launch_brillouin_tc_links(const Geom& g, const void* w80, void* wtc, cudaStream_t st);

// Brillouin sweeps of the split inner solve (apply_brillouin_split.cuh):
// dag = false t(F32) = D p(16), dag = true s(16) = D^+ r(F32), FP32 W; prepare
// uploads the direction table (once per device, before any stream capture)
cudaError_t brillouin_split_prepare(int prec16, cudaStream_t st);
cudaError_t launch_brillouin_split(int prec16, bool dag, const ApplyArgs& a, LaunchCfg c, cudaStream_t st);

// the 80 Brillouin directions and the dir81 code of each of the 40 stored ones
void brillouin_tables(BriDir dirs[80], int rep_dir81[40]);
cudaError_t upload_brillouin_table(cudaStream_t st);

// canonical (complex double if canon_f64 else complex float) <-> internal spinor;
// canon holds the sites site0 .. site0 + nsites - 1 (nsites < 0: all sites)
cudaError_t launch_pack_spinor(int prec, int nsc, const Geom& g, int Nv, const void* canon,
                               bool canon_f64, void* internal, cudaStream_t st, long site0 = 0,
                               long nsites = -1);
cudaError_t launch_unpack_spinor(int prec, int nsc, const Geom& g, int Nv, const void* internal,
                                 void* canon, bool canon_f64, cudaStream_t st, long site0 = 0,
                                 long nsites = -1);

// column c of a canonical FP64 field with Nsrc right-hand sides <-> slot v of an
// internal FP64 field
cudaError_t launch_pack_column64(int nsc, const Geom& g, int Nsrc, int c, const void* canon, int v, void* internal,
                                 cudaStream_t st);
cudaError_t launch_unpack_column64(int nsc, const Geom& g, int v, const void* internal, int Nsrc, int c, void* canon,
                                   cudaStream_t st);

// canonical links V[s][mu][a][b] -> FP64 internal [mu][9][s]
cudaError_t launch_links_to_f64(const Geom& g, const void* canon, bool canon_f64, void* V64,
                                cudaStream_t st);
// FP64 internal [m][9][s] -> storage precision internal [m][9][s] (nmat matrices per site)
cudaError_t launch_convert_links(int prec, const Geom& g, int nmat, const void* src64, void* dst,
                                 cudaStream_t st);
// Tab. tab:off-axis: FP64 links V64 [4][9][s] -> FP64 W64 [40][9][s]; tmp81 holds
// 81 * 9 * vol complex doubles.
cudaError_t launch_build_W81(const Geom& g, const void* V64, void* tmp81, cudaStream_t st);
cudaError_t launch_build_W(const Geom& g, const void* V64, void* tmp81, void* W64, cudaStream_t st);

// link gradient of Re <g, D psi> (staggered, Wilson); F canonical link layout
// Brillouin link gradient: W81, G81 are FP64 scratch fields of 81 * 9 * vol complex
cudaError_t launch_force_brillouin(int prec, const Geom& g, int Nv, const void* psi, const void* gv,
                                   const void* V64, void* W81, void* G81, void* F, cudaStream_t st);
cudaError_t launch_force(int op, int prec, const Geom& g, int Nv, const void* psi, const void* gv, void* F,
                         cudaStream_t st);

}  // namespace dirac
