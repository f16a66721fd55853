/*
 * dirac.h -- C ABI of the GB300 multi-right-hand-side Dirac mat-vec library
 * (libdirac_gb300.so).
 *
 * The library computes out = D in for Nv right-hand sides at once, for the
 * three discretisations of S. Duerr, "Three Dirac operators on two
 * architectures with one piece of code and no hassle" (arXiv:1808.05506):
 *   DIRAC_STAGGERED  D_S, Sec. 3 (one-hop stencil with smeared links V_mu and
 *                    phases eta_mu), plus a mass term m
 *   DIRAC_WILSON     D_W, Sec. 4, Eq. def_wils at c_SW = 0
 *   DIRAC_BRILLOUIN  D_B, Sec. 5, Eqs. def_bril, def_der, def_lap at c_SW = 0,
 *                    with the off-axis links W_dir of Tab. tab:off-axis
 * Only Nc = 3 is built.  The clover term (c_SW != 0) is not offered.
 *
 * Conventions (fixed readings where the paper is silent):
 *   - site index s = x + Nx (y + Ny (z + Nz t)), coordinates 0-based,
 *     mu = 0..3 <-> x, y, z, t; periodic boundaries in all directions.
 *   - eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z).
 *   - V_mu(x) is the transporter from x+mu to x; V_{-mu}(x) = V_mu(x-mu)^+.
 *   - Euclidean chiral gamma basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *     gamma_4 = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1).
 *   - lattice spacing a = 1.
 *
 * Canonical layouts (C order, complex numbers as interleaved re, im):
 *   links   V[s][mu][a][b]                     (the transpose of the paper's
 *                                               Fortran U(Nc,Nc,4,...) matrix order)
 *   spinor  Wilson / Brillouin [s][v][spin][colour]  == the paper's vec(Nc,4,Nv,...)
 *           staggered          [s][v][colour]        == the paper's suv(Nc,Nv,...)
 *   Canonical spinors are complex double for DIRAC_F64 handles and complex
 *   float for every other precision.
 * Internal layout (blocked structure of arrays, in the storage precision;
 * allocate with dirac_field_bytes, convert with dirac_pack / dirac_unpack):
 *   spinor  [v][s/32][k][s%32] with k over the elements of one right-hand
 *           side (Wilson/Brillouin: 12 complex per site split into 16-byte
 *           elements of 2 complex (F32), 1 (F64) or 4 (BF16/F16); staggered:
 *           3 elements of one complex each); the sites go in blocks of 32,
 *           the last block padded, so a field holds ceil(vol / 32) * 32 sites.
 *
 * Pointers: unless a function says otherwise, spinor and field pointers are
 * DEVICE pointers owned by the caller, 16-byte aligned (else
 * DIRAC_ERR_INVALID_ARG); the library never frees them.  Work is
 * enqueued on the handle's CUDA stream and is asynchronous with respect to
 * the host unless stated.  One handle must not be used from two host threads
 * at once.
 *
 * Errors: every function returns a dirac_status; none aborts, throws or traps.
 * After an error, dirac_last_error(h) gives a one-line description.
 */
#ifndef DIRAC_GB300_H
#define DIRAC_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DIRAC_API __attribute__((visibility("default")))
#else
#define DIRAC_API
#endif

typedef enum {
    DIRAC_OK = 0,
    DIRAC_ERR_INVALID_ARG = 1,   /* bad pointer, size, aliasing, or call order */
    DIRAC_ERR_UNSUPPORTED = 2,   /* valid request this build does not offer (e.g. Nc != 3) */
    DIRAC_ERR_OOM = 3,           /* device allocation failed */
    DIRAC_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    DIRAC_NOT_CONVERGED = 5,     /* solver hit its iteration limit */
    DIRAC_BREAKDOWN = 6,         /* solver met a zero/NaN/Inf scalar */
    DIRAC_TIMEOUT = 7            /* a bounded device-side wait ran out */
} dirac_status;

typedef enum { DIRAC_STAGGERED = 0, DIRAC_WILSON = 1, DIRAC_BRILLOUIN = 2 } dirac_op;

/* storage precision of links and internal spinors (arithmetic is FP64 for
 * DIRAC_F64 and FP32 otherwise) */
typedef enum { DIRAC_F64 = 0, DIRAC_F32 = 1, DIRAC_BF16 = 2, DIRAC_F16 = 3 } dirac_prec;

typedef enum { DIRAC_CANONICAL = 0, DIRAC_INTERNAL = 1 } dirac_layout;

typedef struct dirac_handle dirac_handle;

/* Library version string (static storage). */
DIRAC_API const char* dirac_version(void);

/* Human-readable name of a status code (static storage). */
DIRAC_API const char* dirac_status_string(dirac_status st);

/* Create a handle for one operator on one lattice.
 *   op            DIRAC_STAGGERED / DIRAC_WILSON / DIRAC_BRILLOUIN
 *   Nc            number of colours; only 3 is supported (else UNSUPPORTED)
 *   Nx..Nt        lattice extents, each >= 2 (else INVALID_ARG); odd extents
 *                 are accepted (the staggered phases are then not
 *                 translation invariant across the boundary)
 *   Nv            right-hand sides per sweep, >= 1
 *   mass          staggered: m;  Wilson: the hopping parameter kappa > 0
 *                 (m0 = 1/(2 kappa) - 4, Sec. 4 def_wils);  Brillouin: m0
 *   prec          storage precision
 *   stream        cudaStream_t to enqueue on (NULL = the legacy default stream)
 * The handle is bound to the CUDA device current at creation.  It owns its
 * link storage and workspaces.  Returns INVALID_ARG for a NULL h. */
DIRAC_API dirac_status dirac_create(dirac_handle** h, dirac_op op, int Nc, int Nx, int Ny, int Nz,
                          int Nt, int Nv, double mass, dirac_prec prec, void* stream);

/* Release a handle and everything it owns (NULL is a no-op). */
DIRAC_API dirac_status dirac_destroy(dirac_handle* h);

/* Change the mass parameter (same meaning as in dirac_create). */
DIRAC_API dirac_status dirac_set_mass(dirac_handle* h, double mass);

/* Change the stream the handle enqueues on. */
DIRAC_API dirac_status dirac_set_stream(dirac_handle* h, void* stream);

/* Load the gauge links V_mu(x) (Sec. 2 array U, Sec. 3 smeared links).
 *   V          canonical links [s][mu][a][b], complex, Nx Ny Nz Nt * 4 * 9 entries
 *   V_prec     DIRAC_F64 (complex double) or DIRAC_F32 (complex float)
 *   on_device  1: V is a device pointer; 0: a host pointer (copied)
 * Converts to the internal layout in the storage precision and, for
 * Brillouin, builds the 40 stored off-axis links W_dir of Tab. tab:off-axis
 * (the average over the k! hop orderings, computed in FP64 by the recursion
 * W_dir(x) = (1/k) sum_{hops a} V_a(x) W_{dir-a}(x+a), then rounded).
 * Synchronous: returns after the links are in place.  The caller keeps
 * ownership of V. */
DIRAC_API dirac_status dirac_set_links(dirac_handle* h, const void* V, dirac_prec V_prec, int on_device);

/* Bytes of one spinor field with the handle's Nv right-hand sides. */
DIRAC_API dirac_status dirac_field_bytes(const dirac_handle* h, dirac_layout layout, size_t* bytes);

/* Convert a canonical spinor field (complex double for F64 handles, complex
 * float otherwise) into the internal layout and storage precision, and back.
 * Device pointers; out must not alias in. */
DIRAC_API dirac_status dirac_pack(dirac_handle* h, void* internal_out, const void* canonical_in);
DIRAC_API dirac_status dirac_unpack(dirac_handle* h, void* canonical_out, const void* internal_in);

/* out = D in for all Nv right-hand sides (Sec. 3 / def_wils / def_bril).
 * layout DIRAC_CANONICAL: in/out canonical (packed to the internal layout in
 * a handle-owned workspace, applied, unpacked); DIRAC_INTERNAL: in/out in the
 * internal layout and storage precision.  Device pointers, out != in.
 * Requires dirac_set_links first (else INVALID_ARG).  Asynchronous. */
DIRAC_API dirac_status dirac_apply(dirac_handle* h, void* out, const void* in, dirac_layout layout);

/* out = D in (dagger = 0) or D^+ in (dagger != 0) with out and in canonical
 * fields in HOST memory (no counterpart in the paper, whose fields live in
 * the memory of the node that sweeps them): the same result as copying in
 * to the device, dirac_apply(..., DIRAC_CANONICAL) and copying out, with the
 * copies overlapped with the work.  The lattice is cut into about 16 slabs of
 * t-slices; the host-to-device copy of one slab, the pack / sweep / unpack
 * of an earlier one and the device-to-host copy of a finished one run at
 * the same time on two copy streams of the handle and the handle's stream.
 *   out, in   host pointers (complex double for F64 handles, complex float
 *             otherwise), Nx Ny Nz Nt * Nv * spin * 3 entries; page-locked
 *             memory (cudaHostAlloc / cudaHostRegister) lets the copies
 *             overlap, pageable memory works with copies that block the
 *             calling thread; they must not overlap (INVALID_ARG), device
 *             pointers are rejected (INVALID_ARG).
 * Launch shape: the handle's kernel configuration when it is variant 0, 1, 2,
 * 5, 6 or 7 (the ones that can sweep a t-slab), else variant 1 with the same R.
 * Holds two staging buffers per direction of one slab each (allocated on
 * the first call, kept in the handle) and the handle's apply workspace.
 * Requires dirac_set_links first.  Asynchronous: out is complete when the
 * handle's stream has reached this point (dirac_sync). */
DIRAC_API dirac_status dirac_apply_host(dirac_handle* h, void* out, const void* in, int dagger);

/* out = D^+ in.  Staggered: D_S^+ = m - (hopping part of D_S) (the hopping
 * part is anti-hermitian, Sec. 3); Wilson, Brillouin: D^+ = gamma5 D gamma5.
 * Same contract as dirac_apply. */
DIRAC_API dirac_status dirac_apply_dagger(dirac_handle* h, void* out, const void* in, dirac_layout layout);

/* Link gradient of the loss L = Re <g, D psi> = Re sum_x g(x)^+ (D psi)(x)
 * (the backward pass of out = D psi with respect to the links; the backward
 * pass with respect to psi is dirac_apply_dagger on g).  Convention for a
 * real function of complex links (PyTorch's): F = dL/dRe V + i dL/dIm V.
 * Staggered (Sec. 3):  F_mu(x) = 1/2 eta_mu(x) sum_v [g_v(x) psi_v(x+mu)^+ - psi_v(x) g_v(x+mu)^+]
 * Wilson (def_wils):   F_mu(x) = -1/2 sum_v,s [(1-gamma_mu) g_v(x)]_s psi_v(x+mu)_s^+
 *                                -1/2 sum_v,s psi_v(x)_s [(1+gamma_mu) g_v(x+mu)]_s^+
 * Brillouin (Sec. 5, Tab. tab:off-axis): through the transporters W, which
 *   are rebuilt from V in FP64 here (not kept from the forward pass):
 *   G_dir(y) = sum_v,s g_v(y)_s (M_dir psi_v(y+dir))_s^+ is passed down the
 *   recursion W_dir(x) = (1/k) sum_a H_a(x) W_{dir-a}(x+a) to the links.
 *   Holds two FP64 scratch fields of 81 * 9 complex per site (11.7 KB per
 *   site each) during the call.
 *   F        device, canonical link layout [s][mu][a][b], complex double for
 *            F64 handles and complex float otherwise; written once per link
 *   psi, g   device spinor fields in `layout`
 * Asynchronous. */
DIRAC_API dirac_status dirac_force(dirac_handle* h, void* F, const void* psi, const void* g,
                                   dirac_layout layout);

/* Statistics of one dirac_solve call. */
typedef struct {
    int outer_iterations;   /* refinement steps (inner solves) taken */
    int inner_iterations;   /* inner CGLS iterations summed over the refinement steps */
    int sweeps;             /* storage-precision applications of D or D^+ (with even-odd
                               inner solves, each pair of half-lattice sweeps counts one) */
    int fp64_sweeps;        /* FP64 applications of D (outer residuals) */
    int even_odd;           /* 1 if the inner solves took the even-odd Schur complement */
    int df_residual;        /* 1 if the outer residuals ran in double-float arithmetic */
    int split_fields;       /* 1 if the inner solves kept split fields (dirac_set_inner_fields) */
    double residual_max;    /* max over right-hand sides of |b - D x| / |b|, FP64 */
    double seconds;         /* host wall time of the call */
} dirac_solve_stats;

/* Solve D x = b for all Nv right-hand sides (each with its own scalars and
 * convergence test) by defect correction: the outer loop forms the true
 * residual r = b - D x with FP64 links, an FP64 sweep and FP64 norms, and
 * stops when |r_v| / |b_v| <= tol for every v; each refinement step solves
 * D e = r / |r| approximately by CGLS (conjugate gradients on D^+ D, carrying
 * the residual of D e = r_hat) with fields in the handle's storage precision
 * and FP32 arithmetic (FP64 for DIRAC_F64 handles), to |r_hat - D e| <=
 * inner_tol |r_hat| or max_inner iterations, then updates x += |r| e in FP64.
 * With even-odd preconditioning (dirac_set_preconditioner; on by default where
 * it applies) the inner solve runs on the Schur complement of the odd sites
 * instead (see there); the outer loop and its FP64 residual are the same.
 *   x            canonical FP64 device field; on entry the starting guess
 *                (resume = call again with the previous result)
 *   b            canonical FP64 device field, not aliasing x
 *   tol          target relative residual, > 0 (e.g. 1e-10)
 *   max_outer    maximum refinement steps, >= 1
 *   max_inner    maximum CGLS iterations per step, >= 1
 *   inner_tol    relative residual reduction per step, in (0, 1); 0 picks the
 *                reduction the inner fields can reach: FP64 1e-10, FP32 (and
 *                split fields, see dirac_set_inner_fields) 1e-5, FP16 2e-3,
 *                BF16 1e-2
 *   rel_residual host array of Nv doubles for the final |b - D x| / |b| (or NULL)
 *   stats        host struct (or NULL)
 * Blocks until done.  Returns DIRAC_OK, DIRAC_NOT_CONVERGED (x holds the
 * last iterate), DIRAC_BREAKDOWN (non-finite residual) or an error. */
DIRAC_API dirac_status dirac_solve(dirac_handle* h, void* x, const void* b, double tol, int max_outer,
                                   int max_inner, double inner_tol, double* rel_residual,
                                   dirac_solve_stats* stats);

/* Per-system result of dirac_solve_batched. */
typedef struct {
    int converged;          /* 1 if every column of the system reached tol */
    int outer_iterations;   /* refinement steps, max over the system's columns */
    double residual_max;    /* max over its columns of |b - D x| / |b|, FP64 */
} dirac_system_stats;

/* Solve nsys systems D(m_i) x_i = b_i that share the handle's gauge field,
 * each with its own number of right-hand sides Nv_i and mass m_i (same
 * meaning as in dirac_create: staggered m, Wilson kappa, Brillouin m0), by the
 * defect correction of dirac_solve.  The handle's Nv is the number of
 * resident right-hand-side slots: columns of the systems are admitted from a
 * queue (in system order) into free slots; all resident columns share every
 * sweep (one launch for all systems, the mass entering as a per-column
 * diagonal), each has its own scalars and stopping test, and a column is
 * written back to x_i and its slot refilled as soon as it converges.  Groups
 * of 8 inner iterations run as one captured CUDA graph.
 *   Nv_i, mass_i      host arrays of nsys entries
 *   x_i, b_i          host arrays of nsys device pointers to canonical FP64
 *                     fields with Nv_i right-hand sides; x_i holds the start
 *   rel_residual      host array of sum_i Nv_i doubles (system-major) or NULL
 *   sys_stats         host array of nsys entries or NULL
 *   stats             host struct (totals) or NULL
 * Blocks until every column converged or hit max_outer.  Returns DIRAC_OK,
 * DIRAC_NOT_CONVERGED, DIRAC_BREAKDOWN or an error. */
DIRAC_API dirac_status dirac_solve_batched(dirac_handle* h, int nsys, const int* Nv_i, const double* mass_i,
                                           void* const* x_i, const void* const* b_i, double tol, int max_outer,
                                           int max_inner, double inner_tol, double* rel_residual,
                                           dirac_system_stats* sys_stats, dirac_solve_stats* stats);

/* out = D in (dagger = 0) or D^+ in (dagger != 0) on canonical device fields,
 * with the same result as dirac_apply(h, out, in, DIRAC_CANONICAL) /
 * dirac_apply_dagger, but allocating no device memory: the two internal-layout
 * work fields of the canonical apply live in a fixed 64 MiB array inside the
 * library's device image instead of memory the handle allocates.  (This entry
 * point has no counterpart in the paper; it exists for callers that cannot
 * allocate while they run: loops that cannot afford the device
 * synchronisation cudaMalloc / cudaFree may cause, and hosts whose device
 * memory is reserved up front by their own allocator, where a library
 * allocation would fail or take memory the host has promised elsewhere.)
 *   - The array is reserved on every GPU that loads the library and kept
 *     until the process exits.
 *   - The first call on a device (and the first after that device's context
 *     was destroyed and recreated, e.g. by cudaDeviceReset) looks up the
 *     array's device address with that device current; make that first call
 *     before any stream capture.  The handle's device must be the current
 *     device.
 *   - Fields whose two internal copies need more than 64 MiB (2 x
 *     dirac_field_bytes(h, DIRAC_INTERNAL), each rounded up to 256 bytes) are
 *     rejected with DIRAC_ERR_INVALID_ARG; use dirac_apply for those.  An
 *     FP32 Wilson or Brillouin field takes 96 bytes per site and right-hand
 *     side, so 2 x 96 x Nv x sites <= 64 MiB: 16^4 with Nv <= 5, 8^4 with
 *     Nv <= 85 (BF16 / FP16 half of that, FP64 twice, staggered a quarter).
 *   - Every call uses the same array, and a call leaves its contents behind
 *     (the padding sites of the last block of 32 are never read, so nothing
 *     needs clearing).  Calls whose work overlaps on the GPU (other streams,
 *     other handles, other host threads) race on it: serialise them.
 * Requires dirac_set_links first.  Asynchronous on the handle's stream. */
DIRAC_API dirac_status dirac_apply_static(dirac_handle* h, void* out, const void* in, int dagger);

/* Preconditioning of the inner solves of dirac_solve and dirac_solve_batched
 * (Sec. 4 names the even-odd decomposition as the next step of tuning).
 *   mode 1 (default): even-odd where it applies -- Wilson and staggered
 *          operators, every lattice extent even, and a nonzero diagonal
 *          (4 + m0, or the staggered mass m) for every system.  With D = a + H
 *          and H linking only sites of opposite parity, the inner solve of
 *          D e = r takes the Schur complement S = a - H_oe H_eo / a on the odd
 *          sites, S e_o = r_o - H_oe r_e / a (CGLS for Wilson; CG for
 *          staggered, where S = m + H_eo^+ H_eo / m is hermitian and
 *          definite), then e_e = (r_e - H_eo e_o) / a.  Its fields hold half
 *          the sites; one application of S costs two half-lattice sweeps.
 *   mode 0: the inner solve on the whole lattice (CGLS on D).
 * Elsewhere (Brillouin: its 2- and 4-hop terms link sites of equal parity; an
 * odd extent; a zero mass) mode 1 falls back to mode 0.  The stats field
 * even_odd reports which one ran.  Errors: DIRAC_ERR_INVALID_ARG for another
 * mode. */
DIRAC_API dirac_status dirac_set_preconditioner(dirac_handle* h, int mode);
DIRAC_API dirac_status dirac_get_preconditioner(const dirac_handle* h, int* mode);

/* Fields of the inner solves of 16-bit handles (Wilson with even-odd inner
 * solves, Brillouin with its whole-lattice inner solve).
 *   mode 0: every inner field in the handle's 16-bit precision.
 *   mode 1 (split, the default): the search directions p and s = A^+ r (and
 *          the Wilson adjoint sweep's intermediate) in 16 bits; the solution
 *          e, the residual r, the products t = A p and the links (Brillouin:
 *          all 80 W per site, as in link format 1) in FP32.  Because t is formed exactly (to FP32)
 *          from the 16-bit p that also updates e, the recursive residual stays
 *          the true one to FP32 accuracy, so an inner solve reaches FP32-level
 *          reductions (the rounding of p only perturbs the search directions)
 *          while half of its vector traffic and the sweeps' direction inputs
 *          stay 16-bit.
 * Other handles (FP32, FP64, staggered, Wilson whole-lattice inner solves)
 * ignore the mode.  The stats field split_fields reports it.
 * Measured (4 Wilson systems on 32^3 x 64, 24 slots, to 1e-10): split BF16
 * 5.26 s and FP16 5.20 s, against 7.27 s / 6.48 s with all fields in 16 bits
 * and 5.61 s for FP32 storage; the split solve takes the FP32 solve's
 * iteration counts.
 * Errors: DIRAC_ERR_INVALID_ARG for another mode. */
DIRAC_API dirac_status dirac_set_inner_fields(dirac_handle* h, int mode);
DIRAC_API dirac_status dirac_get_inner_fields(const dirac_handle* h, int* mode);

/* Arithmetic of the outer residual r = b - D x of dirac_solve and
 * dirac_solve_batched (the FP64 step of the defect correction).
 *   mode 0: FP64 links, fields and arithmetic (the default of DIRAC_F64 handles).
 *   mode 1: the same FP64 links and fields, with the sweep D x in double-float
 *           arithmetic -- each value an unevaluated sum of two FP32 numbers,
 *           48-bit significand, relative precision about 4e-15 -- and b - D x
 *           and the norms in FP64 (the default of the other handles).  FP64
 *           arithmetic runs at a small fraction of the FP32 rate on this GPU,
 *           so this sweep is several times faster, and it resolves
 *           |r| / |b| well below 1e-10.
 * Mode 1 needs values within FP32's exponent range: a call falls back to
 * mode 0 when a right-hand side's mean square |b|^2 / n lies outside
 * (1e-36, 1e36).  The stats field df_residual reports which one ran.
 * Errors: DIRAC_ERR_INVALID_ARG for another mode. */
DIRAC_API dirac_status dirac_set_residual_arithmetic(dirac_handle* h, int mode);
DIRAC_API dirac_status dirac_get_residual_arithmetic(const dirac_handle* h, int* mode);

/* Kernel configuration (the launch shape of the sweeps):
 *   R        right-hand sides per thread (1..4 for Wilson and Brillouin; 1, 2, 4
 *            or 6 for staggered); each link is loaded once per thread and
 *            applied to its R right-hand sides from registers
 *   block    threads per block (variants 0 and 3; a multiple of 32, 32..256;
 *            variant 5: 32..192) or sites per block (variants 1, 2 and 6: 32
 *            or 64, variant 2 also 128)
 *   variant  0: the right-hand-side groups of a site run in consecutive blocks;
 *            1: the groups of the same sites share one block, so that each link
 *               comes from L2 once per block and is reused through L1;
 *            2: (Wilson, R <= 2) variant 1 over site columns: each thread walks up
 *               to 8 consecutive t-slices of its (x, y, z) site, reading each
 *               spinor and t-link along t once (the t hops are carried from
 *               one slice to the next in registers);
 *            4: not used;
 *            3: (Wilson) variant 0 with a three-stage cp.async pipeline that
 *               keeps the next two hops in flight in shared memory; needs
 *               3 * block * (R * spinor bytes + link bytes) <= 227 KB;
 *            5: (Wilson, FP32/BF16/FP16, R <= 2) variant 2 with a warp on 32
 *               consecutive sites of the (x, y, z) volume: the x hops are
 *               exchanged between lanes by warp shuffles instead of loaded;
 *               needs Lx to divide 32 and Lx * Ly * Lz divisible by 32;
 *               block / 32 right-hand-side groups share a block;
 *            6: (Wilson with R <= 2, and staggered; FP32/BF16/FP16; the
 *               lattice rule of variant 5) variant 1 with the x hops done
 *               last by lane exchange: each site's own spinor, loaded once,
 *               serves the diagonal term and both x hops, so two of the nine
 *               spinor loads and one of the eight link loads per site
 *               disappear; 32 or 64 sites per block;
 *            7: (Brillouin, BF16/FP16 storage, R = 1, block = 128) the sweep on
 *               the tensor cores (tcgen05.mma, 16-bit operands, FP32
 *               accumulation in tensor memory): per site the colour sums
 *               T_j = sum_d C_j(d) W_d(x) psi(x + d) of the five coefficient
 *               classes (C_0 = -lambda_k / 2, C_{1+mu} = rho_k d_mu) are one
 *               real matrix product, the spin matrices and the diagonal are
 *               applied afterwards; one CTA per SM walks x-rows (about 200 KB
 *               of shared memory, all 512 tensor-memory columns).  The C_j W
 *               are rounded to the storage type (rho_k first rounded to it),
 *               so results differ from variants 0 and 1 by a few units of
 *               the storage rounding.  Selecting it selects link format 1.
 * UNSUPPORTED for other values. */
DIRAC_API dirac_status dirac_set_kernel_config(dirac_handle* h, int R, int block, int variant);

DIRAC_API dirac_status dirac_get_kernel_config(const dirac_handle* h, int* R, int* block, int* variant);

/* Site order of the sweeps of variants 0, 1 and 6 (no counterpart in the paper,
 * whose KNL code walks the lattice in its storage order): the order in which
 * consecutive thread blocks take the sites.
 *   tchunk = 0    lexicographic (x fastest, then y, z, t);
 *   0 < tchunk <= Nt   the (z, t) planes of Nx*Ny sites are taken in chunks
 *                 of tchunk t-slices, t faster than z inside a chunk, so that
 *                 the t-neighbours of a site are swept a few planes after it
 *                 and are still in L2 (with 12 FP32 right-hand sides a 32^3
 *                 t-slice and its output are larger than half the L2).
 * Results do not depend on it.  Kept across dirac_set_kernel_config; chosen
 * by dirac_autotune.  INVALID_ARG outside 0..Nt. */
DIRAC_API dirac_status dirac_set_site_order(dirac_handle* h, int tchunk);
DIRAC_API dirac_status dirac_get_site_order(const dirac_handle* h, int* tchunk);

/* Link format of the apply sweeps (gauge compression; Sec. 4, last
 * paragraph, names it as a next step, and the caption of Tab. tab:off-axis
 * gives W_{-dir}(x) = W_dir(x - dir)^+, which lets D_B store 40 of its 80 W).
 *   fmt 0 (default): Wilson and staggered read all nine entries of each link;
 *          Brillouin reads the 40 stored W, W_{-dir} as the adjoint of W_dir at
 *          the neighbour x - dir.
 *   fmt 1: Wilson and staggered (FP32, BF16, FP16 storage) read only the
 *          first two rows of each link and rebuild the third as
 *          U_2c = conj(U_0 x U_1)_c, which holds for special unitary links:
 *          two thirds of the link bytes.  Selecting it checks the links in
 *          FP64: max |U_2c - conj(U_0 x U_1)_c| must be <= 1e-6 (FP32) or
 *          <= 1e-2 (16-bit storage), else DIRAC_ERR_INVALID_ARG and format 0
 *          stays.  Brillouin (every precision) reads all 80 W stored at x
 *          (W_{-dir}(x) precomputed, copied without rounding): twice the W
 *          bytes, local reads only.
 * Format 1 is read by the launch variants that support it (Wilson and
 * staggered: variants 1 and 6; Brillouin: variants 0, 1 and 7) in the apply
 * and in the whole-lattice inner sweeps of the solvers; other variants and
 * the even-odd sweeps read the plain links; variant 7 reads only format 1.
 * The format-1 copy (Wilson/staggered: 4 x 6 complex per site; Brillouin:
 * 80 x 9, and for BF16/FP16 a second, site-major copy that variant 7 reads)
 * is held by the handle and rebuilt by dirac_set_links; links that fail the
 * check there switch the handle back to format 0 (dirac_get_link_format
 * reports it).  Called before dirac_set_links, fmt 1 is recorded and built
 * (and checked) there.  dirac_autotune times both formats and keeps the
 * faster.  Results agree with format 0 to rounding (Brillouin: bit for bit).
 * Errors: DIRAC_ERR_INVALID_ARG (fmt not 0 or 1, links not special unitary),
 * DIRAC_ERR_UNSUPPORTED (two-row links of an FP64 handle). */
DIRAC_API dirac_status dirac_set_link_format(dirac_handle* h, int fmt);
DIRAC_API dirac_status dirac_get_link_format(const dirac_handle* h, int* fmt);

/* Autotuner (the paper's "best of breed" selection, Sec. 4 and Sec. 6: time
 * every built variant on this machine and keep the winner): times each
 * supported (R, block, variant) of dirac_set_kernel_config, variants 0 and 1
 * with both site orders 0 and min(8, Nt), on the handle's own
 * workspace and keeps the fastest in the handle.  With the environment
 * variable DIRAC_TUNE_CACHE naming a writable file, results are cached per
 * (operator, precision, lattice, Nv, GPU name) and reused unless force != 0.
 * It also times link format 1 (dirac_set_link_format) on the shapes that read
 * it (variant 7 only there), when the links allow it, and keeps the faster
 * format.
 * Synchronous.  R, block, variant, ms (host, may be NULL) receive the choice
 * and its median time per sweep in milliseconds (from the cache when reused). */
DIRAC_API dirac_status dirac_autotune(dirac_handle* h, int force, int* R, int* block, int* variant, double* ms);

/* Wait for the handle's stream and report kernel-side failures: returns
 * DIRAC_TIMEOUT (and clears the record) if a kernel recorded that a bounded
 * device-side wait ran out since the last call (the tensor-core sweep,
 * variant 7, waits on its own CTA's barriers for at most half a second per
 * wait), else DIRAC_OK or the CUDA error of the stream. */
DIRAC_API dirac_status dirac_sync(dirac_handle* h);

/* One-line description of the last error on h (or of the last failed
 * dirac_create when h is NULL).  Static or handle-owned storage. */
DIRAC_API const char* dirac_last_error(const dirac_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* DIRAC_GB300_H */
