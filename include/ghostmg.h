/*
 * ghostmg.h - C ABI of the GB300 (sm_103a) geometric multigrid solver for the
 * nodal ghost finite element method of Dilip & Coco, "Multigrid methods for
 * the ghost finite element approximation of elliptic problems"
 * (arXiv 2505.05105).
 *
 * Problem (Sec. 2, Eq. poisson_model_prob with a Dirichlet boundary):
 *     -Laplace u = f in Omega = {psi < 0},   u = g on {psi = 0},
 * discretised with Q1 elements on the active cells of an N x N Cartesian grid
 * (Eq. Vhact) and Nitsche terms on the cut cells (Eq. disc_bil_form,
 * Eq. disc_rhs), with the local stabilisation lambda_K = gamma C(K) of
 * Sec. 5.2 (or one global lambda, MG_LAMBDA_GLOBAL) and snapping back to
 * grid with threshold h^alpha (Sec. 2).  Neumann data on marked cut cells
 * and strong Dirichlet box sides are options (mg_bc).  The
 * system A u = F is solved by V(nu1, nu2)-cycles (Sec. 3.2) with a 4-colour
 * Gauss-Seidel smoother (Sec. 4.1) plus eta extra sweeps on the cut-cell
 * vertices (Sec. 5.3), bilinear prolongation P and restriction R = P^T
 * (Sec. 5.1) and Galerkin coarse operators (Eq. galerkin); W-cycles, the
 * two-grid scheme (Alg. 1) and re-discretised coarse levels are options
 * (mg_stab).  Batches of independent problems (mg_batch_*) and the 1D model
 * of Sec. 4 (mg1d_cycles) have their own calls at the end of this file.
 *
 * Arrays: every nodal array has (N+1)^2 doubles, row-major with node index
 * k = i + j (N+1) (Sec. 5.1), node (i, j) at (x0 + i h, y0 + j h).
 * Array arguments may be device pointers (used on the handle's stream) or
 * host pointers.  Pinned host memory mapped into the device's address space
 * is read and written in place by the kernels (only the entries they use);
 * pageable host memory is staged through handle-owned device buffers, and
 * the mg_export_* calls always copy.  Every call returns after its results
 * are in the caller's arrays.
 * The caller owns every array; no pointer is kept after a call returns.
 *
 * Errors: every int-returning call returns MG_OK (0) or one of the MG_ERR_*
 * codes below; nothing is thrown across the ABI.  After MG_ERR_CUDA the
 * handle should be destroyed.  mg_strerror() gives a message, including the
 * last CUDA error text when there was one.
 *
 * Threading: one handle per CUDA stream; calls on different handles are
 * independent, with one exception: mg_residual_static calls share one
 * library-wide scratch array, so those that overlap on the GPU race (see
 * there).  A handle must not be used from two threads at once.
 */
#ifndef GHOSTMG_H
#define GHOSTMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,    /* bad size, NULL pointer, NaN/Inf input,
                                domain touching the outer ring of nodes */
  MG_ERR_CUDA = 2,           /* a CUDA runtime call or kernel failed */
  MG_ERR_NOT_CONVERGED = 3,  /* max_cycles reached; outputs and info filled */
  MG_ERR_DIVERGED = 4,       /* residual not finite or 1e3 x above its best */
  MG_ERR_NOT_SPD = 5,        /* coarsest Cholesky met a pivot <= 0 */
  MG_ERR_TIMEOUT = 6,        /* a bounded device wait ran out (mg_set_wait_limit) */
  MG_ERR_UNIMPLEMENTED = 7,  /* option not supported (e.g. Neumann data) */
  MG_ERR_INTERNAL = 8,       /* internal consistency check failed */
  MG_ERR_OUT_OF_MEMORY = 9   /* device allocation failed */
};

enum { MG_BC_DIRICHLET = 0,       /* weak Dirichlet on the whole of {psi = 0} */
       MG_BC_MIXED = 1 };         /* Dirichlet / Neumann by a per-cell mask */
enum { MG_LAMBDA_LOCAL = 0,       /* lambda_K = gamma C(K) per cut cell (Sec. 5.2) */
       MG_LAMBDA_GLOBAL = 1 };    /* lambda = gamma c_global on every cut cell (Sec. 5.2) */
enum { MG_COARSE_GALERKIN = 0,    /* A_2h = P^T A_h P (Eq. galerkin) */
       MG_COARSE_REDISCRETISE = 1 };  /* A_2h assembled on the coarse grid */
enum { MG_FP64 = 0,               /* fp64 V-cycles */
       MG_MIXED = 1 };            /* fp32 V-cycle inside fp64 iterative refinement */

typedef struct mg_ctx* mg_handle;

/* Grid of Omega_art (Sec. 2): n_cells x n_cells cells of side h with the
 * lower-left node at (x0, y0).  n_cells is a power of two >= 8;
 * coarsest_cells (a power of two, 2..32, dividing n_cells; default 8) is the
 * size of the level solved exactly (Alg. 1, step 3). */
typedef struct {
  int n_cells;
  double x0, y0;
  double h;
  int coarsest_cells;
} mg_grid;

/* Boundary conditions (Eq. poisson_model_prob: u = g_D on Gamma_D,
 * n . grad u = g_N on Gamma_N).
 *   kind = MG_BC_DIRICHLET, neumann_mask = NULL: all of {psi = 0} is
 *     Dirichlet, imposed weakly (Nitsche terms of Eq. disc_bil_form).
 *   kind = MG_BC_MIXED: neumann_mask holds n_cells^2 bytes (host or device,
 *     read during mg_setup only), cell (ic, jc) at ic + jc n_cells; a cut
 *     cell with a nonzero byte has its piece of the boundary in Gamma_N: it
 *     keeps only its volume stiffness (Eq. disc_bil_form has no boundary
 *     term on Gamma_N) and adds int_{K cap Gamma_N} g_N phi_i to the load
 *     (Eq. disc_rhs, g_N through its Q1 interpolant of nodal values, see
 *     mg_solve_bc).  Bytes of other cells are ignored.  Some Dirichlet
 *     data must remain (a Dirichlet cut cell or box_sides): with Neumann
 *     data alone u is fixed only up to a constant, A is singular, and setup
 *     fails with MG_ERR_NOT_SPD or the solves do not converge.
 * Any other combination is MG_ERR_INVALID_ARG.
 *   box_sides != 0: strong Dirichlet conditions on the sides of the box
 *     (the rectangle example of Sec. 5.3): every node with i or j equal to
 *     0 or n_cells is a Dirichlet node with value g_D (the g array of
 *     mg_solve), not a DOF; Omega may then reach the box sides.  Its
 *     couplings to the DOFs move to the right-hand side (F - A_pq g_q), the
 *     coarse levels keep their box nodes out too, and u is 0 there on
 *     output; mg_adjoint's dL/dg then also holds the box nodes' share,
 *     -(B^T w)_q for the couplings B moved to the right-hand side. */
typedef struct {
  int kind;
  const uint8_t* neumann_mask;
  int box_sides;
} mg_bc;

/* Method parameters (defaults from mg_default_stab):
 *   gamma = 2     lambda_K = gamma C(K)                       (Sec. 5.3)
 *   alpha = 1.75  snapping threshold h^alpha                   (Sec. 5.3)
 *   eta = 4       extra cut-cell sweeps per smoothing step     (Sec. 5.3), 0..8
 *   nu1 = 2, nu2 = 1  pre/post smoothing steps                 (Sec. 5.3), 0..8
 *   lambda_mode = MG_LAMBDA_LOCAL: lambda_K = gamma C(K), C(K) the largest
 *                 generalized eigenvalue of the cell's pencil (Sec. 5.2);
 *                 MG_LAMBDA_GLOBAL: lambda = gamma c_global on every cut
 *                 cell, c_global the largest generalized eigenvalue of the
 *                 global pencil K v = Lambda M v of Sec. 5.2 (K: normal
 *                 derivatives on Gamma_D, M: stiffness on Omega_h, both over
 *                 the whole FE space), in 1/length units: the caller's
 *                 value when c_global > 0; with c_global = 0 mg_setup
 *                 computes it on the GPU (the pencil taken modulo constants,
 *                 Lanczos with inner conjugate-gradient solves; n_cells <=
 *                 1024 and no box_sides, else MG_ERR_UNIMPLEMENTED;
 *                 mg_get_c_global reads it back).  Negative or non-finite
 *                 c_global: MG_ERR_INVALID_ARG.  Not with
 *                 MG_COARSE_REDISCRETISE nor in batches
 *                 (MG_ERR_UNIMPLEMENTED).  C(K) is still reported per cell.
 *   precision = MG_FP64 or MG_MIXED
 *   max_cycles = 100  V-cycles in total (both precisions)
 *   inner = 0     V-cycles between two fp64 residual checks, 0..8:
 *                 0 = chosen after each check from the contraction seen so
 *                 far, as the number predicted to reach tol (first group 4,
 *                 at most 8); k > 0 = always k.  In MG_MIXED each group is
 *                 one refinement step: fp64 residual, `k` fp32 V-cycles on
 *                 the correction equation (the first from e = 0), u += e.
 *   cycle = 1     cycles on each coarse level per visit (Alg. 1, gamma*):
 *                 1 = V-cycle, 2 = W-cycle (batches: V only); 0 = the
 *                 two-grid correction scheme of Alg. 1 (the coarse equation
 *                 of the finest level solved exactly -- by 40 V-cycles of
 *                 the coarser hierarchy, which leave an error at rounding
 *                 level -- for convergence studies; MG_FP64 only).
 *   coarse_op = MG_COARSE_GALERKIN  coarse operators A_2h = P^T A_h P
 *                 (Eq. galerkin); MG_COARSE_REDISCRETISE: each coarse level
 *                 assembled from scratch on its own grid from the level set
 *                 at its nodes (snapped with h_l^alpha, its own cut cells
 *                 and lambda_K), the alternative the paper describes beside
 *                 Eq. galerkin (not with MG_BC_MIXED: MG_ERR_UNIMPLEMENTED).
 *   fuse_max_tiles = 0  kernel choice on the levels between the finest and
 *                 the 64 x 64-cell tail (MG_MIXED only; the arithmetic is
 *                 the same either way): a level with at most this many
 *                 active 64 x 32-node tiles runs each smoothing step as one
 *                 fused kernel, a larger one runs the separate sweep, extra
 *                 sweep, restriction and prolongation kernels.  0 = the
 *                 device's SM count (one wave of the fused kernel); -1 =
 *                 never fused; >= -1 otherwise (MG_ERR_INVALID_ARG). */
typedef struct {
  double gamma, alpha;
  int eta, nu1, nu2;
  int lambda_mode, precision, max_cycles;
  int inner;
  int cycle;
  int coarse_op;
  double c_global;        /* MG_LAMBDA_GLOBAL only; default 0 */
  int fuse_max_tiles;
} mg_stab;

/* Result summary of a solve. */
typedef struct {
  int cycles;             /* V-cycles run (both precisions) */
  double rel_res;         /* final ||F - A u||_inf / ||F||_inf, in fp64 */
  double res_hist[64];    /* rel_res at check 0 (before cycle 1), 1, 2, ... */
  int n_dof;              /* fine-level DOFs (vertices of active cells) */
  int n_cut;              /* fine-level cut cells */
  int n_levels;           /* levels including the coarsest */
  float setup_ms;         /* wall time of mg_setup */
  float solve_ms;         /* wall time of the last mg_solve (device events) */
  int checks;             /* fp64 residual checks after the initial one */
} mg_info;

/* Fills *out with the defaults above.  Returns MG_ERR_INVALID_ARG if out is
 * NULL. */
int mg_default_stab(mg_stab* out);

/* Builds the discretisation and the multigrid hierarchy on the GPU.
 *   levelset  (N+1)^2 nodal psi (Omega = {psi < 0}); copied, then snapped
 *             (Sec. 2) and classified (Sec. 5.2).  psi after snapping must be
 *             >= 0 on the outer ring of nodes (i or j equal to 0 or N).
 *   grid, bc, stab  as documented above; stab may be NULL (defaults).
 *   cuda_stream     cudaStream_t to run on (NULL = legacy default stream).
 * Runs: snapping and cell classes (Sec. 2); cut geometry, element matrices
 * with exact quadrature and C(K) (Sec. 5.2, Eq. c_triangle, Eq. c_pentagon,
 * the local eigenvalue definition for quadrilaterals); per-node operator
 * rows; Galerkin coarse levels A_2h = P^T A_h P (Eq. galerkin); the
 * coarsest-level inverse.  On success *out owns all device memory of the
 * hierarchy; release it with mg_destroy.  Errors: MG_ERR_INVALID_ARG,
 * MG_ERR_UNIMPLEMENTED, MG_ERR_NOT_SPD, MG_ERR_OUT_OF_MEMORY, MG_ERR_CUDA
 * (*out is left NULL). */
int mg_setup(mg_handle* out, const double* levelset, const mg_grid* grid, const mg_bc* bc,
             const mg_stab* stab, void* cuda_stream);

/* Solves A u = F with F = M f + G g (Eq. disc_rhs; f and g enter through
 * their Q1 interpolants, g being any extension of the Dirichlet data to the
 * nodes).  u holds the initial guess on entry (non-DOF entries ignored) and
 * the solution on exit, with 0 on nodes that are not DOFs.  Cycles stop when
 * ||F - A u||_inf / ||F||_inf <= tol (fp64 residual) or after max_cycles.
 * info may be NULL.  f, g, u: (N+1)^2 doubles, device or host.  Host arrays
 * in page-locked memory mapped into the device's address space (pinned
 * allocations) are read and written in place by the kernels, which touch
 * only the entries the computation uses; other host arrays are copied
 * through device buffers.  Only these entries are read: f at the vertices
 * of active cells, g at the vertices of cut cells (and the box nodes with
 * strong box sides), u at the DOFs.
 * Errors: MG_ERR_INVALID_ARG (NULL pointer, NaN/Inf in an entry that is
 * read: f or g where it enters F, u at a DOF),
 * MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED (u and info still filled),
 * MG_ERR_CUDA. */
int mg_solve(mg_handle h, const double* f, const double* g, double* u, double tol,
             mg_info* info);

/* mg_solve with Neumann data: F = M f + G g_D + N g_N (Eq. disc_rhs), N
 * the Neumann cut cells' boundary mass.  g_D and g_N are nodal arrays like
 * f ((N+1)^2 doubles, device or host); g_N may be NULL (g_N = 0) and is
 * ignored on a handle without Neumann cells; only its values at vertices of
 * Neumann cut cells matter (an extension of the Neumann data off Gamma_N,
 * e.g. grad u . n with n extended smoothly, and only those are read).
 * Errors as mg_solve (NaN/Inf in g_N at such a vertex: MG_ERR_INVALID_ARG). */
int mg_solve_bc(mg_handle h, const double* f, const double* g_D, const double* g_N, double* u,
                double tol, mg_info* info);

/* Adjoint of mg_solve for a loss L(u): solves A w = dL/du (A is symmetric,
 * Sec. 4.1) to the tolerance of the last mg_solve (1e-10 if none) by
 * transposed V-cycles in fp64 (mg_cycles_transposed; the same stop test
 * and check schedule as mg_solve, whatever the handle's precision), then
 * dL/df = M^T w and dL/dg = G^T w (F is linear in f and g, Eq. disc_rhs).
 * dLdu, dLdf, dLdg: (N+1)^2 doubles, device or host; dLdf or dLdg may be
 * NULL to skip it (not both).  dL/du off the DOFs is ignored; both outputs
 * are 0 off the DOFs, dL/dg also away from cut cells.  The right-hand side
 * dL/du has no h^2 mass factor, so the fp64 rounding floor of this solve
 * relative to ||dL/du||_inf is about eps / h^2: ask for a tolerance above it.
 * Errors as mg_solve (MG_ERR_NOT_CONVERGED: outputs still written). */
int mg_adjoint(mg_handle h, const double* dLdu, double* dLdf, double* dLdg);

/* mg_adjoint with mixed boundary conditions: also dL/dg_N = N^T w (F holds
 * N g_N, Eq. disc_rhs; zero away from Neumann cut cells, and everywhere on
 * a handle without Neumann cells).  Any of dLdf, dLdg, dLdgN may be NULL
 * (not all three). */
int mg_adjoint_bc(mg_handle h, const double* dLdu, double* dLdf, double* dLdg, double* dLdgN);

/* Releases the handle and its device memory (NULL is ignored). */
void mg_destroy(mg_handle h);

/* Static message for a status code (with the last CUDA error text after
 * MG_ERR_CUDA). */
const char* mg_strerror(int code);

/* ---------------------------------------------------------------------------
 * Step-level entry points (the same kernels as mg_solve, exposed so that
 * each step can be checked on its own).  Arrays as above.
 * ------------------------------------------------------------------------- */

/* The global constant of Sec. 5.2 a handle set up with MG_LAMBDA_GLOBAL
 * uses (the caller's c_global, or the one mg_setup computed when c_global
 * was 0; 0 under MG_LAMBDA_LOCAL), and for a computed one the Lanczos steps
 * and conjugate-gradient iterations it took (0 otherwise).  Any output may
 * be NULL. */
int mg_get_c_global(mg_handle h, double* c_global, int* lanczos_steps, int* cg_iterations);

/* The bounds-checked debug build (a library variant compiled with
 * -DMG_CHECK_BOUNDS; not a part of the method).  Its kernels check every
 * node index, boundary-row index and boundary-list position where it is
 * formed; a failed check sets a per-device word and the access is redirected
 * inside its array (no fault), and every call that synchronizes then returns
 * MG_ERR_INTERNAL.  *enabled = 1 in that build, 0 in the normal one (where
 * *hits is always 0).  *hits: nonzero when a check failed on the current
 * device since the last reset; reset != 0 clears it.  Synchronizes the
 * current device.  Any output may be NULL.  Errors: MG_ERR_CUDA. */
int mg_bounds_check(int* enabled, unsigned* hits, int reset);

/* Poll budget of the handle's bounded device waits (the completion waits of
 * the shared-memory tensor and bulk copies; not a part of the method).
 * Every such wait gives up after `polls` polls of its mbarrier (polls < 0:
 * the default, 2^22, seconds at least); the kernel then records the timeout,
 * waits with the default budget for its own copy still in flight, and stops
 * without using the data, and the call returns MG_ERR_TIMEOUT at its next
 * check (u is then not a solution).  polls = 0 makes every wait give up at
 * once: a way to exercise that path.  The handle stays usable.
 * MG_ERR_INVALID_ARG for a NULL handle or polls above 2^32 - 1. */
int mg_set_wait_limit(mg_handle h, long long polls);

/* Sizes of the hierarchy: levels, fine DOFs, fine cut cells, boundary nodes
 * (vertices of cut cells) on the fine level.  Any pointer may be NULL. */
int mg_get_counts(mg_handle h, int* n_levels, int* n_dof, int* n_cut, int* n_boundary);

/* Cells per side of level `level` (0 = finest), or -1 for a bad level. */
int mg_level_cells(mg_handle h, int level);

/* DOFs of level `level` (0 = finest), or -1 for a bad level. */
int mg_level_dofs(mg_handle h, int level);

/* The 9-point rows of the level-`level` operator: out[9 k + s] = A_{k, k'}
 * with k' the neighbour at offset (s mod 3 - 1, s / 3 - 1), k = i + j (n+1);
 * zero rows on nodes that are not DOFs.  out: 9 (n+1)^2 doubles. */
int mg_export_stencil(mg_handle h, int level, double* out);

/* Fine-level cut cells in increasing cell index c = ic + jc N.  For each of
 * the first max_cells: cells[t] = c; data[52 t ..] = C(K), lambda_K,
 * |K cap Omega_h|, |Gamma_h cap K|, Ke (16, row-major, local vertex order
 * (0,0),(1,0),(0,1),(1,1)), Mk (16), Gk (16).  Returns the number of cut
 * cells in *n_total.  cells/data: host or device. */
int mg_export_cut_cells(mg_handle h, int max_cells, int* cells, double* data, int* n_total);

/* F = M f + G g on the fine level (Eq. disc_rhs), zero off the DOFs.  Reads
 * f and g as mg_solve does; MG_ERR_INVALID_ARG if a NaN/Inf among them
 * enters F. */
int mg_rhs(mg_handle h, const double* f, const double* g, double* F);
/* F = M f + G g_D + N g_N (as mg_solve_bc; g_N may be NULL). */
int mg_rhs_bc(mg_handle h, const double* f, const double* g_D, const double* g_N, double* F);

/* Exactly k cycles from u with right-hand side F (no stopping test):
 * precision MG_FP64 runs k V-cycles; MG_MIXED runs k refinement steps (fp64
 * residual, stab.inner fp32 V-cycles -- one if inner = 0 -- on the
 * correction equation from e = 0, fp64 update).  u in/out. */
int mg_cycles(mg_handle h, const double* F, double* u, int k, int precision);

/* Exactly k transposed V-cycles (fp64) from u with right-hand side F: the
 * cycle whose approximate inverse is B^T for the V-cycle's B (u <- u +
 * B (F - A u), Sec. 3.2): nu2 transposed smoothing steps (the eta cut-node
 * sweeps, then the full sweep, colours in the reverse order), restriction,
 * the transposed cycle below, prolongation, nu1 transposed smoothing steps.
 * A is symmetric, so k of them from u = 0 give the transpose of k V-cycles
 * from 0; mg_adjoint solves with them.  u in/out. */
int mg_cycles_transposed(mg_handle h, const double* F, double* u, int k);

/* r = F - A u on the fine level (fp64); norms[0] = ||r||_inf,
 * norms[1] = ||r||_2 (host array of 2, may be NULL); r may be NULL. */
int mg_residual(mg_handle h, const double* F, const double* u, double* r, double* norms);

/* ---------------------------------------------------------------------------
 * Allocation-free residual.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory while they use the
 * solver -- real-time loops that cannot take the device-wide
 * synchronisation that cudaMalloc or cudaFree may cause, and frameworks
 * whose own caching allocator must own all device memory (a hard memory
 * cap, no fragmentation by a library's private allocations).
 *
 * Same result as mg_residual (r = F - A u on the fine level, norms[0] =
 * ||r||_inf, norms[1] = ||r||_2), but it allocates nothing and uses no
 * handle-owned scratch: F, u and r are read and written in place in the
 * caller's (N+1)^2 layout, and the norm reduction uses a file-scope device
 * array of 2 MG_NOALLOC_MAX_TILES + 2 doubles (1 MiB), which every GPU that
 * loads the library keeps until the process exits.  ||r||_2 is summed in a
 * fixed order, so it is reproducible.
 *   F, u, r  device pointers on the handle's device; r may be NULL (norms
 *            only); u is read as 0 on nodes that are not DOFs; r gets 0
 *            there.
 *   norms    host or device array of 2 doubles, or NULL.
 * The work runs on the handle's stream and device (the caller's current
 * device is restored), and the call waits for it: it synchronises the
 * handle's stream before returning, so the results are in place on return.
 * Errors: MG_ERR_INVALID_ARG for NULL or host F/u/r, arrays on another
 * device than the handle's, or a fine level with more than
 * MG_NOALLOC_MAX_TILES active 64 x 32-node tiles (every n_cells <= 8192
 * fits); MG_ERR_CUDA.
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  All calls share the one array, and each
 * call writes every slot it reads before reading it, so nothing carries
 * over from one call to the next; but calls that overlap on the GPU (other
 * threads, streams or handles) race on it and must be serialised.
 * ------------------------------------------------------------------------- */
#define MG_NOALLOC_MAX_TILES 65536
int mg_residual_static(mg_handle h, const double* F, const double* u, double* r, double* norms);

/* ---------------------------------------------------------------------------
 * Profiling: device time per kernel class, measured with CUDA events
 * recorded around each launch on the handle's stream while enabled, and a
 * count of every kernel the handle launches.  Slots:
 * ------------------------------------------------------------------------- */
enum {
  MG_PROF_SWEEP = 0,     /* fine-level Gauss-Seidel sweeps */
  MG_PROF_BAND = 1,      /* fine-level extra sweeps on cut-cell vertices */
  MG_PROF_RESTRICT = 2,  /* fine-level residual + restriction */
  MG_PROF_PROLONG = 3,   /* fine-level prolongation + correction */
  MG_PROF_RESIDUAL = 4,  /* fine-level fp64 residual (stopping test, refinement) */
  MG_PROF_UPDATE = 5,    /* refinement update u += e */
  MG_PROF_COARSE = 6,    /* other coarse-level kernels (coarsest solve,
                            the fp64 transposed cycle) */
  MG_PROF_IO = 7,        /* right-hand side, input checks, pack/unpack */
  MG_PROF_LEVELS = 8,    /* sweeps on the levels between the finest and the
                            tail that do not run fused steps */
  MG_PROF_FUSED = 9,     /* fused smoothing steps (fp32 intermediate levels) */
  MG_PROF_TAIL = 10,     /* the single-block V-cycle of the smallest levels */
  MG_PROF_LEVELS_BAND = 11,      /* extra sweeps on those levels */
  MG_PROF_LEVELS_RESTRICT = 12,  /* residual + restriction, prolongation there */
  MG_PROF_SLOTS = 13
};

/* enable != 0: clear the accumulators and start recording; 0: stop. */
int mg_set_profiling(mg_handle h, int enable);

/* Kernel launches since profiling was last enabled (*launches), and per
 * slot the number of timed launch groups (counts[MG_PROF_SLOTS]) and their
 * total device milliseconds (ms[MG_PROF_SLOTS]).  Any pointer may be NULL. */
int mg_get_profile(mg_handle h, long long* launches, long long* counts, double* ms);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent problems, each with its own level set and
 * grid size, solved together in mixed precision (the fp32 V(nu1, nu2)-cycle
 * of mg_solve inside fp64 iterative refinement, with the adaptive check
 * schedule of mg_stab.inner = 0, or a fixed one).  One persistent kernel
 * takes the members from a work queue, largest first, and runs each
 * member's whole solve in one thread block: the levels above 64 x 64 cells
 * block-wide in global memory, the smaller ones in shared memory.  A solve
 * is one CUDA graph (input check, right-hand sides, the persistent kernel,
 * output copy and status read-back).
 *
 * Packed arrays: member p has (N_p + 1)^2 nodes, N_p = grids[p].n_cells,
 * stored row-major as above from offset off_p = sum over q < p of
 * (N_q + 1)^2 doubles; a packed array holds all members, total_nodes
 * doubles.
 * ------------------------------------------------------------------------- */
typedef struct mg_batch_ctx* mg_batch;

/* Per-member result of mg_batch_solve. */
typedef struct {
  int status;        /* MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, or
                        MG_ERR_INVALID_ARG (NaN/Inf in the member's f or g
                        where it enters F; its u is 0) */
  int cycles;        /* fp32 V-cycles run */
  int checks;        /* fp64 residual checks after the initial one */
  int n_dof;         /* fine-level DOFs */
  double rel_res;    /* final ||F - A u||_inf / ||F||_inf (fp64) */
} mg_batch_info;

/* Sets up count >= 1 members: levelsets is a packed array (host or device)
 * of the members' nodal psi; grids[count] their grids (host).  bc and stab
 * as for mg_setup and shared by all members, except that with MG_BC_MIXED
 * bc->neumann_mask holds the members' cell masks one after another (member
 * p's n_cells^2 bytes after those of members 0 .. p-1); stab->precision
 * must be MG_MIXED (or stab NULL).  cuda_stream: the caller's stream; the
 * batch orders its work after the work queued there when a call starts, and
 * runs on a stream of its own (a graph cannot be captured on the legacy
 * stream).  Errors as mg_setup, and MG_ERR_UNIMPLEMENTED for MG_FP64 or a
 * W-cycle. */
int mg_batch_setup(mg_batch* out, int count, const mg_grid* grids, const double* levelsets,
                   const mg_bc* bc, const mg_stab* stab, void* cuda_stream);

/* *total_nodes: doubles in a packed array; f, g, u (any may be NULL): the
 * batch's own device packed arrays, valid until mg_batch_destroy. */
int mg_batch_buffers(mg_batch b, long long* total_nodes, double** f, double** g, double** u);

/* Solves every member: f, g, u packed arrays (host or device; u is output
 * only, every member starts from u = 0).  Device arrays and host arrays in
 * mapped page-locked memory are read and written in place (f and g only
 * where they enter F: f at the vertices of active cells, g at the vertices
 * of cut cells); other host arrays are copied through the batch's own
 * buffers.  info: count entries or NULL.
 * Returns MG_OK when every member converged, else the most severe member
 * status (MG_ERR_INVALID_ARG, then MG_ERR_DIVERGED, then
 * MG_ERR_NOT_CONVERGED; u and info filled for all members); MG_ERR_TIMEOUT
 * if a bounded shared-memory copy wait ran out; MG_ERR_CUDA. */
int mg_batch_solve(mg_batch b, const double* f, const double* g, double* u, double tol,
                   mg_batch_info* info);

/* mg_batch_solve with Neumann data: g_N a packed array like f (ignored on a
 * batch set up without MG_BC_MIXED; NULL: g_N = 0).  A member with NaN/Inf
 * in its g_N at a vertex of a Neumann cut cell fails alone with
 * MG_ERR_INVALID_ARG. */
int mg_batch_solve_bc(mg_batch b, const double* f, const double* g, const double* g_N, double* u,
                      double tol, mg_batch_info* info);

/* Launch shape of the persistent kernel. */
typedef struct {
  int threads;        /* threads per block: 256, 512 or 1024 */
  int first_group;    /* V-cycles before the first fp64 check (adaptive
                         schedule), 1..8 */
  int cluster;        /* blocks per thread-block cluster: 1, 2, 4 or 8 */
  int coop_min_dof;   /* members with at least this many fine-level DOFs and
                         levels above 64 x 64 cells are solved by a whole
                         cluster, each block on its own SM (cluster > 1) */
} mg_batch_shape;

/* Sets the launch shape (default 1024 threads, first group 4, clusters of 2
 * for members above 8192 DOFs; 512 threads without clusters where that
 * shape cannot be resident).
 * MG_ERR_INVALID_ARG for values outside the lists above or a shape that
 * cannot be resident on the device (the previous shape is kept). */
int mg_batch_set_shape(mg_batch b, const mg_batch_shape* shape);
int mg_batch_get_shape(mg_batch b, mg_batch_shape* shape);

/* Autotuner: times `reps` graph replays (after one warm-up) of the solve of
 * (f, g) to tol for candidate shapes, in three stages -- threads per block
 * x cluster size; then cluster size in {2, 4, 8} x the sharing threshold
 * coop_min_dof in {0, 8192, 32768, 65536, 131072}; then, with the adaptive
 * schedule, first_group in {2, 3, 4, 6} -- and keeps the fastest shape whose
 * members all converge.  best and ms (mean time per solve) may be NULL.
 * Errors as mg_batch_solve (MG_ERR_NOT_CONVERGED if no candidate converged
 * everywhere; the previous shape is kept). */
int mg_batch_tune(mg_batch b, const double* f, const double* g, double tol, int reps,
                  mg_batch_shape* best, float* ms);

/* Wall time of mg_batch_setup and device time of the last solve's graph. */
int mg_batch_timing(mg_batch b, float* setup_ms, float* solve_ms);

/* Releases the batch (NULL is ignored). */
void mg_batch_destroy(mg_batch b);

/* ---------------------------------------------------------------------------
 * The one-dimensional model of Sec. 4 (convergence studies of Sec. 4.5).
 *
 * Omega_art = [0, 1] with n_cells cells of side h = 1/n_cells, Omega = (a, b),
 * a = (1 - theta1) h, b = 1 - (1 - theta2) h; the P1 hats phi_0..phi_n are all
 * DOFs; Dirichlet data at a by Nitsche's terms with penalty lambda, Neumann
 * data at b: the matrix of Eq. ls1dA.  Smoother: lexicographic Gauss-Seidel
 * (P = L_h, Sec. 4.1); restriction Eq. resop, prolongation its transpose;
 * Galerkin coarse operators (Eq. galerkin) down to 8 cells, solved exactly.
 * ------------------------------------------------------------------------- */
#define MG1D_MAX_CELLS 2048

typedef struct {
  int n_cells;            /* power of two, 16..MG1D_MAX_CELLS */
  double theta1, theta2;  /* in (0, 1] (taken as given: no snapping) */
  double lambda;          /* Nitsche penalty, finite and > 0 (Sec. 4.4:
                             lambda = gamma / (theta1 h) is the local choice) */
} mg1d_problem;

/* Runs `cycles` multigrid cycles on each of `count` independent problems
 * (one thread block each, all on cuda_stream).
 *   problems: host array of count problems.
 *   F: device, the right-hand sides packed one after another (n_cells + 1
 *      values per problem, in the order of problems), or NULL for F = 0 (the
 *      homogeneous problem of Sec. 4.5).
 *   u: device, packed the same way; in: the first iterate (u^(0) = 1 for
 *      Sec. 4.5), out: the iterate after `cycles` cycles.
 *   res: host, count x (cycles + 1) values: ||F - A u^(m)||_inf for
 *      m = 0..cycles, problem by problem (the convergence factor of Sec. 3.1
 *      is the ratio of successive entries).
 *   cycle: 0 = the two-grid correction scheme of Alg. 1 (coarse equation
 *      solved exactly), 1 = V-cycle, 2 = W-cycle (gamma* of Sec. 3.2);
 *   nu1, nu2 in 0..8 (not both 0); cycles in 0..1000.
 * Returns MG_ERR_INVALID_ARG for values outside these ranges or pointers of
 * the wrong kind, MG_ERR_NOT_SPD if an exact solve met a pivot <= 0, and
 * MG_ERR_CUDA on a CUDA error.  Blocks until the results are on the host. */
int mg1d_cycles(int count, const mg1d_problem* problems, int cycle, int nu1, int nu2,
                int cycles, const double* F, double* u, double* res, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GHOSTMG_H */
