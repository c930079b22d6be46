/*
 * sipg.h -- C ABI of the GB300 (sm_103a) matrix-free multigrid library for the
 * symmetric interior penalty (SIPG) DG discretisation of the Poisson problem
 * on Cartesian meshes of the unit square / cube, after Cui & Kanschat,
 * "Multilevel Interior Penalty Methods on GPUs" (arXiv 2405.18982).
 *
 * Problem (Sec. 2, Eqs. model, bilinear_form, weak_form, mat_form):
 *   find u_h in V_h (discontinuous Q_k, Lagrange basis on Gauss-Lobatto
 *   points, Appendix A) with kappa * a_h(u_h, v) = (f, v) for all v, a_h the
 *   SIPG form with penalty gamma_e = eta k(k+1)(1/h+ + 1/h-), also on
 *   boundary faces (h- := h+), homogeneous Dirichlet conditions imposed
 *   weakly.  Matrix form A x = b.
 *
 * Solver (Sec. 3): flexible CG (or the paper's GMRES, sipg_gmres_solve) on
 * the finest level, preconditioned by one multigrid V-cycle (Sec. 3) with the
 * colourised multiplicative vertex-patch smoother (Algorithm 1; Dirichlet,
 * full or clamped local solver, sipg_smoother), fast-diagonalisation local
 * solvers (Eqs. inverse2d, inverse3d, fast_inverse), canonical-embedding
 * prolongation and its transpose as restriction, and an exact coarse solve.
 * The V-cycle may run in FP32 inside the FP64 outer solver (Sec. 5.2).
 *
 * Data layout (Sec. 4.1): every vector is cell-wise lexicographic.  On a level
 * with N cells per direction and n = k+1 nodes per direction, DoF (cell c,
 * local node i) is at index c * n^d + i with c = c0 + N (c1 + N c2) and
 * i = i0 + n (i1 + n i2), index 0 fastest.  With nrhs > 1 the right-hand
 * sides are stored one after another: column r starts at r * n_dofs.
 *
 * Memory and streams: the caller owns all device memory.  sipg_create only
 * validates parameters and sizes; the caller then allocates
 * sipg_workspace_bytes() bytes of device memory (256-byte aligned) and binds
 * it with sipg_bind_workspace(), which runs the device-side level setup.  No
 * entry point allocates device memory.  Vector arguments are device pointers
 * unless stated otherwise, must be 16-byte aligned and must not alias unless
 * stated.  `stream` is a cudaStream_t (NULL = legacy default stream); all work
 * is ordered on it.  Only sipg_solve, sipg_adjoint_solve, sipg_solve_host
 * and sipg_gmres_solve synchronise (their stream), because convergence is
 * decided on the host.
 *
 * Errors: every call returns a sipg_status; failures never abort or trap.
 * sipg_last_error(h) returns a message for the last failure on h.
 *
 * Tuning (read by sipg_create): SIPG_FUSED_SMOOTHING=0 in the environment
 * turns off the single cooperative launch per smoothing step on small levels
 * (the colours are then launched one by one; the results are the same);
 * SIPG_AUTOTUNE=0 skips the bind-time autotuning (sipg_tuning); SIPG_TILE=0..4
 * pins the interior tile of the 3D FP32 colour pass on every level, whatever
 * the autotuner measured: 0 the default patches per CTA, 1 half as many, 2 the
 * default tile with b and x on V_j loaded ahead of the sweeps that use them, 3
 * that tile at three CTAs per SM (more registers per thread), 4 tile 3 with
 * the x and y sweeps on whole warps (each patch's lines on its own warps).
 * SIPG_BOUNDARY_FIRST=0 launches the interior-patch kernel of a colour pass
 * before the boundary-patch kernel (default: boundary patches first, at the
 * greatest stream priority; the results are the same).
 */
#ifndef SIPG_H
#define SIPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SIPG_OK = 0,
  SIPG_EINVAL = -1,           /* bad argument (null pointer, size, range)           */
  SIPG_ENOMEM_WORKSPACE = -2, /* workspace missing or too small                      */
  SIPG_ECUDA = -3,            /* a CUDA runtime call failed                          */
  SIPG_ENOCONV = -4,          /* solver hit maxit before rtol                        */
  SIPG_EBREAKDOWN = -5,       /* non-finite or non-positive Krylov scalar            */
  SIPG_ETIMEOUT = -6,         /* a bounded device-side wait ran out                  */
  SIPG_EUNSUPPORTED = -7,     /* valid but unsupported configuration                 */
  SIPG_ESTATE = -8            /* call out of order (e.g. workspace not bound)        */
} sipg_status;

/* Arithmetic of the V-cycle (operator apply, smoother, transfer); the outer
 * Krylov solver, its residual, dot products and updates, the 1D eigenpair
 * setup and the coarse solve are always FP64.  SIPG_TF32 (params only) is
 * the FP32 V-cycle whose interior 3D colour passes at degree 7 run the six
 * eigenvector sweeps of the fast-diagonalisation local solve (Eq. inverse3d)
 * on the tensor cores with TF32 operands and FP32 accumulation; everything
 * else, and the vector type of every call (prec arguments), is FP32. */
typedef enum {
  SIPG_FP64 = 0,
  SIPG_FP32 = 1,
  SIPG_TF32 = 2
} sipg_precision;

/* Local residual of the Dirichlet-kernel patch solver (Sec. 3.1). */
typedef enum {
  /* r_j = R_j (b - A x): exact residual, including the face-node layer of
   * the cells around the patch (default; symmetric V-cycle). */
  SIPG_SMOOTHER_CONSISTENT = 0,
  /* r_j = R_j b - Abar_j Rbar_j x with only the patch cells (the paper's
   * Dirichlet kernel, inconsistent residual): Abar_j is the form on the
   * patch cells in which the last face term -[[u]].{grad v} of the
   * patch-boundary faces inside the domain is left out (Sec. 3.1). */
  SIPG_SMOOTHER_PAPER = 1,
  /* The paper's full kernel (Sec. 3.1, Table 1): V_j is every DoF of the
   * 2^d patch cells and A_j the principal block of A on them, inverted by
   * fast diagonalisation with the 1D eigenpairs of the whole 2n-node patch.
   * The residual b - A x is updated globally once per colour (the choice
   * Sec. 3.1 makes for this kernel), then every patch of the colour adds its
   * correction: same-colour patches share faces but no DoFs, so inside a
   * colour the corrections are additive. */
  SIPG_SMOOTHER_FULL = 2,
  /* The paper's clamped kernel (Sec. 3.1, Table 2 right): V_j is the
   * functions on the patch cells whose value and normal derivative vanish on
   * the patch boundary inside the domain ((2k-2)^d of them for an interior
   * patch; no condition at a patch end on the domain boundary).  All face
   * terms of the patch boundary vanish for these test functions, so the
   * residual is exact.  The paper spans V_j by a Hermite-type basis; this
   * library keeps the Gauss-Lobatto Lagrange basis and applies the same
   * subspace correction (B (B^T A_D B)^{-1} B^T R_D r by fast
   * diagonalisation on the subspace), with the full kernel's launch
   * structure.  Needs degree >= 2. */
  SIPG_SMOOTHER_CLAMPED = 3
} sipg_smoother;

typedef struct {
  int dim;               /* 2 or 3                                                       */
  int degree;            /* k, 1..7                                                      */
  int log2_cells;        /* finest level has N = 2^log2_cells cells per direction        */
  int n_levels;          /* >= 1; level l has N >> (n_levels-1-l) cells, coarsest >= 2  */
  double kappa;          /* > 0, scalar diffusion coefficient multiplying the form      */
  double penalty_factor; /* eta > 0; gamma_e = eta k(k+1)(1/h+ + 1/h-) (paper: eta = 1) */
  int vcycle_precision;  /* sipg_precision                                               */
  int smoother;          /* sipg_smoother                                                */
  int nrhs;              /* >= 1 right-hand sides solved together                        */
  int use_graphs;        /* != 0: FCG iterations and GMRES cycles as CUDA graphs         */
} sipg_params;

typedef struct {
  int iterations;        /* outer FCG iterations done                                   */
  int status;            /* sipg_status of the solve                                    */
  double rel_residual;   /* max over rhs of ||b - A x||_2 / ||b||_2 (true residual)     */
  double nu;             /* fractional iteration count of Sec. 3.3 (8 digits), rhs 0    */
  double* history;       /* caller buffer (host) or NULL: ||r_i||_2 of rhs 0 per iter   */
  int history_capacity;  /* entries available in history                                */
  int history_len;       /* entries written                                             */
} sipg_info;

typedef struct sipg_handle sipg_handle;

/* Validate params and compute sizes; no CUDA call.  *out = NULL on error. */
sipg_status sipg_create(const sipg_params* params, sipg_handle** out);
void sipg_destroy(sipg_handle* h);
const char* sipg_last_error(const sipg_handle* h);
const char* sipg_version(void);

/* Bytes of device workspace the handle needs (level vectors, Krylov vectors,
 * reduction scratch, level constants). */
size_t sipg_workspace_bytes(const sipg_handle* h);
/* Bind caller-owned device memory (256-byte aligned, >= workspace bytes) and
 * run the FP64 device setup of all levels on `stream` (1D Gauss-Lobatto
 * basis, 1D SIPG blocks, patch eigenpairs of Eq. fast_inverse by Cholesky and
 * cyclic Jacobi, coarse-level eigenpairs, transfer matrices).  May be called
 * again with another buffer; the handle then uses the new one. */
sipg_status sipg_bind_workspace(sipg_handle* h, void* dev_ptr, size_t bytes, void* stream);

/* Number of DoFs of one right-hand side on `level` (0 = coarsest). */
size_t sipg_ndofs(const sipg_handle* h, int level);
/* Launches of library kernels issued since creation (kernels inside a CUDA
 * graph launch are counted once per graph launch). */
uint64_t sipg_launch_count(const sipg_handle* h);

/* b = M_h f on the finest level (Eq. weak_form with f given by nodal values
 * in V_h): the exact block-diagonal mass applied cell by cell.  FP64, nrhs
 * columns.  Also serves as dJ/df = M_h lambda in the adjoint. */
sipg_status sipg_rhs(sipg_handle* h, const double* f, double* b, void* stream);

/* f = d pi^2 prod_e sin(pi x_e) at the nodes of the finest level (the
 * manufactured source of u = prod_e sin(pi x_e)), written to every column. */
sipg_status sipg_manufactured_source(sipg_handle* h, double* f, void* stream);

/* y = A_level x (Eq. mat_form on that level, Sec. 2.2 matrix-free,
 * sum-factorised).  prec selects double* or float* vectors. nrhs columns. */
sipg_status sipg_apply(sipg_handle* h, int level, int prec, const void* x, void* y, void* stream);
/* r = b - A_level x (fused). r may alias b. */
sipg_status sipg_residual(sipg_handle* h, int level, int prec, const void* b, const void* x,
                          void* r, void* stream);
/* y = (dA/dgamma) x on the finest level: the penalty face terms with unit
 * penalty, times kappa (derivative with respect to the uniform fine-level
 * face penalty gamma). FP64. */
sipg_status sipg_apply_penalty(sipg_handle* h, const double* x, double* y, void* stream);

/* One colour pass of Algorithm 1 on `level`: for all vertex patches j of
 * colour c (c = sum_e (v_e mod 2) 2^e, v the vertex index), in parallel,
 * r_j = local residual, x[V_j] += (S (x) S (x) S) Lambda^{-1} (S^T (x) ...) r_j.
 * x is updated in place.  With the full or clamped kernel the pass first
 * writes b - A x for the whole level into the level's residual buffer of the
 * workspace (so passes of one handle must not overlap on the GPU). */
sipg_status sipg_smooth_colour(sipg_handle* h, int level, int prec, int colour, const void* b,
                               void* x, void* stream);
/* One smoothing step S_l(x, b): colours 0..2^d-1, or 2^d-1..0 if reverse. */
sipg_status sipg_smooth(sipg_handle* h, int level, int prec, int reverse, const void* b, void* x,
                        void* stream);
/* r_coarse = P^T r_fine between level `fine_level` and fine_level-1
 * (transpose of the canonical embedding, Sec. 3). */
sipg_status sipg_restrict(sipg_handle* h, int fine_level, int prec, const void* r_fine,
                          void* r_coarse, void* stream);
/* x_fine += P e_coarse (canonical embedding, Sec. 3). */
sipg_status sipg_prolongate_add(sipg_handle* h, int fine_level, int prec, const void* e_coarse,
                                void* x_fine, void* stream);
/* x0 = A_0^{-1} b0 on the coarsest level, exact, FP64 arithmetic (global fast
 * diagonalisation); prec selects the vector type. */
sipg_status sipg_coarse_solve(sipg_handle* h, int prec, const void* b0, void* x0, void* stream);
/* x = P_L^{-1} b: one V-cycle from x = 0 (Sec. 3), 1 pre- and 1
 * post-smoothing step (post-smoothing visits the colours in reverse).
 * prec = vector type of b and x; with SIPG_FP32 the whole V-cycle except the
 * coarse solve runs in FP32. */
sipg_status sipg_vcycle(sipg_handle* h, int prec, const void* b, void* x, void* stream);

/* Flexible CG on the finest level with the V-cycle (params.vcycle_precision)
 * as preconditioner, until ||b - A x||_2 <= rtol ||b||_2 for every column or
 * maxit iterations.  b, x: FP64, nrhs columns; x holds the initial guess on
 * entry and the solution on exit.  info may be NULL.  Synchronises stream. */
sipg_status sipg_solve(sipg_handle* h, const double* b, double* x, double rtol, int maxit,
                       sipg_info* info, void* stream);
/* sipg_solve from the initial guess x = 0: x is output only (its contents on
 * entry are ignored and overwritten).  The first residual is then b itself,
 * so the first true-residual operator apply of sipg_solve is skipped; the
 * final true residual b - A x is still verified.  Same iterates as sipg_solve
 * with x zeroed on entry.  Synchronises stream. */
sipg_status sipg_solve_zero(sipg_handle* h, const double* b, double* x, double rtol, int maxit,
                            sipg_info* info, void* stream);
/* Adjoint solve A^T lambda = g.  The SIPG matrix is symmetric, so this is
 * the same MG-preconditioned FCG applied to g. */
sipg_status sipg_adjoint_solve(sipg_handle* h, const double* g, double* lambda, double rtol,
                               int maxit, sipg_info* info, void* stream);
/* Same as sipg_solve with HOST buffers f (nodal source, FP64, nrhs columns)
 * and u (solution): copies f in, forms b = M_h f, solves from x = 0 on
 * `stream`, and copies u out on a second stream of its own as soon as the
 * iteration ends, beside the final true residual (a restart waits for that
 * copy and the final x is copied again).  Synchronises both. */
sipg_status sipg_solve_host(sipg_handle* h, const double* f_host, double* u_host, double rtol,
                            int maxit, sipg_info* info, void* stream);

/* Largest GMRES restart length (Krylov vectors kept per cycle). */
#define SIPG_GMRES_MAX_RESTART 64

/* Device bytes that sipg_gmres_solve needs for restart length `restart`
 * (1..SIPG_GMRES_MAX_RESTART): restart+1 Arnoldi vectors, restart
 * preconditioned vectors (FP64, finest level, one right-hand side each) and
 * reduction scratch.  0 for a bad argument.  No GPU needed. */
size_t sipg_gmres_workspace_bytes(const sipg_handle* h, int restart);
/* GMRES, the paper's outer solver (Sec. 3.3, Tables 1 and 2), on the finest
 * level, preconditioned from the right by one V-cycle (params.vcycle_precision)
 * in flexible form: the preconditioned directions are stored, so the FP32
 * V-cycle may serve as preconditioner.  Arnoldi with classical Gram-Schmidt
 * applied twice; plane rotations give ||b - A x||_2 after every step; a cycle
 * ends after `restart` steps or at ||b - A x||_2 <= rtol ||b||_2, then x is
 * updated and the true residual recomputed (it ends the history of the
 * cycle); the solve stops once that is <= rtol ||b||_2 or after maxit steps,
 * else restarts from x.  With params.smoother = SIPG_SMOOTHER_PAPER this is
 * the setting of Table 2 (Dirichlet kernel).  b, x: FP64, one column (nrhs
 * must be 1, else SIPG_EUNSUPPORTED); x holds the initial guess on entry.
 * work: caller-owned device memory of at least
 * sipg_gmres_workspace_bytes(h, restart) bytes, 256-byte aligned, not shared
 * with any other argument.  info->iterations counts GMRES steps (V-cycles);
 * info->nu is computed from the history as for sipg_solve.  Returns
 * SIPG_ENOCONV after maxit steps, SIPG_EBREAKDOWN on a non-finite scalar.
 * Synchronises stream.  With params.use_graphs = 1 each restart cycle runs
 * on the device as one CUDA graph launch (a conditional while node over the
 * Arnoldi step; Hessenberg matrix, rotations and stopping test in device
 * memory), so the host synchronises once per cycle; the graph is recorded
 * on the first call for a given work pointer, restart length and side of
 * preconditioning.  Otherwise the host drives every step and synchronises
 * after each. */
sipg_status sipg_gmres_solve(sipg_handle* h, const double* b, double* x, double rtol, int maxit,
                             int restart, void* work, size_t work_bytes, sipg_info* info, void* stream);
/* The same GMRES preconditioned from the left: Arnoldi on B A, the residual
 * (history, nu and the stopping test ||B (b - A x)||_2 <= rtol ||B b||_2) is
 * the one after the V-cycle, and x is updated from the Arnoldi vectors.  The
 * reading of the paper's Table 2 clamped-kernel column (Sec. 3.3).  Same
 * arguments, workspace and errors as sipg_gmres_solve; B must be a fixed
 * linear operator (every V-cycle of one handle is). */
sipg_status sipg_gmres_solve_left(sipg_handle* h, const double* b, double* x, double rtol, int maxit,
                                  int restart, void* work, size_t work_bytes, sipg_info* info, void* stream);

/* out[r] = <a_r, b_r> for every column r (FP64, deterministic order),
 * written to device memory. */
sipg_status sipg_dot(sipg_handle* h, const double* a, const double* b, double* out, void* stream);

/* Autotuned launch choices of one level (no counterpart in the paper: a
 * property of this implementation).  sipg_bind_workspace times, per level and
 * for the V-cycle precision, every launch path of one smoothing step on the
 * level's scratch vectors and keeps the fastest; this reports the choice.
 * *path: -1 not tuned (default rules), 0 one fused launch per step, 1 colour
 * by colour.  *tile: interior tile of the 3D FP32 colour pass (0..4, as
 * SIPG_TILE above).  precision: SIPG_FP64 or SIPG_FP32.
 * EINVAL for a bad level or precision or null outputs. */
sipg_status sipg_tuning(const sipg_handle* h, int level, int precision, int* path, int* tile);

/* ---- ragged batch: independent problems (any dim, degree, size) solved
 * together.  Each member is a full handle (its own levels, workspace slice,
 * CUDA graph); sipg_batch_solve advances all members' flexible CG iterations
 * in lockstep, each on its own internal stream joined to `stream` by events,
 * so the members' kernels overlap on the GPU and the host waits once per
 * round.  Members converge independently. */
typedef struct sipg_batch sipg_batch;
sipg_status sipg_batch_create(const sipg_params* params, int count, sipg_batch** out);
void sipg_batch_destroy(sipg_batch* b);
const char* sipg_batch_last_error(const sipg_batch* b);
int sipg_batch_count(const sipg_batch* b);
/* Member i (owned by the batch): use it for sipg_ndofs, sipg_rhs, ... */
sipg_handle* sipg_batch_member(sipg_batch* b, int i);
/* Sum of the members' workspaces (each 256-byte aligned inside); with
 * SIPG_BATCH_FUSED=1 and a batch of 2D problems with the FP32 V-cycle, one
 * right-hand side each, degrees 2..6, a Dirichlet-kernel smoother and the
 * 2 x 2 coarsest level, also the plan of the batched smoothing stages
 * (sipg_batch_solve). */
size_t sipg_batch_workspace_bytes(const sipg_batch* b);
/* Bind one caller-owned buffer for all members (runs every member's setup). */
sipg_status sipg_batch_bind_workspace(sipg_batch* b, void* dev_ptr, size_t bytes, void* stream);
/* b[i], x[i]: device vectors of member i (host arrays of count pointers);
 * x[i] holds the initial guess on entry.  infos: NULL or count entries.
 * Returns the first member failure (sipg_batch_last_error names it).
 * Synchronises the internal streams.  Batches of 2D FP32 problems (see
 * sipg_batch_workspace_bytes) run the flexible CG of all members in lockstep
 * with one V-cycle of the whole batch per iteration: every smoothing step of a
 * level is one cooperative launch over all members that have that level (all
 * colours, bounded grid barriers between them), the per-member work (zeroing,
 * residual and restriction, coarse solve, prolongation, Krylov updates) runs
 * on the members' streams, and each iteration is one CUDA graph; every
 * member's final true residual is verified (restarting that member alone if
 * it drifted).  That fused path is selected by SIPG_BATCH_FUSED=1 in the
 * environment at sipg_batch_create; by default every member runs on its own
 * stream with its own V-cycles and CUDA graph (faster on GB300: the members'
 * kernels overlap across members and levels). */
sipg_status sipg_batch_solve(sipg_batch* b, const double* const* bvecs, double* const* xvecs, double rtol,
                             int maxit, sipg_info* infos, void* stream);

/* Same result as sipg_dot, for callers that cannot allocate device memory
 * (an application whose allocator already holds all of it, or a latency path
 * where cudaMalloc would synchronise the device): needs a created handle (for
 * sizes and error messages) but no bound workspace, and allocates nothing.
 * Its reduction scratch is a fixed 128 KiB device array inside the library
 * (kept on every GPU that loads it until exit), so at most 64 columns are
 * supported (nrhs > 64 -> SIPG_EINVAL).  All calls share that array: calls
 * whose kernels overlap on the GPU race.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress); make it before any
 * stream capture.  The paper has no counterpart to this call. */
sipg_status sipg_dot_noalloc(sipg_handle* h, const double* a, const double* b, double* out,
                             void* stream);

/* Self-test of the tensor-core path (no counterpart in the paper): one CTA
 * computes D = A B^T with A 256 x 16 and B 16 x 16 (row-major FP32 device
 * arrays, rounded to TF32, FP32 accumulation) through the same operand
 * layouts, MMA issue, completion wait and tensor-memory loads as the TF32
 * colour pass, and writes D (256 x 16, row-major).  Needs a bound workspace
 * (for the status word); SIPG_ETIMEOUT if the bounded completion wait ran
 * out.  Synchronises stream. */
sipg_status sipg_selftest_mma_tf32(sipg_handle* h, const float* a, const float* b, float* d, void* stream);
/* Self test of the bounded device-side waits (fused smoothing steps separate
 * their colours by a grid barrier whose waits give up after about half a
 * second, set a status word and return, so a stuck barrier is reported as
 * SIPG_ETIMEOUT instead of hanging the GPU).  Launches two cooperative CTAs
 * on a barrier that expects `extra` more CTAs: extra = 0 must pass
 * (SIPG_OK); extra > 0 can never open, so both waits must run out and the
 * call returns SIPG_ETIMEOUT.  Resets the barrier state.  Synchronises stream.
 * The paper has no counterpart to this call. */
sipg_status sipg_selftest_barrier(sipg_handle* h, int extra, void* stream);

/* Copy FP64 level constants to host memory for inspection.  which:
 *  0 Lself (3 x n x n), 1 neighbour blocks [l_lo, l_hi] (2 x n x n),
 *  2 cell mass (n x n), 3 patch eigenvectors S of type t (p x p),
 *  4 patch eigenvalues of type t (p), 5 transfer [P_0, P_1] (2 x n x n),
 *  6 coarse eigenvectors (m0 x m0), 7 coarse eigenvalues (m0),
 *  8 Gauss-Lobatto nodes (n).  `type` is the patch type for 3/4 (bit 0: low
 * end on the boundary, bit 1: high end).  Writes at most cap doubles; returns
 * the count in *count.  Synchronises stream. */
sipg_status sipg_get_constants(sipg_handle* h, int level, int which, int type, double* host_out,
                               int cap, int* count, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SIPG_H */
