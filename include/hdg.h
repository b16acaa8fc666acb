/*
 * hdg.h - C ABI of the GB300 HDG trace solver for the implicit, linearised,
 * rotating shallow-water step
 *
 *      u + tau (f u_perp + g grad h) = r_u,      h + tau H div u = r_h,
 *
 * discretised with the upwind hybridised DG method of Betteridge, Gibson,
 * Graham & Mueller, "Multigrid preconditioners for the hybridised
 * discontinuous Galerkin discretisation of the shallow water equations"
 * (arXiv 2004.09389): cell fields u in [P^p(K)]^2, h in P^p(K), a scalar
 * trace lambda in P^p(e) on every facet (Eq. DG_space_def, Eq. DG_trace_def),
 * the upwind HDG form of Eq. bilinear_HDG_upwind written with tau for
 * alpha*Delta t, g for c_g*phi_B, H for c_g and tau_s = sqrt(g H) for
 * c_g*sqrt(phi_B), plus the Coriolis term taken implicitly.
 *
 * A solve is the three steps of Sec. 4.2: condensed right-hand side
 * (step 1), the trace system S lambda = g (Eq. schur_system, step 2, solved by
 * FGMRES preconditioned with the non-nested two-level V-cycle of
 * Alg. twolevel_vcycle whose coarse space is P1, Sec. 4.4), and local
 * recovery of (u, h) (Eq. reconstruct_solution, step 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh: triangles, cell_vertices counter-clockwise (seen from outside on the
 *   sphere).  Flat periodic meshes (dim = 2) give wrapped vertex coordinates
 *   plus cell_shift[K][i][2] offsets that unwrap vertex i of cell K.  Sphere
 *   meshes (dim = 3) give 3-D vertices; every cell is the flat triangle
 *   through its vertices.
 * Cell unknowns: n_p = (p+1)(p+2)/2 Lagrange nodes per cell; node k runs row
 *   by row (b = 0..p outer, a = 0..p-b inner) at X0 + (a/p)(X1-X0) +
 *   (b/p)(X2-X0).  Velocities are Cartesian (flat) or in the cell frame
 *   e1 = (X1-X0)/|X1-X0|, e2 = n x e1 (sphere).
 *   r_u, u: double [n_cells][2][n_p];  r_h, h: double [n_cells][n_p]
 *   (nodal values of the right-hand-side functions / of the solution).
 * Facets: numbered in order of first appearance over (cell, local edge),
 *   local edge i being opposite local vertex i.  The p+1 trace nodes of a
 *   facet are equispaced, endpoints included, from its lower global vertex id
 *   to the higher.  lambda: double [n_facets][p+1].
 *
 * Ownership and errors: the caller owns every buffer it passes; the library
 * copies what it keeps.  The handle owns its device memory.  Every function
 * returns HDG_OK (0) or a negative HDG_E* code; hdg_last_error() describes
 * the last failure on a handle.  A handle must not be used by two host
 * threads at once.  A handle belongs to the CUDA device that was current at
 * hdg_setup: make that device current for every call on it; a device reset
 * invalidates every handle on that device.  Host-pointer entry points copy to and from the device
 * and synchronise; *_dev entry points take device pointers, run on the
 * handle's stream and return once the work is enqueued (they synchronise only
 * where a result decides the control flow, e.g. the convergence test).
 */
#ifndef HDG_H
#define HDG_H

#include <stdint.h>

#if defined(__GNUC__)
#define HDG_API __attribute__((visibility("default")))
#else
#define HDG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define HDG_OK          0
#define HDG_EINVAL     -1   /* bad argument: sizes, p outside 1..4, tau <= 0, mesh not closed ... */
#define HDG_ESINGULAR  -2   /* a zero pivot in a cell or facet block factorisation            */
#define HDG_ENOCONV    -3   /* max_iter reached; lambda holds the last iterate                */
#define HDG_EBREAKDOWN -4   /* Krylov breakdown without convergence                           */
#define HDG_ENAN       -5   /* NaN or Inf met in the iteration or the input                   */
#define HDG_ECUDA      -6   /* a CUDA runtime call failed                                     */
#define HDG_ETIMEOUT   -7   /* a bounded device-side wait ran out                             */
#define HDG_ENOMEM     -8   /* device allocation failed                                       */
#define HDG_ESTATE     -9   /* call out of order (e.g. solve before condense)                 */

#define HDG_FP64        0   /* every step in double precision                                 */
#define HDG_MIXED_FP32  1   /* FP32 inner FGMRES + V-cycle, iterative refinement with the
                               residual, right-hand side, iterate and recovery in two-float
                               arithmetic (about 48 bits); lambda returned in FP64         */
#define HDG_MIXED_BF16  2   /* as HDG_MIXED_FP32, with a BF16 copy of the trace operator for the
                               smoother and V-cycle residual (FP32 accumulation)              */
#define HDG_MIXED_FGMRES64 3 /* FP64 FGMRES (basis, orthogonalisation, residual, update, RHS and
                               recovery in FP64) preconditioned by the two-level V-cycle in FP32
                               (FP32 operator copies; the coarsest P1 solve stays FP64)       */

typedef struct hdg_handle hdg_handle;

/* One mesh level.  For coarse P1 levels, parent[i] = (a, b) says that vertex i
 * of the next finer level lies at the midpoint of this level's vertices a and
 * b (a == b: the vertex exists on both levels).  parent is ignored on the
 * fine level. */
typedef struct {
    int32_t        n_vertices;
    int32_t        n_cells;
    int32_t        dim;            /* 2: flat periodic, 3: sphere                   */
    const double  *vertex_xyz;     /* [n_vertices][dim]                              */
    const int32_t *cell_vertices;  /* [n_cells][3]                                   */
    const double  *cell_shift;     /* [n_cells][3][2] (dim 2) or NULL                */
    const int32_t *parent;         /* [n_vertices of next finer level][2] or NULL    */
} hdg_mesh_level;

typedef struct {
    hdg_mesh_level        fine;
    int32_t               n_coarse;   /* number of coarse P1 levels (0: P1 on the fine mesh only) */
    const hdg_mesh_level *coarse;     /* [n_coarse], next-coarser first                         */
} hdg_mesh_desc;

typedef struct {
    int32_t       p;            /* polynomial degree, 1..4                               */
    double        tau;          /* alpha * Delta t > 0                                   */
    double        g, H;         /* gravity and mean depth (> 0)                          */
    double        tau_s;        /* upwind stabilisation; <= 0 selects sqrt(g H)          */
    const double *f_vertex;     /* Coriolis parameter at fine vertices, P1 per cell; NULL = 0 */
    int32_t       precision;    /* HDG_FP64, HDG_MIXED_FP32, HDG_MIXED_BF16 or HDG_MIXED_FGMRES64 */
    double        rtol;         /* stop at ||g - S lambda|| <= rtol ||g|| (FP64 residual) */
    int32_t       restart;      /* FGMRES restart length m (1..64)                        */
    int32_t       max_iter;     /* total Krylov iterations allowed                        */
    int32_t       n_pre, n_post;/* block-Jacobi sweeps before / after the coarse correction */
    double        omega;        /* block-Jacobi damping                                   */
    int32_t       p1_nu_pre, p1_nu_post; /* Jacobi sweeps per level of the P1 V-cycle     */
    double        p1_omega;     /* Jacobi damping of the P1 V-cycle                       */
    double        inner_rtol;   /* mixed modes: relative tolerance of each inner solve   */
    int32_t       coarse_mode;  /* P1 coarse operator (Sec. 4.4 recipe: eliminate u from the
                                   time-implicit continuum equations, divided by tau):
                                   0 = with the implicit Coriolis term, per cell
                                       (phi,psi) + tau^2 g H kappa_K [(grad phi,grad psi)
                                       - tau f_K (J grad phi,grad psi)], kappa_K = 1/(1+tau^2 f_K^2);
                                   1 = as printed in Eq. coarse_problem_upwind (no rotation).
                                   Both agree when f = 0.
                                   2 = the Galerkin choice of the Sec. 4.4 footnote:
                                       pi^T S pi on the fine P1 level, P^T A P on the
                                       coarser ones (P linear interpolation)             */
    int32_t       reorth;       /* Arnoldi orthogonalisation (GMRES, Sec. 5.1 setup):
                                   0 = one classical Gram-Schmidt pass (the solver
                                       configuration of the paper's experiments sets no
                                       orthogonalisation option, i.e. the library default
                                       of classical Gram-Schmidt without refinement);
                                   1 = classical Gram-Schmidt twice (CGS2).              */
    int32_t       smoother;     /* facet smoother of Alg. twolevel_vcycle (lines 1 and 6):
                                   0 = damped block-Jacobi (omega);
                                   1 = Chebyshev iteration preconditioned by block-Jacobi
                                       (the paper's smoother is a Chebyshev iteration,
                                       Sec. 5.2.1), tuned to an ellipse around the spectrum
                                       of D^-1 S: stays contractive under strong rotation  */
    double        cheb_theta;   /* smoother 1: ellipse centre; <= 0 selects the estimate
                                   made at condensation (Arnoldi on D^-1 S)               */
    double        cheb_delta2;  /* smoother 1: squared focal half-distance of the ellipse
                                   (used only when cheb_theta > 0; < 0 for a tall ellipse) */
    int32_t       cheb_steps;   /* smoother 1: Arnoldi steps of the estimate (2..64)      */
    int32_t       flux;         /* 0 = upwind (Eq. bilinear_HDG_upwind: scalar trace, P1 coarse
                                       space);
                                   1 = Lax-Friedrichs (Eq. bilinear_HDG_lax: vector trace
                                       u_hat in [P^p(e)]^2, Cartesian components, 2(p+1) dofs
                                       per facet (component-major, nodes lo -> hi); RT0 coarse
                                       space with the grad-div operator of
                                       Eq. coarse_problem_LF divided by tau, solved
                                       approximately by n_coarse Chebyshev steps).  Flat
                                       meshes, HDG_FP64, p = 1 or 2, coarse_mode 0 or 1.   */
    int32_t       n_coarse;     /* flux 1: Chebyshev steps of the RT0 coarse solve (1..200) */
    int32_t       keep_rhs;     /* HDG_MIXED_FP32 / HDG_MIXED_BF16, upwind flux: 1 (default) =
                                   each solve's step 1 keeps z_K = A_K^-1 M_K r_K for a
                                   recovery with NULL right-hand sides and forms C_K z_K
                                   from the cell geometry (step 1 reads A_K^-1 M_K instead
                                   of C_K A_K^-1 M_K: more bytes there, far fewer in step 3);
                                   0 = step 1 reads C_K A_K^-1 M_K and keeps nothing (for
                                   solves that are not followed by a recovery)           */
} hdg_params;

typedef struct {
    int32_t iters;            /* Krylov iterations (inner iterations in mixed mode)    */
    int32_t outer;            /* restarts (FP64) / refinement steps (mixed)            */
    int32_t status;           /* same code as the return value                         */
    int32_t fallback_used;    /* reserved: 1 if a fallback preconditioner took over    */
    double  true_rel_res;     /* ||g - S lambda|| / ||g|| in FP64 at exit              */
    double  est_rel_res;      /* last Arnoldi residual estimate                        */
} hdg_solve_info;

/* Fill *prm with the defaults: p = 1, tau = 1, g = H = 1, tau_s = sqrt(gH),
 * FP64, rtol 1e-8, restart 30, max_iter 500, 2 + 2 sweeps, omega = 2/3,
 * 2 + 2 P1 sweeps, p1_omega = 2/3, inner_rtol 1e-4, coarse_mode 0, reorth 0,
 * smoother 0 (cheb_theta 0: estimated, cheb_steps 20), flux 0, n_coarse 20. */
HDG_API void hdg_default_params(hdg_params *prm);

/* Build a handle: validate and copy the mesh (facet numbering, orientation,
 * cell frames, P1 hierarchy and its geometric mass / stiffness matrices) to
 * the device.  stream: a cudaStream_t to run on, or NULL for a new
 * non-blocking stream owned by the handle.  On failure *out is NULL and the
 * error text is available from hdg_last_error(NULL).
 * Two environment variables, read here, select equivalent launch structures
 * (for timing comparisons; results agree up to summation order):
 * HDG_TAIL_MAX_VERTICES (16..4096; default 1024 for the FP32 levels, 256 for
 * the FP64 levels) bounds the P1 levels run by the single-block coarse cycle; HDG_P1_FUSED=0 replaces the patch-fused P1
 * kernels by one launch per smoothing / transfer step; HDG_FACET_BLOCK
 * (64, 128 or 256; default 128 for HDG_FP64 handles, 256 otherwise) sets the
 * threads per block of the facet-row kernels.  HDG_PDL (a bit mask, read once
 * per process; default 6) selects the kernel families launched with
 * programmatic dependent launch, so that a kernel's blocks are scheduled
 * while its predecessor drains: 1 the facet-row kernels, 2 the P1 kernels,
 * 4 the Krylov kernels; 0 none.  HDG_SPECULATE (read once per process) lets
 * an FGMRES cycle queue Arnoldi step j + 1 behind step j before step j's
 * residual estimate has reached the host, when the last two estimates,
 * extrapolated geometrically, put step j's above the margin times the target:
 * unset = margin 8, a number > 1 = that margin, 0 = off.  A step queued ahead
 * whose predecessor meets the target runs for nothing and is not used. */
HDG_API int hdg_setup(const hdg_mesh_desc *mesh, const hdg_params *prm, void *stream, hdg_handle **out);

/* (Re)build the cell operators for the handle's parameters: for every cell the
 * local blocks A_K, B_K, C_K and tau_s M_dK of the ABCM split (Eq. ABCMform,
 * App. B), A_K^-1 B_K, A_K^-1 M_K, S_K = tau_s M_dK + C_K A_K^-1 B_K and
 * C_K A_K^-1 M_K; then the facet-row trace operator (the S_K summed onto the
 * facets), the inverted facet diagonal blocks of the block-Jacobi smoother and
 * the P1 level operators (Eq. coarse_problem_upwind, divided by tau).
 * FP64 handles eliminate in FP64.  Handles in HDG_MIXED_FP32 / HDG_MIXED_BF16,
 * which use these matrices only as two-float pairs, invert A_K in FP32 and
 * refine A_K^-1 [B_K | M_K] twice with two-float residuals (about 48-bit
 * results, written directly as the pairs); the environment variable
 * HDG_CONDENSE_FP64=1 (read once per process) gives them the FP64
 * elimination too.  A coarsest P1 level of more than 256 vertices is inverted
 * by one pivot and one update launch per column.
 * HDG_ESINGULAR if a cell or facet block has a zero pivot. */
HDG_API int hdg_condense(hdg_handle *h);

/* Change tau (and with it the operators); equivalent to a new hdg_condense. */
HDG_API int hdg_set_tau(hdg_handle *h, double tau);

/* Steps 1 and 2 with host buffers: r_u, r_h in, lambda out ([n_facets][p+1]).
 * info may be NULL.  Returns HDG_ENOCONV / HDG_EBREAKDOWN / HDG_ENAN with the
 * last iterate in lambda.  Step 2 (Sec. 4.2) is driven from the calling
 * thread: after each Arnoldi step it spins on a word the GPU writes to
 * page-locked memory (the residual estimate decides whether to go on), so the
 * calling thread keeps one CPU core busy for the length of the solve; the same
 * holds for hdg_solve_dev and each thread of hdg_solve_batch_dev. */
HDG_API int hdg_solve(hdg_handle *h, const double *r_u, const double *r_h, double *lambda,
              hdg_solve_info *info);
/* The same with device pointers. */
HDG_API int hdg_solve_dev(hdg_handle *h, const double *r_u, const double *r_h, double *lambda,
                  hdg_solve_info *info);

/* Steps 1 to 3 with host buffers in one call (Sec. 4.2): hdg_solve, then the
 * recovery of its solution (hdg_recover with NULL lambda and right-hand
 * sides), with one stream synchronisation at the end instead of one per call.
 * lambda ([n_facets][p+1]), u and h_out receive the results, info may be NULL.
 * Returns the solve's status when it is not HDG_OK (HDG_ENOCONV / HDG_EBREAKDOWN
 * / HDG_ENAN with the last iterate and its recovery), else the recovery's. */
HDG_API int hdg_solve_recover(hdg_handle *h, const double *r_u, const double *r_h, double *lambda, double *u,
                              double *h_out, hdg_solve_info *info);

/* Step 3 with host buffers: (u, h) from lambda and the right-hand side.
 * lambda may be NULL to use the handle's last solution; r_u and r_h may both
 * be NULL to use the right-hand side of the handle's last hdg_solve (one NULL
 * and one not: HDG_EINVAL).  Explicit inputs serve this call only: a later
 * call with NULLs still selects the last solve's data. */
HDG_API int hdg_recover(hdg_handle *h, const double *r_u, const double *r_h, const double *lambda,
                double *u, double *h_out);
/* The same with device pointers on the handle's stream: u and h_out are
 * required (HDG_EINVAL if NULL); lambda may be NULL to use the handle's last
 * solution; r_u and r_h may both be NULL to use the last solve's right-hand
 * side (one NULL and one not: HDG_EINVAL).  With NULL right-hand sides a
 * HDG_MIXED_FP32 / HDG_MIXED_BF16 handle reads what the last solve's step 1
 * kept of it, z_K = A_K^-1 M_K r_K per cell (two-float pairs), and forms
 * q_K = z_K - A_K^-1 B_K lambda_K: the recovery then reads no right-hand side
 * and no A_K^-1 M_K (Eq. reconstruct_solution split at the solve's step 1).
 * Other handles use the copies hdg_solve keeps; HDG_ESTATE if there is nothing
 * kept (no solve yet, or the operator changed since, by hdg_condense or
 * hdg_set_tau).  Results are complete once the stream has been synchronised. */
HDG_API int hdg_recover_dev(hdg_handle *h, const double *r_u, const double *r_h, const double *lambda,
                    double *u, double *h_out);

/* Many independent solves at once: handle i solves r_u[i], r_h[i] into
 * lambda[i] (device pointers), as hdg_solve_dev would, while the others run
 * concurrently on their own streams (the handles must be distinct and have
 * distinct streams).  n_threads host threads (<= 0: up to 16) drive the
 * solves; every Arnoldi step is a replayed CUDA graph.  infos (may be NULL)
 * gets one entry per handle; the return value is the first non-OK status in
 * handle order.  Like hdg_solve_dev, results are complete once each handle's
 * stream has been synchronised.  (Batching beyond the paper, which solves one
 * system at a time.) */
HDG_API int hdg_solve_batch_dev(hdg_handle *const *hs, int n, const double *const *r_u, const double *const *r_h,
                                double *const *lambda, hdg_solve_info *infos, int n_threads);

/* Merged batched solves: one host thread drives n independent solves whose
 * kernels run as merged launches.  Every problem follows exactly the steps of
 * hdg_solve_dev (the same kernels with the same arguments, so the same
 * results bit for bit); the launches that the problems issue between two
 * decisions of their host logic (a residual estimate or a norm read back)
 * form one wave.  Within a wave, the launches of different problems that run
 * the same kernel with the same block size become one launch whose blocks
 * cover all of them (at most 64 problems per launch; each problem's
 * arguments travel in the kernel's parameter block), ordered as a DAG of
 * per-problem chains and run as a CUDA graph; a graph is kept and replayed
 * whenever the same wave recurs (same kernels, shapes and arguments).  The
 * number of launches per wave therefore depends on the kernels in play (the
 * degrees, the coarse-level structures), not on the number of problems.
 *
 * hdg_batch_create checks and records the handles (n >= 1, distinct, on the
 * current device, condensed; upwind flux; precision HDG_MIXED_FP32 or
 * HDG_MIXED_BF16; reorth = 0): HDG_EINVAL / HDG_ESTATE otherwise, with the
 * reason in hdg_last_error(NULL).  hdg_batch_solve_dev solves r_u[i], r_h[i]
 * (device pointers) into lambda[i] for every handle i, on a stream of the
 * batch ordered after each handle's stream, and each handle's stream is
 * ordered after the batch on return (the host also waits for the last wave,
 * so the results are complete on return).  The handles must not be used
 * elsewhere during the call, kernel timing (hdg_profile_enable) must be off
 * and the learned smoother not enabled (HDG_ESTATE).  infos (may be NULL) gets
 * one entry per handle; the return value is the first non-OK status in handle
 * order, with its message in hdg_last_error(NULL).  hdg_batch_stats fills
 * stats[0..7] = waves, merged launches, per-problem launches they carried,
 * graphs replayed, graphs built, and host nanoseconds spent running the
 * problems' host logic, merging and launching waves, and waiting for the
 * last waves (totals since creation).  hdg_batch_destroy(NULL) is a no-op;
 * destroy the batch before its handles.
 *
 * The problems are split into groups, each with its own stream, waves and
 * graphs: while one group's wave runs, the host prepares another's, and the
 * groups' launches fill each other's gaps on the GPU.  HDG_BATCH_GROUPS = G
 * (1..64, default 4) sorts the problems by size (trace unknowns) and cuts
 * them into G contiguous size classes of about equal total size, so that a
 * merged launch covers problems of similar size (HDG_BATCH_DEAL=rr deals them
 * round robin instead); 0 groups them by degree. */
typedef struct hdg_batch hdg_batch;
HDG_API int hdg_batch_create(hdg_handle *const *hs, int n, hdg_batch **out);
HDG_API int hdg_batch_solve_dev(hdg_batch *b, const double *const *r_u, const double *const *r_h,
                                double *const *lambda, hdg_solve_info *infos);
/* The same with host buffers (r_u[i], r_h[i] in, lambda[i] out, layouts as for
 * hdg_solve): the right-hand sides are copied to each handle's staging buffers
 * on its stream, the merged solve runs on them, and lambda is copied back
 * before the call returns; hdg_recover with NULL right-hand sides then uses
 * this solve's.  Return values as hdg_batch_solve_dev. */
HDG_API int hdg_batch_solve(hdg_batch *b, const double *const *r_u, const double *const *r_h, double *const *lambda,
                            hdg_solve_info *infos);
HDG_API int hdg_batch_stats(const hdg_batch *b, int64_t *stats);
HDG_API int hdg_batch_destroy(hdg_batch *b);

/* Pick launch shapes for this handle by timing one Arnoldi step (preconditioner,
 * operator application, Gram-Schmidt) for each candidate: threads per block of
 * the facet-row kernels (64 / 128 / 256), blocks of the fused Gram-Schmidt
 * kernels (152 / 304 / 608 / 1216) and the largest level of the single-CTA coarse
 * cycle (256 / 1024 / 4096 vertices), one parameter at a time.  Needs
 * hdg_condense.  choice[0..2] (may be NULL) receives the three picks.  Results
 * do not depend on the choice beyond floating-point summation order. */
HDG_API int hdg_autotune(hdg_handle *h, int32_t *choice);

/* Operator entry points on device vectors in the lambda layout [n_facets][p+1]. */
/* y = S x, S the assembled trace operator of Eq. schur_system. */
HDG_API int hdg_trace_apply_dev(hdg_handle *h, const double *x, double *y);
/* g = sum_K P_K^T C_K A_K^-1 F_K, the condensed right-hand side of step 1. */
HDG_API int hdg_condensed_rhs_dev(hdg_handle *h, const double *r_u, const double *r_h, double *g);
/* Same result as hdg_condensed_rhs_dev, for callers that must not cause any
 * device allocation once their handles exist: an application that hands all
 * device memory to its own pool at start-up (a late allocation by a library
 * would fail or force the pool to give memory back), or one that cannot
 * afford the device-wide synchronisation that cudaMalloc / cudaFree may
 * impose on its other streams.  The paper has no counterpart: this is an
 * engineering variant.  Its scratch is a fixed 32 MiB array (2^22 doubles)
 * inside the library's device image, shared by every call on the device;
 * sizes needing more (n_cells * 3(p+1), rounded up to 32, plus
 * n_facets * (p+1) doubles) return HDG_EINVAL.  hdg_setup places the array on
 * the handle's device and looks up its device address there; from then on
 * the device keeps it until the process exits, and this call allocates
 * nothing: no cudaMalloc / cudaFree, no allocating library routine, no
 * module load.  The array keeps the last call's contents (nothing in it has
 * to start at zero: every entry a call reads, that call wrote first); calls
 * whose GPU work overlaps (two streams, two handles on one device) race on it
 * and must be serialised by the caller.  HDG_ESTATE before hdg_condense. */
HDG_API int hdg_condensed_rhs_noalloc_dev(hdg_handle *h, const double *r_u, const double *r_h, double *g);
/* z = V(v): one application of the two-level V-cycle (Alg. twolevel_vcycle)
 * with zero initial guess. */
HDG_API int hdg_precond_apply_dev(hdg_handle *h, const double *v, double *z);

/* z = V(v) in FP32 as used by the inner solves of the mixed modes (with the
 * learned sweep when it is enabled); v, z: FP32, lambda layout. */
HDG_API int hdg_precond_apply32_dev(hdg_handle *h, const float *v, float *z);

/* Inspection (host buffers) for checking against an independent code. */
/* sizes[0..5] = n_cells, n_facets, n_trace, n_p, 3(p+1), number of P1 levels. */
HDG_API int hdg_get_sizes(const hdg_handle *h, int64_t *sizes);
/* facet_of [n_cells][3], flip [n_cells][3] (1: local edge runs high -> low id),
 * facet_verts [n_facets][2] (lo, hi).  Any pointer may be NULL. */
HDG_API int hdg_get_facets(const hdg_handle *h, int32_t *facet_of, int32_t *flip, int32_t *facet_verts);
/* Per-cell S_K in the local trace order (edge i, node j along the edge from
 * local vertex (i+1)%3 to (i+2)%3), [n_cells][3(p+1)][3(p+1)].  Needs condense. */
HDG_API int hdg_get_cell_schur(hdg_handle *h, double *S);

/* The Chebyshev smoother's ellipse (smoother 1, after hdg_condense):
 * ellipse[0] = theta, ellipse[1] = delta^2.  The estimate runs cheb_steps
 * Arnoldi steps on D^-1 S (FP64 operator, classical Gram-Schmidt twice) from
 * the start vector v_i = 1 + ((37 i) mod 101) / 101, i the index in the
 * lambda layout; the ellipse spans [0.1 b, b] on the real axis with
 * b = 1.1 max Re(Ritz) and is 1.1 times as tall as needed to hold every Ritz
 * value in that range.  ritz (may be NULL) receives up to 64 Ritz values as
 * (re, im) pairs, *n_ritz their number (0 when the ellipse was given).
 * HDG_ESTATE if the handle does not use smoother 1 or is not condensed. */
HDG_API int hdg_get_chebyshev(const hdg_handle *h, double *ellipse, double *ritz, int32_t *n_ritz);
/* The same for the Chebyshev coarse solve of the Lax-Friedrichs solver
 * (flux 1): the ellipse of D_c^-1 S_c (S_c the RT0 coarse operator, D_c its
 * diagonal) fitted to cheb_steps Arnoldi Ritz values from the start vector
 * v_f = 1 + ((37 f) mod 101) / 101 over the facets.  HDG_ESTATE unless the
 * handle uses flux 1 and is condensed. */
HDG_API int hdg_get_rt0_chebyshev(const hdg_handle *h, double *ellipse, double *ritz, int32_t *n_ritz);

/* Kernel accounting.  Launch counts per category are always kept; with
 * timing enabled every launch is bracketed by CUDA events on the handle's
 * stream and the elapsed times are summed per category (read at the
 * library's own synchronisation points).  hdg_profile_enable resets both.
 * timing_on: 0 = counts only; 1 = event timing (caches as the solve leaves
 * them); 2 = event timing with the L2 cache evicted before every timed launch
 * (a buffer of three times the L2 size, allocated here, is read outside the
 * events), so each kernel's operands come from DRAM.  While timing is on the
 * Arnoldi steps run as direct launches instead of replayed graphs.
 * ms / launches: arrays of HDG_PROF_N entries (either may be NULL). */
#define HDG_PROF_APPLY64        0   /* y = S x, FP64                         */
#define HDG_PROF_RESIDUAL64     1   /* r = b - S x, FP64                     */
#define HDG_PROF_SMOOTH64       2   /* block-Jacobi sweep, FP64              */
#define HDG_PROF_SMOOTH_FIRST64 3   /* first sweep from zero, FP64           */
#define HDG_PROF_APPLY32        4
#define HDG_PROF_RESIDUAL32     5
#define HDG_PROF_SMOOTH32       6
#define HDG_PROF_SMOOTH_FIRST32 7
#define HDG_PROF_TRANSFER       8   /* trace <-> P1 restriction / prolongation */
#define HDG_PROF_P1             9   /* P1 V-cycle kernels                    */
#define HDG_PROF_KRYLOV        10   /* dots, updates, Givens, conversions    */
#define HDG_PROF_RHS           11   /* step 1                                */
#define HDG_PROF_RECOVER       12   /* step 3                                */
#define HDG_PROF_LAYOUT        13   /* lambda layout conversions             */
#define HDG_PROF_CONDENSE      14   /* condensation and assembly             */
#define HDG_PROF_IMEX          15   /* IMEX stage rates and combinations     */
#define HDG_PROF_N             16
HDG_API int hdg_profile_enable(hdg_handle *h, int timing_on);
HDG_API int hdg_profile_read(hdg_handle *h, double *ms, int64_t *launches);

/* Measured FMA throughput of this GPU in TFLOP/s (2 flops per FMA) for
 * bytes = 8 (FP64) or 4 (FP32): independent FMA chains on every SM of the
 * current device, timed by CUDA events (best of three launches).  The paper
 * has no counterpart; it is the arithmetic roof the FP64 kernels are measured
 * against.  HDG_EINVAL for other sizes. */
HDG_API int hdg_fma_rate(int bytes, double *tflops);

/* Learned facet-patch smoother (an extension beyond the paper, which has no learned
 * component).  In the FP32 inner solves of the mixed modes it replaces the last
 * post-smoothing sweep of the V-cycle by x += c(r), r = v - S x:
 *   X_e = (r_e, r of the four facets sharing a cell with e) / s_e, s_e their RMS,
 *   y_e = W3 tanh(W2 tanh(W1 X_e + b1) + b2) + b3 + omega X_e[0:p+1],
 *   c_e = D_e^-1 (s_e y_e)          (zero weights: the damped block-Jacobi sweep).
 * It is trained on the GPU by the library's own forward / backward kernels to
 * minimise mean ||r - S c(r)||^2 / ||r||^2 over residuals that the plain solver
 * produces before its last sweep.  While it is enabled, a solve whose residual
 * estimate drops by less than 10 % over three iterations switches back to the
 * plain V-cycle for the rest of that solve (hdg_solve_info.fallback_used = 1).
 * Parameters: theta = [W1 (hidden x 5(p+1)) | b1 | W2 | b2 | W3 ((p+1) x hidden) | b3], FP32. */
/* Allocate the network (hidden = 32 or 64), seed its weights, and room for
 * `capacity` training residuals.  Needs hdg_condense and a mixed mode. */
HDG_API int hdg_learned_init(hdg_handle *h, int hidden, int capacity, uint64_t seed, int32_t *n_params);
/* Run one plain solve (device pointers) and store the normalised residual seen
 * before the last post-smoothing sweep of every preconditioner call, up to the
 * capacity; *n_stored receives the number stored so far. */
HDG_API int hdg_learned_collect_dev(hdg_handle *h, const double *r_u, const double *r_h, int32_t *n_stored);
/* Adam on minibatches of stored residuals; losses of the first and last step. */
HDG_API int hdg_learned_train(hdg_handle *h, int steps, int batch, double lr, double *loss_first,
                              double *loss_last);
/* Copy the parameters out (get = 1) or in (get = 0), host buffer of n_params floats. */
HDG_API int hdg_learned_params(hdg_handle *h, float *theta, int get);
/* Use the learned sweep in later solves: 0 = off; 1 = FP32 network on the CUDA
 * cores; 2 = the network's three layers as tcgen05 GEMMs over tiles of 128 facets
 * (BF16 weights and activations, FP32 accumulation in tensor memory; the damped
 * block-Jacobi part, the scale and the D^-1 solve stay FP32). */
HDG_API int hdg_learned_enable(hdg_handle *h, int on);
/* Loss mean_i ||r_i - S c(r_i)||^2 / ||r_i||^2 and its gradient (host buffer of
 * n_params floats) for n residuals given on the device in the lambda layout
 * [n][n_facets][p+1] (FP32). */
HDG_API int hdg_learned_loss_grad_dev(hdg_handle *h, const float *R, int n, float *grad, double *loss);

/* IMEX time stepping around the solve (Sec. 3.3: Eq. theta_method and the
 * IMEX Runge-Kutta form of Eqs. IMEX_HDG_I / IMEX_HDG_II; the tableaux of
 * Sec. 5.1).  The semi-discrete system M dq/dt = N(q) + L(q) splits into the
 * gravity-wave terms with the upwind stabilisation, L (implicit), and the
 * Coriolis term, N (explicit, as in the paper):
 *   L_u(q).w = g (h, div w) - g <lambda, w.n>_dK,
 *   L_h(q) psi = -H (div u, psi) - tau_s <h - lambda, psi>_dK,
 *   N_u(q).w = -(f u_perp, w),  N_h = 0,
 * with lambda = {h} + H / (2 tau_s) (u_1.n_1 + u_2.n_2) on each facet (the
 * transmission condition solved pointwise).  An implicit stage
 * M Q - a_ii dt L(Q) = M r is this library's solve with f = 0 and
 * tau = a_ii dt (re-condensed by hdg_set_tau when tau changes) followed by
 * the recovery; explicit parts act through the inverse cell mass matrices on
 * nodal function values.  The handle must have been set up with
 * f_vertex = NULL (its implicit operator has no Coriolis term). */
#define HDG_IMEX_THETA 0   /* (M + theta dt K) q1 = M q0 + dt (N(q0) - (1 - theta) K q0), K = -L    */
#define HDG_IMEX_ARS2  1   /* ARS2(2,3,2): gamma = 1 - 1/sqrt(2), delta = -2 sqrt(2)/3, two solves     */
#define HDG_IMEX_SSP2  2   /* SSP2(3,2,2): three implicit stages with a_ii = 1/2                       */
#define HDG_IMEX_ARS3  3   /* ARS3(4,4,3): four implicit stages with a_ii = 1/2                        */
/* Store the Coriolis field of the explicit term (host array [n_vertices], P1
 * per cell like hdg_params.f_vertex; NULL: no rotation) and allocate the
 * stage buffers (3 + 10 state vectors of n_cells * 3 n_p doubles).
 * HDG_EINVAL if the handle was set up with a non-zero f_vertex. */
HDG_API int hdg_imex_init(hdg_handle *h, const double *f_vertex);
/* The stage rates of a state (device pointers, caller layouts u [N][2][n_p],
 * h [N][n_p]): (nu, nh) = M^-1 N(q) (both NULL to skip) and (lu, lh) =
 * M^-1 L(q), as nodal values.  Needs hdg_imex_init. */
HDG_API int hdg_imex_rates_dev(hdg_handle *h, const double *u, const double *hh, double *nu, double *nh,
                               double *lu, double *lh);
/* Advance (u, h) (device pointers, updated in place) by one step of length dt
 * of the scheme: for each stage i, r_i = q0 + dt sum_{j<i} (a_ij n~_j +
 * a~_ij l~_j); Q_i = q0 for an explicit first stage, the stage solve of r_i
 * where a~_ii != 0; then q1 = q0 + dt sum_i (b_i n~_i + b~_i l~_i), with
 * n~ = M^-1 N, l~ = M^-1 L.  theta is used by HDG_IMEX_THETA only (0 < theta
 * <= 1).  info (may be NULL) sums the stage solves' iterations and keeps the
 * largest residual; the return value is the first non-OK stage status (the
 * step is still completed unless it is HDG_ECUDA or HDG_ENAN).  Synchronises
 * once per stage solve (the convergence test). */
HDG_API int hdg_imex_step_dev(hdg_handle *h, int scheme, double theta, double dt, double *u, double *hh,
                              hdg_solve_info *info);

/* The CUDA stream (cudaStream_t) the handle runs on: the one given to
 * hdg_setup, or the non-blocking stream the handle created and owns. */
HDG_API void *hdg_get_stream(const hdg_handle *h);

HDG_API int hdg_destroy(hdg_handle *h);
HDG_API const char *hdg_last_error(const hdg_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* HDG_H */
