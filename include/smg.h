/*
 * smg.h -- C ABI of the GB300 surface multigrid library (libsmg.so).
 *
 * Method: Liu, Zhang, Ben-Chen, Jacobson, "Surface Multigrid via Intrinsic
 * Prolongation", ACM TOG 40(4), 2021.  Alg. 1 is the overall structure: the
 * hierarchy P_1..P_H is precomputed from the mesh (V, F) alone; the system
 * A x = b may change afterwards; V-cycles (Alg. 2) run until the error is
 * below a tolerance.  Fig. "fourSteps" is the reason for the split between
 * setup (geometry) and update (matrix) below.
 *
 * Conventions for every entry point
 *   - Return value: SMG_OK (0) or one of the SMG_ERR_* codes; no exception or
 *     longjmp ever crosses this boundary.  smg_last_error() gives a message
 *     for the most recent failure on the calling thread.
 *   - Host pointers are read during the call only and stay owned by the caller.
 *   - Device pointers (suffix _dev) are owned by the caller, must hold the
 *     documented number of elements, and are accessed in stream order on the
 *     `stream` argument (a cudaStream_t passed as void*; NULL = legacy default).
 *   - All floating-point arrays are IEEE binary64 unless stated otherwise.
 *   - Vectors indexed by "unknowns" are in ascending original vertex order,
 *     restricted to the vertices that are not Dirichlet-known.  Multi-RHS
 *     arrays are row-major n x nrhs (the nrhs values of one vertex adjacent).
 *   - A handle may be used by one host thread at a time.
 */
#ifndef SMG_H
#define SMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define SMG_OK                0
#define SMG_ERR_INVALID_ARG   1  /* null pointer, size or index out of range      */
#define SMG_ERR_NONMANIFOLD   2  /* mesh is not an oriented 2-manifold            */
#define SMG_ERR_DECIMATION    3  /* hierarchy could not be built                  */
#define SMG_ERR_NOT_SPD       4  /* a coarsest pivot was not positive             */
#define SMG_ERR_NOT_CONVERGED 5  /* max_cycles reached above rtol (x still valid) */
#define SMG_ERR_DIVERGED      6  /* residual became non-finite                    */
#define SMG_ERR_TIMEOUT       7  /* a bounded device wait gave up                 */
#define SMG_ERR_CUDA          8  /* a CUDA runtime call failed                    */
#define SMG_ERR_NO_MEMORY     9  /* host or device allocation failed              */
#define SMG_ERR_STATE        10  /* call out of order (e.g. solve before update)  */
#define SMG_ERR_IO           11  /* plan file could not be read or written        */

#define SMG_FP64  0   /* every cycle in binary64                                          */
#define SMG_MIXED 1   /* binary32 V-cycles inside binary64 iterative refinement; the
                         residual, the update and the coarsest Cholesky stay binary64 */

#define SMG_SMOOTHER_GS     0  /* multicolour Gauss-Seidel (Sec. 5, App. "Multi-Color Gauss Seidel") */
#define SMG_SMOOTHER_JACOBI 1  /* damped Jacobi x <- x + omega D^{-1} (b - A x), the alternative
                                  App. "Ablation Study" compares; two launches per sweep instead of
                                  one per colour class; the cluster tail is not used with it */

#define SMG_SOLVER_VCYCLE 0  /* Alg. 1: repeat V-cycles while the relative residual exceeds rtol */
#define SMG_SOLVER_PCG    1  /* conjugate gradients preconditioned by one V-cycle from a zero start
                                (Sec. "Limitations & Future Work"); the cycle is symmetric when
                                mu_pre == mu_post and post_reverse = 1 (the defaults).  CG vectors
                                and scalars are binary64; with SMG_MIXED the preconditioner cycle is
                                binary32.  smg_info.cycles counts CG iterations (one cycle each). */

typedef void *smg_stream;   /* a cudaStream_t */

/*
 * Options.  Defaults (smg_default_options) follow Sec. 5 and App. "Ablation":
 * Gauss-Seidel with mu_pre = mu_post = 2, coarsening ratio 0.25, coarsest level
 * no smaller than 500 vertices.
 *   min_coarse   paper rule: stop when the next level would have fewer vertices
 *   max_coarse   if > 0, replaces the rule above: coarsen while n > max_coarse
 *   max_levels   if > 0, at most this many levels (finest included)
 *   rtol         stop when max over right-hand sides of ||b - A x|| / ||b|| <= rtol
 *   post_reverse 1: post-relaxation visits the colour classes in reverse order
 *                (symmetric cycle); 0: same order as pre-relaxation
 *   solver       SMG_SOLVER_VCYCLE (default) or SMG_SOLVER_PCG
 *   smoother     SMG_SMOOTHER_GS (default) or SMG_SMOOTHER_JACOBI (jacobi_omega)
 *   pattern_rings, block_size  plan options (see the fields)
 *   autotune     1: smg_create times the smoother kernels of every level with
 *                1, 2, 4, 8 and 16 lanes per matrix row and keeps the fastest,
 *                then times whole cycles to choose the first level of the
 *                cluster-resident tail (binary64 and binary32 separately);
 *                0: fixed size rules
 */
typedef struct smg_options {
    int32_t mu_pre;
    int32_t mu_post;
    double  ratio;
    int64_t min_coarse;
    int64_t max_coarse;
    int32_t max_levels;
    int32_t max_cycles;
    double  rtol;
    int32_t precision;     /* SMG_FP64 or SMG_MIXED */
    int32_t post_reverse;
    int32_t autotune;
    int32_t solver;        /* SMG_SOLVER_VCYCLE or SMG_SOLVER_PCG */
    int32_t smoother;      /* SMG_SMOOTHER_GS (default) or SMG_SMOOTHER_JACOBI */
    double  jacobi_omega;  /* damping of SMG_SMOOTHER_JACOBI, in (0, 2); default 2/3 */
    int32_t pattern_rings; /* level-0 sparsity: 1 (default) the 1-ring of the cotangent
                              Laplacian; 2 the 2-ring of the Bilaplacian and squared-Hessian
                              energies (Sec. 6 "Applications"), filled by smg_update_matrix */
    int32_t block_size;    /* unknowns per vertex: 1 (default) or 3 (3|V| systems such as the
                              shell Hessians of Sec. 6): every level has 3 unknowns per vertex
                              (x, y, z adjacent), prolongation P (x) I_3, patterns of 3 x 3
                              blocks; smg_update_positions then assembles (M + t L) (x) I_3 and
                              smg_update_matrix takes any SPD matrix on that pattern */
} smg_options;

/* Result of one solve (host struct filled by smg_solve). */
typedef struct smg_info {
    int32_t cycles;         /* V-cycles (or refinement steps) executed          */
    int32_t status;         /* SMG_OK, SMG_ERR_NOT_CONVERGED or SMG_ERR_DIVERGED */
    double  rel_residual0;  /* before the first cycle                           */
    double  rel_residual;   /* after the last cycle                             */
    double  rho;            /* (rel_residual / rel_residual0)^(1/cycles)        */
} smg_info;

void        smg_default_options(smg_options *opts);
const char *smg_status_string(int status);
const char *smg_last_error(void);

/* =====================================================================
 * Host-only setup ("plan"): decimation, self-parameterization, P, the
 * symbolic coarse patterns, colourings.  Needs no GPU.
 * ===================================================================== */
typedef struct smg_plan smg_plan;

/*
 * Build the hierarchy from a triangle mesh (Alg. 1, "precompute multigrid
 * hierarchy"; Sec. 4 and App. "SSP").
 *   V  host n x 3 positions; F host m x 3 vertex indices, consistently oriented.
 *   dirichlet_mask  host n bytes (nonzero = value known, zero Dirichlet data) or
 *                   NULL; the system is reduced to the unknowns as in App.
 *                   "Dirichlet Boundary Conditions" (the finest P keeps the rows
 *                   of unknowns and drops all-zero columns together with the
 *                   matching rows of the next P).
 *   opts            NULL = defaults.
 * The plan is owned by the library; free it with smg_plan_destroy.
 */
int  smg_plan_build(const double *V, int64_t n, const int32_t *F, int64_t m,
                    const uint8_t *dirichlet_mask, const smg_options *opts, smg_plan **out);
void smg_plan_destroy(smg_plan *plan);

/* Number of levels H + 1 (level 0 = finest, level H = coarsest, solved directly). */
int  smg_plan_num_levels(const smg_plan *plan);

/* Level l operator: n rows, nnz structural entries (diagonal included) and the
 * number of colour classes of Alg. 3 (0 at the coarsest level). */
int  smg_plan_level_info(const smg_plan *plan, int level, int64_t *n, int64_t *nnz, int32_t *ncolours);

/* Geometry of mesh level l (positions after decimation).  Pointers stay valid
 * until the plan is destroyed. */
int  smg_plan_mesh(const smg_plan *plan, int level, int64_t *n, int64_t *m,
                   const double **V, const int32_t **F);

/* P_l (level >= 1) as produced by the self-parameterization, before any
 * Dirichlet reduction: n_{l-1} x 3 coarse vertex indices (-1 = unused slot) and
 * weights, in the vertex numbering of mesh levels l-1 and l (Sec. 4.5: each row
 * holds the barycentric coordinates of a fine vertex in a coarse triangle). */
int  smg_plan_prolongation(const smg_plan *plan, int level, int64_t *n_fine, int64_t *n_coarse,
                           const int32_t **idx, const double **w);

/* Symbolic pattern of A_l (CSR, sorted columns, diagonal included) in the
 * natural numbering of the reduced level (level 0: unknowns; level 1: kept
 * coarse vertices), and its Alg. 3 colouring (level < H). */
int  smg_plan_pattern(const smg_plan *plan, int level, const int64_t **rowptr, const int32_t **col);
int  smg_plan_colouring(const smg_plan *plan, int level, const int32_t **colour);

/* Level-0 unknowns (ascending original vertex ids) and the kept level-1
 * vertices after the Dirichlet column drop. */
int  smg_plan_unknowns(const smg_plan *plan, int64_t *nu, const int32_t **vertex_of_unknown);
int  smg_plan_kept_coarse(const smg_plan *plan, int64_t *nk, const int32_t **kept);

/* Decimation statistics of level l -> l+1: out[0..8] = collapses, rejected
 * (link, boundary, flip, angle, quality, solve), clamped, and 1e15 x the most
 * negative barycentric before clamping. */
int  smg_plan_stats(const smg_plan *plan, int level, int64_t out[9]);

/* Checkpoint / resume of the geometry-only setup (versioned binary file). */
int  smg_plan_save(const smg_plan *plan, const char *path);
int  smg_plan_load(const char *path, smg_plan **out);

/* =====================================================================
 * Device hierarchy: upload, per-frame update and solve (sm_103a kernels).
 * ===================================================================== */
typedef struct smg_hierarchy smg_hierarchy;

/*
 * Upload a plan to the current CUDA device (the plan may be destroyed after).
 * Allocates every device workspace the solves need; later calls allocate only
 * when a new right-hand-side count is first used.
 */
int  smg_create(const smg_plan *plan, const smg_options *opts, smg_hierarchy **out);
/* smg_plan_build + smg_create. */
int  smg_setup(const double *V, int64_t n, const int32_t *F, int64_t m,
               const uint8_t *dirichlet_mask, const smg_options *opts, smg_hierarchy **out);
void smg_destroy(smg_hierarchy *h);

/* Replace rtol / max_cycles / precision / mu / post_reverse / solver for later
 * solves (decimation fields are ignored). */
int  smg_set_options(smg_hierarchy *h, const smg_options *opts);

/*
 * Per-frame update (Alg. 1 "build left-hand-side" followed by the cached
 * Galerkin hierarchy A_{h+1} = P_{h+1}^T A_h P_{h+1}, Eq. gca, and the
 * Cholesky factor of A_H):
 *   smg_update_positions  V_dev: n x 3 positions of ALL mesh vertices (same
 *                         numbering as setup); assembles A = M + t L with the
 *                         cotangent Laplacian L (positive semi-definite sign)
 *                         and the barycentric lumped mass M.
 *   smg_update_t          same with the last positions and a new t.  Uses the
 *                         split of App. "Fast Data Smoothing": the first call
 *                         after new positions computes P^T L P and P^T M P of
 *                         every level (device memory: two more value arrays per
 *                         level); every call then forms A_l = P^T M P + t P^T L P
 *                         with one pass per level and refactors the coarsest.
 *   smg_update_matrix     vals_dev: user-supplied A on the level-0 pattern
 *                         (smg_plan_pattern level 0, nnz values); must be
 *                         symmetric positive definite.
 * Asynchronous on `stream` except that smg_update_* returns SMG_ERR_NOT_SPD
 * only from the next smg_solve (the pivot check is read there).
 */
int  smg_update_positions(smg_hierarchy *h, const double *V_dev, double t, smg_stream stream);
int  smg_update_t(smg_hierarchy *h, double t, smg_stream stream);
int  smg_update_matrix(smg_hierarchy *h, const double *vals_dev, smg_stream stream);

/*
 * Solve A x = b (Alg. 1 loop with Alg. 2 cycles), x_dev holding the initial
 * guess on entry and the result on return.  b_dev, x_dev: nu x nrhs.
 * One CUDA-graph launch runs every cycle and the device-side stopping test;
 * the call then synchronises `stream` to fill `info` (may be NULL).
 * Returns SMG_OK when converged, SMG_ERR_NOT_CONVERGED / SMG_ERR_DIVERGED
 * otherwise (x_dev then holds the last iterate).  nrhs in 1..4.
 * SMG_ERR_NOT_SPD: the last update's coarsest factor met a pivot that is not
 * positive.  SMG_ERR_TIMEOUT: a bounded wait of the cluster-tail kernels gave
 * up (a step's values never arrived); the result is not valid and the
 * hierarchy keeps reporting it until destroyed.
 */
int  smg_solve(smg_hierarchy *h, const double *b_dev, double *x_dev, int nrhs, smg_info *info,
               smg_stream stream);

/* The same solve, only enqueued: nothing waits on the host.  After the caller
 * has synchronised `stream`, smg_solve_result fills `info` and returns the
 * status smg_solve would have returned.  Calls on one handle must not overlap. */
int  smg_solve_async(smg_hierarchy *h, const double *b_dev, double *x_dev, int nrhs, smg_stream stream);
int  smg_solve_result(smg_hierarchy *h, smg_info *info);

/* Exactly one V-cycle of Alg. 2 from x_dev (precision SMG_FP64), asynchronous. */
int  smg_vcycle(smg_hierarchy *h, const double *b_dev, double *x_dev, int nrhs, smg_stream stream);

/* Lumped mass diagonal of the last smg_update_positions, unknowns order (nu),
 * and y = M x for nu x nrhs arrays. */
int  smg_mass(smg_hierarchy *h, double *m_dev, smg_stream stream);
int  smg_apply_mass(smg_hierarchy *h, const double *x_dev, double *y_dev, int nrhs, smg_stream stream);

/*
 * Derivatives for the differentiable solve x = A(V, t)^{-1} b (the adjoint
 * form): with lambda = A^{-1} g for an upstream gradient g (a second
 * smg_solve, A being symmetric), dl/db = lambda, and
 *   smg_operator_grad: gradV_dev (all n vertices x 3) = -d/dV sum_q lambda_q^T A(V,t) x_q
 *                      and dt_dev[0] = -sum_q lambda_q^T L x_q (dt_dev may be NULL);
 *                      lambda_dev, x_dev: unknowns x nrhs; V_dev: the positions of A.
 *   smg_lumped_mass:   m_dev (unknowns) = lumped mass of positions V_dev.
 *   smg_mass_grad:     gradV_dev = d/dV (w^T m(V)) for w_dev over the unknowns.
 * Known (Dirichlet) vertices count as zero in lambda, x and w.  Per-face
 * analytic derivatives of the areas and cotangents, gathered per vertex in a
 * fixed order (reproducible).  The first derivative call allocates 80 bytes
 * per face of scratch.  Asynchronous on `stream`.
 */
int  smg_operator_grad(smg_hierarchy *h, const double *V_dev, double t, const double *lambda_dev,
                       const double *x_dev, int nrhs, double *gradV_dev, double *dt_dev, smg_stream stream);
int  smg_lumped_mass(smg_hierarchy *h, const double *V_dev, double *m_dev, smg_stream stream);
int  smg_mass_grad(smg_hierarchy *h, const double *V_dev, const double *w_dev, double *gradV_dev,
                   smg_stream stream);

/* Copy the values of A_l to the host, aligned with smg_plan_pattern(level)
 * (natural numbering); synchronises `stream`. */
int  smg_level_matrix(smg_hierarchy *h, int level, double *vals_host, smg_stream stream);

/*
 * Measurement hook: enqueue `count` repetitions of one stage on the
 * hierarchy's internal level buffers (no host synchronisation, no gather or
 * scatter), so a caller can time it with CUDA events on `stream`:
 *   SMG_STAGE_CYCLE     one V-cycle (binary64) or one refinement step
 *                       (SMG_MIXED: binary32 cycle + binary64 update), as a graph
 *   SMG_STAGE_SWEEP     one forward multicolour Gauss-Seidel sweep at `level`
 *   SMG_STAGE_RESIDUAL  r = b - A x at `level`
 *   SMG_STAGE_GALERKIN  A_{level+1} = P^T A_level P
 *   SMG_STAGE_FACTOR    the coarsest Cholesky factor and inverse factor
 *   SMG_STAGE_UPDATE    the whole update graph (Galerkin chain + factor)
 * Needs a previous update; the numerical content of the buffers is whatever
 * the last solve left there.
 */
#define SMG_STAGE_CYCLE    0
#define SMG_STAGE_SWEEP    1
#define SMG_STAGE_RESIDUAL 2
#define SMG_STAGE_GALERKIN 3
#define SMG_STAGE_FACTOR   4
#define SMG_STAGE_UPDATE   5
int  smg_run_stage(smg_hierarchy *h, int stage, int level, int nrhs, int precision, int count,
                   smg_stream stream);

/* Kernel configuration of level l: out[0] lanes per row of the binary64
 * kernels, out[1] of the binary32 kernels, out[2] colour classes, out[3] slices. */
int  smg_level_config(const smg_hierarchy *h, int level, int32_t out[4]);

/* Form of the Gauss-Seidel colour steps of a level (App. "Multi-Color Gauss
 * Seidel"): out[0] / out[1] = 1 when the binary64 / binary32 sweep runs one
 * lane per row with each warp's slice of matrix entries (8 per row) staged in
 * shared memory by bulk (TMA) copies, 0 for the register-prefetching kernel
 * with the lanes per row of smg_level_config (the autotuner times both).
 * level in 0..H. */
int  smg_level_staged(const smg_hierarchy *h, int level, int32_t out[2]);

/* Residual fused with restriction from level l to l + 1 (Alg. 2 "compute
 * residual", "restrict residual" as one product b_{l+1} = P^T b_l - Q x_l with
 * Q = P^T A_l, the first stage of the Galerkin product of Eq. gca): out[0]
 * entries of Q, out[1] entries of P^T, out[2] padded slots of the operator's
 * SELL-32 layout, out[3] / out[4] lanes per row of its binary64 / binary32
 * kernel.  level in 0..H-1. */
int  smg_level_restriction(const smg_hierarchy *h, int level, int64_t out[5]);

/* Cycle configuration: out[0] = H, out[1] / out[2] = first level whose
 * smoothing and transfers run inside one thread-block cluster launch per
 * half-cycle for binary64 / binary32 cycles (H = none), out[3] = CTAs per
 * cluster (0 when the device offers no cluster launch). */
int  smg_cycle_config(const smg_hierarchy *h, int32_t out[4]);

/* Kernel launches of the library's calls, counted from the captured graphs
 * (a measurement aid; the paper has no counterpart), for the current options
 * and nrhs right-hand sides: out[0] per smg_update_positions, out[1] per
 * smg_solve outside its cycle loop, out[2] per loop iteration (one cycle, or
 * one CG iteration).  Builds the solve graph if it does not exist yet. */
int  smg_launch_counts(smg_hierarchy *h, int nrhs, int32_t out[3]);

/*
 * Residual norms of a system the caller holds, with no allocation at all.
 * (The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory when they need it -- real-time frame loops, where
 * cudaMalloc or cudaFree may synchronise the device and stall the frame, and
 * host applications that own every device allocation of a plug-in.)
 *   rowptr_dev  n + 1 row offsets (int64), col_dev / vals_dev the CSR entries
 *               (any order inside a row), all on the device
 *   x_dev, b_dev  n x nrhs row-major, nrhs in 1..4
 *   out_dev     2 nrhs doubles: out[q] = ||b_q - A x_q||_2^2, out[nrhs + q] =
 *               ||b_q||_2^2, written in stream order on `stream`
 * Nothing is allocated: the partial sums of the reduction live in a fixed
 * device array inside the library (608 x 8 doubles, 38 KB), resident on every
 * GPU that loads the library until the process exits.  The first call on a
 * device (and the first after its context changed, e.g. after
 * cudaDeviceReset) looks that array up (cudaGetSymbolAddress); make that
 * first call before any stream capture.  Every call on a device shares the array, so
 * calls whose work may overlap on the GPU (different streams without
 * ordering) race and must be serialised by the caller.  The reduction order is
 * fixed: repeated calls on the same data return identical bits.
 * Returns SMG_ERR_INVALID_ARG for nrhs outside 1..4, n < 1 or a null pointer,
 * SMG_ERR_CUDA if the launch fails.
 */
int  smg_residual_norms_noalloc(int64_t n, const int64_t *rowptr_dev, const int32_t *col_dev,
                                const double *vals_dev, const double *x_dev, const double *b_dev,
                                int nrhs, double *out_dev, smg_stream stream);

/* =====================================================================
 * Batches: many meshes (each with its own hierarchy, sizes free) with nrhs
 * right-hand sides each.  One graph launch updates every mesh (a branch per
 * mesh); one persistent kernel launch solves every mesh: each mesh's Alg. 1
 * loop of Alg. 2 cycles is a program of phases (colour steps, the fused
 * residual-restriction, the coarsest products, prolongation, the stopping
 * test) whose warp-sized work units the resident warps take from per-mesh
 * device queues, so the small coarse-level phases of different meshes run
 * side by side.  The persistent form needs the V-cycle solver, Gauss-Seidel
 * and two levels or more on every mesh; otherwise (or in SMG_BATCH_GRAPH
 * mode) the solve is one graph launch with a branch per mesh.
 * ===================================================================== */
typedef struct smg_batch smg_batch;

#define SMG_BATCH_PERSISTENT 0  /* default */
#define SMG_BATCH_GRAPH      1

/* Reference `count` hierarchies of the current device (they must outlive the
 * batch; options of a hierarchy are read when the batch first uses it). */
int  smg_batch_create(smg_hierarchy *const *hierarchies, int count, smg_batch **out);
void smg_batch_destroy(smg_batch *batch);
/* Offsets of mesh i in the concatenated vectors: unknowns [u[i], u[i+1]),
 * vertices [v[i], v[i+1]) (host arrays of count + 1). */
int  smg_batch_offsets(const smg_batch *batch, int64_t *unknown_offsets, int64_t *vertex_offsets);
/* Solve mode of later smg_batch_solve calls: SMG_BATCH_PERSISTENT or
 * SMG_BATCH_GRAPH.  SMG_ERR_INVALID_ARG for another value. */
int  smg_batch_set_mode(smg_batch *batch, int mode);
/* Watchdog of the persistent launch: a warp that finds no work unit to take
 * for `seconds` (default 2; every unit takes microseconds) makes the launch
 * stop and the solve return SMG_ERR_TIMEOUT.  0 makes every warp give up at
 * its first idle moment (exercises the timeout path; results not valid).
 * seconds in [0, 60], else SMG_ERR_INVALID_ARG. */
int  smg_batch_set_wait_limit(smg_batch *batch, double seconds);
/* smg_update_positions for every mesh: V_dev holds the meshes' positions
 * concatenated (vertex offsets x 3), one t for all. */
int  smg_batch_update_positions(smg_batch *batch, const double *V_dev, double t, smg_stream stream);
/* Solve every mesh: b_dev, x_dev concatenated (unknown offsets x nrhs,
 * row-major per mesh); infos (count entries) may be NULL.  Synchronises
 * `stream`; returns the first failing status over the meshes or SMG_OK;
 * SMG_ERR_TIMEOUT when the persistent launch found no work to take for two
 * seconds (a scheduling fault: the results are not valid). */
int  smg_batch_solve(smg_batch *batch, const double *b_dev, double *x_dev, int nrhs, smg_info *infos,
                     smg_stream stream);

/* Device bytes held by the hierarchy. */
int64_t smg_device_bytes(const smg_hierarchy *h);

#ifdef __cplusplus
}
#endif
#endif /* SMG_H */
