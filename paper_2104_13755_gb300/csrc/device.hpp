// Internal: device-resident hierarchy shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include "plan.hpp"

namespace smg {

constexpr int kMaxRhs = 4;
constexpr int kDenseNB = 32;  // block size of the coarsest dense factorisation

// Device-side solve bookkeeping (one per hierarchy).
struct SolveState {
    double bnorm2[kMaxRhs];  // ||b_r||^2 of the current right-hand sides
    double rel0;             // relative residual before the first cycle
    double rel;              // after the last cycle
    int32_t cycles;
    int32_t status;          // SMG_OK / SMG_ERR_NOT_CONVERGED / SMG_ERR_DIVERGED / -1 running
    int32_t chol_bad;        // nonzero: a coarsest pivot was not positive
    int32_t tail_err;        // nonzero: a cluster-tail step barrier wait timed out
    int32_t bulk_err;        // nonzero: a staged Gauss-Seidel launch's bulk copy did not complete
    double cg_rho[2][kMaxRhs];  // conjugate gradients: r . z of the last two iterations (slot = iteration & 1)
};

struct DLevel {
    int64_t n = 0, sbase = 0, nflat = 0, nslots = 0;
    bool coarsest = false;
    int ncolours = 0, nslices = 0;
    int R = 1;    // lanes per row of the binary64 kernels
    int R32 = 1;  // lanes per row of the binary32 kernels
    bool bulk = false, bulk32 = false;  // one lane per row with TMA-staged entries (gs_colour_bulk)
    int32_t* bulk_err = nullptr;        // SolveState::bulk_err of the hierarchy
    int32_t* colour_slice_dev = nullptr;
    int32_t* colour_row_dev = nullptr;
    int maxw = 0;  // widest slice (off-diagonal entries per row)
    std::vector<int32_t> colour_slice;  // host copy, ncolours + 1
    int32_t seed_rows = 0;              // rows of colour class 0 when they are rows [0, seed_rows), else 0
    // cluster tail: per-CTA work-unit tables (see TailLevel), binary64 and binary32
    struct TailTable {
        int32_t* tab = nullptr;
        int32_t* off = nullptr;
        int ints = 0;                              // largest per-CTA table
        int rlg = 0;                               // log2 lanes per row
        std::vector<std::pair<int, int>> E_nmy;    // per CTA: staged entries, units
    } tt[2];
    SliceMeta* slices = nullptr;
    int32_t* sell_col = nullptr;
    double* vals = nullptr;  // flat A_l
    double *Lg = nullptr, *Mg = nullptr;  // flat P^T L P and P^T M P of this level (fast t updates; level 0: L, M)
    double* dinv = nullptr;
    float* vals32 = nullptr;
    float* dinv32 = nullptr;
    // transfer to level l + 1
    int32_t* p_idx = nullptr;  // [3][n]
    double* p_w = nullptr;
    float* p_w32 = nullptr;
    int32_t* pt_ptr = nullptr;
    int32_t* pt_row = nullptr;
    double* pt_w = nullptr;
    float* pt_w32 = nullptr;
    // 3|V| systems: the operator in 3 x 3 blocks for the block sweep (layout in
    // LevelPlan), gathered from the flat values at every update
    int bs = 1;
    SliceMeta* b_slices = nullptr;
    std::vector<int32_t> b_colour_slice;
    int32_t *b_col = nullptr, *b_src = nullptr, *d_src = nullptr;
    double *b_val = nullptr, *b_dblk = nullptr;
    float *b_val32 = nullptr, *b_dblk32 = nullptr;
    int64_t b_nslots = 0;
    // residual fused with restriction: RQSlice layout over the next level's rows,
    // values [-P^T | Q = P^T A_l] (binary64 and binary32), lanes per row
    RQSlice* rq_slices = nullptr;
    int rq_nslices = 0;
    int32_t* rq_row = nullptr;
    int32_t* rq_col = nullptr;
    double* rq_val = nullptr;
    float* rq_val32 = nullptr;
    double *rq_L = nullptr, *rq_M = nullptr;  // P^T L_l and P^T M_l in the same layout (fast t updates)
    int64_t rq_nslots = 0, rq_nq = 0, rq_npt = 0;
    int Rq = 8, Rq32 = 8;
    // Galerkin stage 1 (Q = P^T A_l into rq_val) and stage 2 (A_{l+1} = Q P)
    int32_t *q_dst = nullptr, *q_ptr = nullptr, *q_src = nullptr, *q_pw = nullptr;
    int32_t *g_ptr = nullptr, *g_src = nullptr, *g_pw = nullptr;
    int64_t g_nnz = 0, q_nnz = 0;
    // vectors, capacity n * kMaxRhs
    double *x = nullptr, *b = nullptr, *r = nullptr;
    double* bdi = nullptr;  // b_i / a_ii (binary64 Gauss-Seidel on scaled rows), n x kMaxRhs
    double* gsv = nullptr;  // SELL values a_ij / a_ii (binary64 Gauss-Seidel on scaled rows)
    float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr;
    // coarsest: padded dense factor, its inverse and the inverse transposed
    int64_t np = 0;
    double *chol = nullptr, *linv = nullptr, *linvT = nullptr, *dblk = nullptr, *y = nullptr;
    double* rinv = nullptr;  // reciprocal diagonal of the coarsest factor
    // read-back map
    std::vector<int64_t> flat_to_csr;
    int64_t nnz_csr = 0;
};

}  // namespace smg

struct smg_hierarchy {
    smg_options opts{};
    int H = 0;
    std::vector<smg::DLevel> L;
    // level-0 assembly
    int64_t nv = 0, nf = 0, nu = 0;
    int32_t* F = nullptr;
    double* facegeom = nullptr;  // 4 per face: cot at corners 0..2, area
    int32_t* inc_ptr = nullptr;
    int32_t* inc_code = nullptr;
    int32_t* opp0 = nullptr;
    int32_t* opp1 = nullptr;
    int64_t* flat_to_user = nullptr;
    int64_t nnz_user = 0;
    double* Lflat0 = nullptr;  // t-independent cotan values on the level-0 flat layout
    double* Mdiag = nullptr;   // lumped mass, permuted level-0 rows
    int32_t* perm0 = nullptr;  // permuted level-0 row -> unknown index
    int32_t* vinc_ptr = nullptr;   // all vertices: incident face corners
    int32_t* vinc_code = nullptr;
    int32_t* vert_unk = nullptr;   // vertex -> unknown index (-1 known)
    double* facegrad = nullptr;    // 9 per face, allocated by the first derivative call
    double* dt_face = nullptr;
    bool have_positions = false, have_matrix = false;
    bool split_valid = false;             // Lg / Mg of every level match the current positions
    double* t_fast = nullptr;             // t of the fast update (device scalar)
    cudaGraphExec_t fast_t_exec = nullptr;  // per-level A = M + t L, level preparation, coarsest factor
    // solve state
    smg::SolveState* state = nullptr;
    smg::SolveState* state_host = nullptr;  // pinned
    double* partials = nullptr;             // [kNormBlocks][2 * kMaxRhs]
    // conjugate gradients (level-0 unknowns x kMaxRhs): iterate, residual, direction, A times direction,
    // and the partials of r . z and p . A p
    double *cg_x = nullptr, *cg_r = nullptr, *cg_p = nullptr, *cg_q = nullptr;
    double *part_rz = nullptr, *part_pq = nullptr;
    cudaStream_t cap = nullptr;             // private capture stream
    cudaStream_t aux = nullptr;             // second capture stream (parallel graph branch)
    std::vector<cudaEvent_t> ev_step;       // fork points of the coarsest factorisation
    cudaEvent_t ev_join = nullptr;
    cudaStream_t aux2 = nullptr;            // third capture stream (look-ahead trailing updates)
    std::vector<cudaEvent_t> ev_rest;       // trailing update of step j done (block columns j + 2 ..)
    std::vector<cudaEvent_t> ev_col;        // look-ahead column of step j updated
    cudaEvent_t ev_join2 = nullptr;
    cudaGraphExec_t update_exec = nullptr;
    cudaGraphExec_t factor_exec = nullptr;       // the coarsest factorisation alone (stage timing)
    std::map<int, cudaGraphExec_t> solve_exec;   // key precision * 16 + nrhs
    std::map<int, std::pair<int, int>> solve_kernels;  // same key: kernel nodes outside / inside the loop
    int update_kernels = 0;                       // kernel nodes of the update graph
    int last_body_kernels = 0;                    // kernel nodes of the last captured solve-loop body
    std::map<int, cudaGraphExec_t> cycle_exec;   // key precision * 16 + nrhs
    std::vector<void*> allocs;
    int64_t bytes = 0;
    int device = 0;
    // cluster tail: levels [tail, H) of a cycle run in one thread-block cluster
    void* tail_lv64 = nullptr;  // TailLevel<double>[H]
    void* tail_lv32 = nullptr;  // TailLevel<float>[H]
    int tail64 = 0, tail32 = 0;  // first tail level per precision (H = no tail)
    std::vector<int> tail_dbase64, tail_dbase32;  // per first tail level: bytes of tables + staged entries
    int tail_cluster = 0;        // CTAs per tail cluster (0 = clusters unavailable)
};

namespace smg {
struct BatchEngine;  // engine.cu: persistent batched solve
}

// Several hierarchies updated by one graph launch (a branch per mesh) and
// solved by one persistent launch (or one graph launch with a branch per mesh).
struct smg_batch {
    std::vector<smg_hierarchy*> hs;        // referenced, owned by the caller
    std::vector<int64_t> uoff, voff;       // unknown / vertex offsets of the concatenated vectors
    double* stage_b = nullptr;             // concatenated user-order right-hand sides (x kMaxRhs)
    double* stage_x = nullptr;             // concatenated user-order iterates (x kMaxRhs)
    double* stage_V = nullptr;             // concatenated positions
    double* t_dev = nullptr;
    double* t_host = nullptr;              // pinned
    smg::SolveState* states = nullptr;     // pinned, one per mesh
    cudaStream_t cap = nullptr;
    cudaGraphExec_t update_exec = nullptr;
    std::map<int, cudaGraphExec_t> solve_exec;
    std::map<int, smg::BatchEngine*> engines;  // key precision * 16 + nrhs
    std::map<int, cudaGraphExec_t> engine_exec;
    int* engine_err = nullptr;             // pinned: error flag of the last persistent solve
    int mode = 0;                          // SMG_BATCH_PERSISTENT or SMG_BATCH_GRAPH
    long long wait_ns = 2000000000ll;      // idle limit of a warp of the persistent launch
    std::vector<void*> allocs;
    int device = 0;
};

namespace smg {
// engine.cu: the persistent batched solve of every mesh of a batch (V-cycle
// solver, Gauss-Seidel smoother, at least two levels per mesh)
bool engine_supported(const smg_batch* B);
BatchEngine* engine_create(smg_batch* B, int K, bool mixed);  // throws on failure
void engine_destroy(BatchEngine* E);
// resets the schedule and launches the solve, then gathers every mesh's state
cudaError_t engine_record(BatchEngine* E, cudaStream_t s);
const int* engine_error_flag(const BatchEngine* E);
const SolveState* engine_states(const BatchEngine* E);
int engine_grid(const BatchEngine* E);
void engine_trace(const BatchEngine* E, const SolveState* host_states);
// dense.cu: record the coarsest factorisation (Cholesky, then the inverse factor
// and its transpose) on `s`; launches only, capturable.
// `alone`: the hierarchy's update has the GPU to itself (its diagonal tiles
// then take an SM each); false inside a batch of meshes updated together.
void record_coarsest_factor(smg_hierarchy* h, cudaStream_t s, bool alone = true);
// dense.cu: x = A_H^{-1} b through the inverse factor; `in`/`out` are binary64 or
// binary32 vectors (n x K row-major) as the flags say.  Launched as programmatic
// dependents (they wait for the preceding kernel before reading `in`).
void record_coarsest_solve(smg_hierarchy* h, int K, const void* in, bool in32, void* out, bool out32,
                           cudaStream_t s);
// Cluster launch (grid = one cluster of `cluster` CTAs) with programmatic stream
// serialization; the kernel must call griddepcontrol.wait before dependent reads.
template <typename... Params, typename... Args>
inline cudaError_t launch_cluster_pdl(void (*kernel)(Params...), int cluster, dim3 block, size_t smem,
                                      cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// launch_pdl (below) with `smem` bytes of dynamic shared memory.
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch with programmatic stream serialization: under stream capture the edge to
// the previous kernel becomes a programmatic dependency, so this kernel may start
// before its predecessor finishes and must call griddepcontrol.wait before
// reading anything that predecessor (or an earlier kernel) writes.
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace smg
