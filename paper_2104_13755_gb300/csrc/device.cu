// Device hierarchy: upload, update (assembly + Galerkin + coarsest factor),
// graph-captured V-cycles and the device half of the C ABI.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>

#include "adjoint.cuh"
#include "tail.cuh"

using namespace smg;

namespace {

struct CudaFail : std::runtime_error {
    using std::runtime_error::runtime_error;
};

inline void ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess) throw CudaFail(std::string(what) + ": " + cudaGetErrorString(e));
}

inline unsigned blocks_for(int64_t work, int threads = kern::kThreads) {
    return (unsigned)((work + threads - 1) / threads);
}

template <class T>
T* dalloc(smg_hierarchy* h, int64_t count) {
    if (count <= 0) count = 1;
    void* p = nullptr;
    ck(cudaMalloc(&p, sizeof(T) * (size_t)count), "cudaMalloc");
    h->allocs.push_back(p);
    h->bytes += (int64_t)(sizeof(T) * (size_t)count);
    return (T*)p;
}

template <class T>
T* upload(smg_hierarchy* h, const std::vector<T>& v) {
    T* p = dalloc<T>(h, (int64_t)v.size());
    if (!v.empty()) ck(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice), "upload");
    return p;
}

std::vector<float> to_f32(const std::vector<double>& v) {
    std::vector<float> o(v.size());
    for (size_t k = 0; k < v.size(); k++) o[k] = (float)v[k];
    return o;
}

void drop_graphs(smg_hierarchy* h);

// ------------------------------------------------------------------ launchers
template <typename T>
struct LevelView {
    const T *sval, *diag, *dinv, *p_w, *pt_w, *rq, *bval, *dblk;
    T *x, *b, *r;
    const T* gsv;  // scaled SELL values and right-hand side of the Gauss-Seidel steps (binary64; null
    T* bdi;        // for binary32, whose steps use sval, dinv and b)
};

template <typename T>
LevelView<T> view(DLevel& L);
template <>
LevelView<double> view<double>(DLevel& L) {
    return {L.vals + L.sbase, L.vals, L.dinv, L.p_w, L.pt_w, L.rq_val, L.b_val, L.b_dblk, L.x, L.b, L.r, L.gsv,
            L.bdi};
}
template <>
LevelView<float> view<float>(DLevel& L) {
    return {L.vals32 + L.sbase, L.vals32, L.dinv32, L.p_w32, L.pt_w32, L.rq_val32, L.b_val32, L.b_dblk32, L.x32, L.b32,
            L.r32, nullptr, nullptr};
}

// Dispatch on the lanes-per-row of a level (compile-time RR inside CALL).
#define SMG_R_SWITCH(R, CALL)                                \
    do {                                                     \
        switch (R) {                                         \
            case 1: { constexpr int RR = 1; CALL; } break;   \
            case 2: { constexpr int RR = 2; CALL; } break;   \
            case 4: { constexpr int RR = 4; CALL; } break;   \
            case 8: { constexpr int RR = 8; CALL; } break;   \
            default: { constexpr int RR = 16; CALL; } break; \
        }                                                    \
    } while (0)

template <typename T>
int lanes(const DLevel& L) {
    return sizeof(T) == 4 ? L.R32 : L.R;
}

constexpr int kBulkEntries = 8;  // entries per row staged by gs_colour_bulk (wider rows read the rest directly)

template <typename T, int K>
void rec_sweep(DLevel& L, const LevelView<T>& v, const T* b, T* x, bool reverse, cudaStream_t s, int first = 0) {
    const int R = lanes<T>(L);
    if (L.bs == 3) {  // 3|V| systems: a vertex class per launch, components in order inside;
                      // R lanes per vertex
        const T* bval = v.bval;
        const T* dblk = v.dblk;
        for (int cc = first; cc < L.ncolours; cc++) {
            const int c = reverse ? L.ncolours - 1 - cc : cc;
            const int s0 = L.b_colour_slice[c], s1 = L.b_colour_slice[c + 1];
            if (s1 <= s0) continue;
            const dim3 grid(blocks_for((int64_t)(s1 - s0) * 32 * R)), block(kern::kThreads);
            const SliceMeta* sl = L.b_slices;
            const int32_t* bcol = L.b_col;
            const int64_t nv = L.n / 3;
            const int rev = reverse ? 1 : 0;
            SMG_R_SWITCH(R, ck(launch_pdl(kern::gs_block3<T, K, RR>, grid, block, s, sl, s0, s1, bcol, bval, dblk, nv,
                                            v.dinv, b, x, rev),
                               "block gs launch"));
        }
        return;
    }
    const bool bulk = R == 1 && (sizeof(T) == 4 ? L.bulk32 : L.bulk);
    const T* gval = kern::ScaledGS<T>::value ? v.gsv : v.sval;  // binary64: rows scaled by 1 / a_ii
    const T* grhs = kern::ScaledGS<T>::value ? v.bdi : b;
    for (int cc = first; cc < L.ncolours; cc++) {
        const int c = reverse ? L.ncolours - 1 - cc : cc;
        const int s0 = L.colour_slice[c], s1 = L.colour_slice[c + 1];
        if (s1 <= s0) continue;
        const dim3 grid(blocks_for((int64_t)(s1 - s0) * 32 * R)), block(kern::kThreads);
        const SliceMeta* sl = L.slices;
        const int32_t* col = L.sell_col;
        if (bulk) {
            constexpr int WC = kBulkEntries;
            ck(launch_pdl_smem(kern::gs_colour_bulk<T, K, WC>, grid, block, (size_t)kern::BulkCfg<T, K, WC>::block_bytes,
                               s, sl, s0, s1, col, gval, v.dinv, grhs, x, (int*)L.bulk_err),
               "staged gs launch");
            continue;
        }
        SMG_R_SWITCH(R, ck(launch_pdl(kern::gs_colour<T, K, RR>, grid, block, s, sl, s0, s1, col, gval, v.dinv,
                                        grhs, x), "gs launch"));
    }
}

template <typename T, int K>
void rec_residual(DLevel& L, const LevelView<T>& v, cudaStream_t s);

// One relaxation sweep of the configured smoother: multicolour Gauss-Seidel,
// or damped Jacobi (r = b - A x into the level's residual buffer, then
// x += omega D^{-1} r).
template <typename T, int K>
void rec_relax(const smg_hierarchy* h, DLevel& L, const LevelView<T>& v, bool reverse, cudaStream_t s,
               int first = 0) {
    if (h->opts.smoother != SMG_SMOOTHER_JACOBI) {
        rec_sweep<T, K>(L, v, v.b, v.x, reverse, s, first);
        return;
    }
    rec_residual<T, K>(L, v, s);
    const T w = (T)h->opts.jacobi_omega;
    const T* di = v.dinv;
    const T* r = v.r;
    ck(launch_pdl(kern::jacobi_update<T, K>, dim3(blocks_for(L.n * K)), dim3(kern::kThreads), s, (int64_t)L.n, w, di,
                  r, v.x),
       "jacobi launch");
}

template <typename T, int K>
void rec_residual(DLevel& L, const LevelView<T>& v, cudaStream_t s) {
    const int R = lanes<T>(L);
    const dim3 grid(blocks_for((int64_t)L.nslices * 32 * R)), block(kern::kThreads);
    const SliceMeta* sl = L.slices;
    const int32_t* col = L.sell_col;
    const T* b = v.b;
    const T* x = v.x;
    SMG_R_SWITCH(R, ck(launch_pdl(kern::residual<T, K, RR>, grid, block, s, sl, L.nslices, col, v.sval, v.diag, b,
                                    x, v.r), "residual launch"));
}

template <typename T>
int rq_lanes(const DLevel& L) {
    return sizeof(T) == 4 ? L.Rq32 : L.Rq;
}

// Residual fused with restriction from level l into level l + 1 (one launch).
template <typename T, int K>
void rec_restrict_fused(DLevel& L, const LevelView<T>& v, const LevelView<T>& vn, int nseed, cudaStream_t s) {
    const int R = rq_lanes<T>(L);
    const dim3 grid(blocks_for((int64_t)L.rq_nslices * 32 * R)), block(kern::kThreads);
    const RQSlice* sl = L.rq_slices;
    const int32_t* row = L.rq_row;
    const int32_t* col = L.rq_col;
    const T* val = v.rq;
    const T* b = v.b;
    const T* x = v.x;
    const T* dinv_n = vn.dinv;
    T* bdi_n = vn.bdi;  // binary64 levels swept on scaled rows also get b / a_ii
    SMG_R_SWITCH(R, ck(launch_pdl(kern::restrict_fused<T, K, RR>, grid, block, s, sl, L.rq_nslices, row, col, val, b,
                                    x, vn.b, vn.x, dinv_n, nseed, bdi_n), "fused restriction launch"));
}

// Shared-memory slots of the cluster tail: per level, the replica of x (n
// rounded up to 32) and the distributed b and r (nloc = 32 * ceil(n / (32 CS))
// rows per CTA), levels packed from the coarsest tail level upwards so a tail
// that starts at level t needs the first tail_slots(t) slots (times K
// right-hand sides and the value size), placed after the tail levels' slice
// tables and staged entries.
int tail_nloc(int64_t n, int cs) { return (int)((n + 32 * cs - 1) / (32 * cs)) * 32; }
int tail_npad(int64_t n) { return (int)((n + 31) / 32) * 32; }
int tail_nwork(const DLevel& L, bool single) {
    const DLevel::TailTable& T = L.tt[single ? 1 : 0];
    int m = 0;
    for (const auto& en : T.E_nmy) m = std::max(m, en.second);
    return m << (5 - T.rlg);  // 32 / R rows per unit
}
int64_t tail_slots(const smg_hierarchy* h, int t, bool single) {
    int64_t slots = 0;
    for (int l = t; l < h->H; l++)
        slots += tail_npad(h->L[l].n) + 2 * (int64_t)tail_nloc(h->L[l].n, h->tail_cluster) +
                 tail_nwork(h->L[l], single);
    return slots;
}
constexpr size_t kTailSmemMax = 226 * 1024;  // 227 KB per block, less room for the static mbarrier

size_t tail_bytes(const smg_hierarchy* h, int t, bool single, int K) {
    const std::vector<int>& db = single ? h->tail_dbase32 : h->tail_dbase64;
    return (size_t)db[t] + (size_t)tail_slots(h, t, single) * K * (single ? sizeof(float) : sizeof(double));
}

// First tail level for K right-hand sides: the tuned level, moved down while its
// shared memory does not fit in one CTA.
int tail_start(const smg_hierarchy* h, bool single, int K) {
    if (h->tail_cluster == 0 || h->H == 0 || h->opts.smoother == SMG_SMOOTHER_JACOBI || h->opts.block_size != 1)
        return h->H;
    int t = std::min(single ? h->tail32 : h->tail64, h->H);
    while (t < h->H && tail_bytes(h, t, single, K) > kTailSmemMax) t++;
    return t;
}

template <typename T, int K>
void rec_tail(smg_hierarchy* h, bool down, int t, cudaStream_t s) {
    const bool single = sizeof(T) == 4;
    const TailLevel<T>* lv = (const TailLevel<T>*)(single ? h->tail_lv32 : h->tail_lv64) + (size_t)t * h->H;
    const dim3 block(kern::TailThreads<T>::value);
    const size_t smem = tail_bytes(h, t, single, K);
    const int lg = h->tail_cluster == 16 ? 4 : 3;
    const int dbase = (single ? h->tail_dbase32 : h->tail_dbase64)[t];
    if (down)
        ck(launch_cluster_pdl(kern::tail_down<T, K>, h->tail_cluster, block, smem, s, lv, t, h->H, h->opts.mu_pre, lg,
                              dbase),
           "tail down");
    else
        ck(launch_cluster_pdl(kern::tail_up<T, K>, h->tail_cluster, block, smem, s, lv, t, h->H, h->opts.mu_post,
                              h->opts.post_reverse != 0 ? 1 : 0, lg, dbase),
           "tail up");
}

// One V-cycle of Alg. 2 on the level buffers (x_0, b_0 of the chosen precision).
// Coarse levels start from x = 0, which the restriction kernel writes. On a
// coarse level that the launched kernels relax with Gauss-Seidel, the first
// pre-relaxation colour step from that zero is x_i = b_i / a_ii on colour
// class 0 (bitwise, as the step computes it), so the restriction writes those
// values and the step is not launched. Levels [t, H) run in the cluster tail
// kernels.
template <typename T, int K>
void rec_vcycle(smg_hierarchy* h, cudaStream_t s) {
    const int H = h->H;
    const bool single = sizeof(T) == 4;
    const int t = tail_start(h, single, K);
    const bool gs = h->opts.smoother != SMG_SMOOTHER_JACOBI && h->opts.mu_pre > 0;
    auto seeded = [&](int l) { return gs && l >= 1 && l < t && h->L[l].seed_rows > 0; };
    for (int l = 0; l < t; l++) {
        DLevel& L = h->L[l];
        DLevel& N = h->L[l + 1];
        LevelView<T> v = view<T>(L);
        LevelView<T> vn = view<T>(N);
        for (int it = 0; it < h->opts.mu_pre; it++)  // pre-relaxation
            rec_relax<T, K>(h, L, v, false, s, (it == 0 && seeded(l)) ? 1 : 0);
        const int nseed = seeded(l + 1) ? N.seed_rows : 0;
        rec_restrict_fused<T, K>(L, v, vn, nseed, s);  // b_{l+1} = P^T (b_l - A_l x_l), x_{l+1} = start
    }
    if (t < H) rec_tail<T, K>(h, true, t, s);
    DLevel& C = h->L[H];
    LevelView<T> vc = view<T>(C);
    record_coarsest_solve(h, K, vc.b, single, vc.x, single, s);  // direct solve at level H
    if (t < H) rec_tail<T, K>(h, false, t, s);
    for (int l = t - 1; l >= 0; l--) {
        DLevel& L = h->L[l];
        DLevel& N = h->L[l + 1];
        LevelView<T> v = view<T>(L);
        LevelView<T> vn = view<T>(N);
        const dim3 grid(blocks_for(L.n)), block(kern::kThreads);
        const T* xc = vn.x;
        ck(launch_pdl(kern::prolong_add<T, K>, grid, block, s, (int)L.n, (const int32_t*)L.p_idx, v.p_w, xc, v.x),
           "prolong launch");
        for (int it = 0; it < h->opts.mu_post; it++) rec_relax<T, K>(h, L, v, h->opts.post_reverse != 0, s);
    }
}

// Level-0 residual norm partials (binary64); with r32 also the binary32 residual
// (next inner right-hand side) and a zero binary32 iterate.
template <int K>
void rec_resnorm(smg_hierarchy* h, bool init, bool r32, cudaStream_t s, double* r64 = nullptr) {
    DLevel& L = h->L[0];
    float* out32 = L.b32;
    float* x32 = L.x32;
    const dim3 grid(kern::kNormBlocks), block(kern::kThreads);
    const double* b = L.b;
    const double* x = L.x;
    const double* vals = L.vals;
    if (L.coarsest) {
        const int n = (int)L.n;
#define SMG_RN(I, R32) ck(launch_pdl(kern::resnorm_dense<K, I, R32>, grid, block, s, n, vals, b, x, h->partials, out32, x32, r64), "resnorm")
        if (init && r32) SMG_RN(true, true);
        else if (init) SMG_RN(true, false);
        else if (r32) SMG_RN(false, true);
        else SMG_RN(false, false);
#undef SMG_RN
        return;
    }
    const SliceMeta* sl = L.slices;
    const int32_t* col = L.sell_col;
    const double* sval = L.vals + L.sbase;
#define SMG_RN(I, R32)                                                                                            \
    SMG_R_SWITCH(L.R, ck(launch_pdl(kern::resnorm<K, RR, I, R32>, grid, block, s, sl, L.nslices, col, sval, vals, b, \
                                    x, h->partials, out32, x32, r64), "resnorm"))
    if (init && r32) SMG_RN(true, true);
    else if (init) SMG_RN(true, false);
    else if (r32) SMG_RN(false, true);
    else SMG_RN(false, false);
#undef SMG_RN
}

template <int K>
void rec_cycle_fp64(smg_hierarchy* h, cudaStream_t s) {
    if (h->H == 0) {
        DLevel& C = h->L[0];
        record_coarsest_solve(h, K, C.b, false, C.x, false, s);
    } else {
        rec_vcycle<double, K>(h, s);
    }
}

template <int K>
void rec_cycle_mixed(smg_hierarchy* h, cudaStream_t s) {
    DLevel& L0 = h->L[0];
    // the binary32 iterate x32_0 was zeroed by the residual kernel that wrote b32_0
    if (h->H == 0) record_coarsest_solve(h, K, L0.b32, true, L0.x32, true, s);
    else rec_vcycle<float, K>(h, s);
    const float* d = L0.x32;
    ck(launch_pdl(kern::ir_update, dim3(blocks_for(L0.n * K)), dim3(kern::kThreads), s, (int64_t)(L0.n * K), d, L0.x),
       "ir update");
}

template <int K>
void rec_final(smg_hierarchy* h, cudaGraphConditionalHandle hnd, bool init, bool use_cond, cudaStream_t s) {
    const double* part = h->partials;
    ck(launch_pdl(kern::norm_final<K>, dim3(1), dim3(kern::kThreads), s, part, (int)kern::kNormBlocks, h->state, hnd,
                  init ? 1 : 0, h->opts.rtol, h->opts.max_cycles, use_cond ? 1 : 0),
       "norm final");
}

// One iteration of conjugate gradients preconditioned by one V-cycle (binary64,
// or binary32 when `mixed`) from a zero start: z = cycle(r), beta, p, q = A p,
// alpha, x and r, and the partials of ||r||^2 for the stopping test.
template <typename T, int K>
void rec_pcg_iteration(smg_hierarchy* h, cudaStream_t s) {
    DLevel& L0 = h->L[0];
    LevelView<T> v0 = view<T>(L0);
    const int64_t n = L0.n, m = n * K;
    const dim3 eg(blocks_for(m)), blk(kern::kThreads), rg(kern::kNormBlocks);
    const double* r = h->cg_r;
    const double* dinv0 = L0.dinv;
    double* bdi0 = (double*)v0.bdi;
    ck(launch_pdl(kern::cg_precond_in<T>, eg, blk, s, m, (int)K, r, v0.b, v0.x, dinv0, bdi0), "cg precond in");
    if (h->H == 0) record_coarsest_solve(h, K, v0.b, sizeof(T) == 4, v0.x, sizeof(T) == 4, s);
    else rec_vcycle<T, K>(h, s);
    const T* z = v0.x;
    ck(launch_pdl(kern::cg_dot<K, T>, rg, blk, s, n, r, z, h->part_rz), "cg dot");
    const double* prz = h->part_rz;
    ck(launch_pdl(kern::cg_p_update<K, T>, rg, blk, s, n, prz, z, h->cg_p, h->state), "cg p");
    const double* p = h->cg_p;
    if (L0.coarsest) {
        ck(launch_pdl(kern::cg_spmv_dense<K>, rg, blk, s, (int)n, (const double*)L0.vals, p, h->cg_q, h->part_pq),
           "cg spmv");
    } else {
        const SliceMeta* sl = L0.slices;
        const int32_t* col = L0.sell_col;
        const double* sval = L0.vals + L0.sbase;
        const double* diag = L0.vals;
        SMG_R_SWITCH(std::max(L0.R, 1), ck(launch_pdl(kern::cg_spmv<K, RR>, rg, blk, s, sl, L0.nslices, col, sval,
                                                       diag, p, h->cg_q, h->part_pq),
                                            "cg spmv"));
    }
    const double* ppq = h->part_pq;
    const double* q = h->cg_q;
    const SolveState* st = h->state;
    ck(launch_pdl(kern::cg_xr_update<K>, rg, blk, s, n, ppq, p, q, h->cg_x, h->cg_r, st, h->partials), "cg x r");
}

template <int K>
void rec_copy(smg_hierarchy* h, const double* src, double* dst, cudaStream_t s) {
    const int64_t m = h->L[0].n * K;
    ck(launch_pdl(kern::cg_copy, dim3(blocks_for(m)), dim3(kern::kThreads), s, m, src, dst), "copy");
}

// Kernel nodes of a graph (memset and conditional nodes not counted).
int count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    int k = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
}

// Append to graph g an independent branch solving one system: optional
// prologue, ||b|| and the first stopping test, a WHILE node running one cycle
// + residual norm + stopping test per iteration, optional epilogue after the
// loop.  Captured on `s`; the branch has no dependency on other nodes of g.
template <int K>
void add_solve_branch(smg_hierarchy* h, cudaGraph_t g, cudaStream_t s, bool mixed,
                      const std::function<void(cudaStream_t)>& prologue,
                      const std::function<void(cudaStream_t)>& epilogue) {
    cudaGraphConditionalHandle hnd;
    ck(cudaGraphConditionalHandleCreate(&hnd, g, 0, 0), "cudaGraphConditionalHandleCreate");
    ck(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal), "capture init");
    const bool pcg = h->opts.solver == SMG_SOLVER_PCG;
    if (prologue) prologue(s);
    if (pcg) {  // r = b - A x0 kept in binary64; the CG iterate leaves x_0 free for the preconditioner
        rec_resnorm<K>(h, true, false, s, h->cg_r);
        rec_copy<K>(h, h->L[0].x, h->cg_x, s);
    } else {
        rec_resnorm<K>(h, true, mixed, s);
    }
    rec_final<K>(h, hnd, true, true, s);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    ck(cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps), "capture info");
    std::vector<cudaGraphNode_t> frontier(deps, deps + ndeps);
    ck(cudaGetLastError(), "init launches");
    cudaGraph_t gg = g;
    ck(cudaStreamEndCapture(s, &gg), "end capture init");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    ck(cudaGraphAddNode(&wnode, g, frontier.data(), nullptr, frontier.size(), &cp), "add while node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ck(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal), "capture body");
    if (pcg) {
        if (mixed) rec_pcg_iteration<float, K>(h, s);
        else rec_pcg_iteration<double, K>(h, s);
    } else {
        if (mixed) rec_cycle_mixed<K>(h, s);
        else rec_cycle_fp64<K>(h, s);
        rec_resnorm<K>(h, false, mixed, s);
    }
    rec_final<K>(h, hnd, false, true, s);
    ck(cudaGetLastError(), "body launches");
    ck(cudaStreamEndCapture(s, &body), "end capture body");
    h->last_body_kernels = count_kernel_nodes(body);
    if (epilogue || pcg) {
        ck(cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal), "capture epilogue");
        if (pcg) rec_copy<K>(h, h->cg_x, h->L[0].x, s);
        if (epilogue) epilogue(s);
        ck(cudaGetLastError(), "epilogue launches");
        gg = g;
        ck(cudaStreamEndCapture(s, &gg), "end capture epilogue");
    }
}

template <int K>
cudaGraphExec_t build_solve_graph(smg_hierarchy* h, bool mixed) {
    cudaGraph_t g = nullptr;
    ck(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    add_solve_branch<K>(h, g, h->cap, mixed, nullptr, nullptr);
    const int key = (h->opts.solver == SMG_SOLVER_PCG ? 32 : 0) + (mixed ? 16 : 0) + K;
    h->solve_kernels[key] = {count_kernel_nodes(g), h->last_body_kernels};
    cudaGraphExec_t exec = nullptr;
    ck(cudaGraphInstantiate(&exec, g, 0), "instantiate solve graph");
    cudaGraphDestroy(g);
    return exec;
}

template <int K>
cudaGraphExec_t build_cycle_graph(smg_hierarchy* h, bool mixed) {
    cudaStream_t s = h->cap;
    cudaGraph_t g = nullptr;
    ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture cycle");
    if (mixed) rec_cycle_mixed<K>(h, s);
    else rec_cycle_fp64<K>(h, s);
    ck(cudaGetLastError(), "cycle launches");
    ck(cudaStreamEndCapture(s, &g), "end capture cycle");
    cudaGraphExec_t exec = nullptr;
    ck(cudaGraphInstantiate(&exec, g, 0), "instantiate cycle graph");
    cudaGraphDestroy(g);
    return exec;
}

cudaGraphExec_t solve_graph(smg_hierarchy* h, int K, bool mixed) {
    const int key = (h->opts.solver == SMG_SOLVER_PCG ? 32 : 0) + (mixed ? 16 : 0) + K;
    auto it = h->solve_exec.find(key);
    if (it != h->solve_exec.end()) return it->second;
    cudaGraphExec_t e = nullptr;
    switch (K) {
        case 1: e = build_solve_graph<1>(h, mixed); break;
        case 2: e = build_solve_graph<2>(h, mixed); break;
        case 3: e = build_solve_graph<3>(h, mixed); break;
        default: e = build_solve_graph<4>(h, mixed); break;
    }
    h->solve_exec[key] = e;
    return e;
}

cudaGraphExec_t cycle_graph(smg_hierarchy* h, int K, bool mixed) {
    const int key = (mixed ? 16 : 0) + K;
    auto it = h->cycle_exec.find(key);
    if (it != h->cycle_exec.end()) return it->second;
    cudaGraphExec_t e = nullptr;
    switch (K) {
        case 1: e = build_cycle_graph<1>(h, mixed); break;
        case 2: e = build_cycle_graph<2>(h, mixed); break;
        case 3: e = build_cycle_graph<3>(h, mixed); break;
        default: e = build_cycle_graph<4>(h, mixed); break;
    }
    h->cycle_exec[key] = e;
    return e;
}

// Lanes per row of the smoother kernels, per level and precision: the fastest
// of 1, 2, 4, 8, 16 over timed forward sweeps (values are irrelevant to the
// cost; the buffers hold zeros at this point).  Without tuning, the fewest
// lanes leaving at most eight entries per lane in the widest slices.
// Value for `level` of a per-level list in an environment variable ("R" for
// every level, or "R0,R1,..."), 0 when unset or not one of 1, 2, 4, 8, 16.
int env_lanes(const char* name, int level) {
    const char* env = std::getenv(name);
    if (!env) return 0;
    std::string spec(env);
    size_t pos = 0;
    int r = 0;
    for (int q = 0; q <= level && pos != std::string::npos; q++) {
        r = std::atoi(spec.c_str() + pos);
        size_t comma = spec.find(',', pos);
        if (q < level) pos = comma == std::string::npos ? std::string::npos : comma + 1;
    }
    return (r == 1 || r == 2 || r == 4 || r == 8 || r == 16) ? r : 0;
}

// Per-level 0/1 list (comma-separated) from the environment: -1 when unset or
// shorter than level + 1 entries.
int env_flag(const char* name, int level) {
    const char* env = std::getenv(name);
    if (!env) return -1;
    const char* p = env;
    for (int q = 0; q < level; q++) {
        p = std::strchr(p, ',');
        if (!p) return -1;
        p++;
    }
    return *p == '1' ? 1 : (*p == '0' ? 0 : -1);
}

// With SMG_LANES_PER_ROW set (a measurement aid: profilers serialise launches,
// which changes what the timing would pick), the lanes of the smoother
// (SMG_LANES_PER_ROW, SMG_LANES_PER_ROW_F32) and of the fused restriction
// (SMG_RQ_LANES, SMG_RQ_LANES_F32) come from the environment instead.
void choose_lanes(smg_hierarchy* h, const Plan& P, bool tune) {
    const char* env = std::getenv("SMG_LANES_PER_ROW");
    cudaEvent_t e0, e1;
    if (tune) {
        ck(cudaEventCreate(&e0), "event");
        ck(cudaEventCreate(&e1), "event");
    }
    for (int l = 0; l < h->H; l++) {
        DLevel& L = h->L[l];
        const LevelPlan& lp = P.L[l];
        std::vector<int32_t> w;
        for (const SliceMeta& s : lp.slices) w.push_back(s.width);
        std::sort(w.begin(), w.end());
        const int p90 = w.empty() ? 0 : w[(size_t)(0.9 * (double)(w.size() - 1))];
        int R = 1;
        while (R < 16 && (p90 + R - 1) / R > 8) R *= 2;
        L.R = L.R32 = R;
        L.bulk = L.bulk32 = false;
        L.bulk_err = &h->state->bulk_err;
        if (env) {
            if (int r = env_lanes("SMG_LANES_PER_ROW", l)) L.R = L.R32 = r;
            if (int r = env_lanes("SMG_LANES_PER_ROW_F32", l)) L.R32 = r;
            if (int r = env_lanes("SMG_RQ_LANES", l)) L.Rq = L.Rq32 = r;
            if (int r = env_lanes("SMG_RQ_LANES_F32", l)) L.Rq32 = r;
            L.bulk = L.R == 1 && env_flag("SMG_STAGED_GS", l) == 1;
            L.bulk32 = L.R32 == 1 && env_flag("SMG_STAGED_GS_F32", l) == 1;
            continue;
        }
        if (!tune) continue;
        for (int prec = 0; prec < 2; prec++) {
            float best = 1e30f;
            int bestR = R;
            bool bestBulk = false;
            // one lane per row (register-prefetching, then staged), then 2..16 lanes per row
            for (int cand = 0; cand < 6; cand++) {
                const int rc = cand <= 1 ? 1 : 1 << (cand - 1);
                const bool form = cand == 1;
                if (prec == 0) {
                    L.R = rc;
                    L.bulk = form;
                } else {
                    L.R32 = rc;
                    L.bulk32 = form;
                }
                float ms = 0.f;
                for (int rep = 0; rep < 2; rep++) {
                    if (prec == 0) {
                        LevelView<double> v = view<double>(L);
                        rec_sweep<double, 1>(L, v, v.b, v.x, false, h->cap);
                        ck(cudaEventRecord(e0, h->cap), "event");
                        for (int it = 0; it < 4; it++) rec_sweep<double, 1>(L, v, v.b, v.x, false, h->cap);
                    } else {
                        LevelView<float> v = view<float>(L);
                        rec_sweep<float, 1>(L, v, v.b, v.x, false, h->cap);
                        ck(cudaEventRecord(e0, h->cap), "event");
                        for (int it = 0; it < 4; it++) rec_sweep<float, 1>(L, v, v.b, v.x, false, h->cap);
                    }
                    ck(cudaEventRecord(e1, h->cap), "event");
                    ck(cudaEventSynchronize(e1), "event sync");
                    float t = 0.f;
                    ck(cudaEventElapsedTime(&t, e0, e1), "elapsed");
                    ms = rep == 0 ? t : std::min(ms, t);
                }
                if (std::getenv("SMG_TRACE_TUNE"))
                    std::fprintf(stderr, "[smg tune] level %d %s sweep, %2d lanes/row%s: %.1f us\n", l,
                                 prec ? "f32" : "f64", rc, form ? " (staged)" : "", ms * 250.0f);
                if (ms < best * 0.97f) {  // a later candidate must win clearly
                    best = ms;
                    bestR = rc;
                    bestBulk = form;
                }
            }
            if (prec == 0) {
                L.R = bestR;
                L.bulk = bestBulk;
            } else {
                L.R32 = bestR;
                L.bulk32 = bestBulk;
            }
        }
        // lanes per row of the fused residual-restriction kernel, the same way
        DLevel& N = h->L[l + 1];
        for (int prec = 0; prec < 2; prec++) {
            float best = 1e30f;
            int bestR = prec == 0 ? L.Rq : L.Rq32;
            for (int cand : {2, 4, 8, 16}) {
                if (prec == 0) L.Rq = cand;
                else L.Rq32 = cand;
                float ms = 0.f;
                for (int rep = 0; rep < 2; rep++) {
                    auto run = [&] {
                        if (prec == 0) rec_restrict_fused<double, 1>(L, view<double>(L), view<double>(N), 0, h->cap);
                        else rec_restrict_fused<float, 1>(L, view<float>(L), view<float>(N), 0, h->cap);
                    };
                    run();
                    ck(cudaEventRecord(e0, h->cap), "event");
                    for (int it = 0; it < 4; it++) run();
                    ck(cudaEventRecord(e1, h->cap), "event");
                    ck(cudaEventSynchronize(e1), "event sync");
                    float t = 0.f;
                    ck(cudaEventElapsedTime(&t, e0, e1), "elapsed");
                    ms = rep == 0 ? t : std::min(ms, t);
                }
                if (std::getenv("SMG_TRACE_TUNE"))
                    std::fprintf(stderr, "[smg tune] level %d %s fused restriction, %2d lanes/row: %.1f us\n", l,
                                 prec ? "f32" : "f64", cand, ms * 250.0f);
                if (ms < best * 0.97f) {
                    best = ms;
                    bestR = cand;
                }
            }
            if (prec == 0) L.Rq = bestR;
            else L.Rq32 = bestR;
        }
    }
    if (tune) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
}

// Per-CTA work-unit tables of every level for a cluster of cs CTAs (layout in
// TailLevel): the units of each colour class (a slice's rows in groups of
// 32 / R) are dealt round-robin over the CTAs.  Binary64 takes the smallest R
// for which kern::kTailPre entries per lane cover the widest row (its steps are
// bound by FP64 issue, and every lane of a row repeats the reduction and the
// update); binary32 takes at least 8 (latency-bound, cheap FLOPs).
int tail_rlg(int maxw, bool single) {
    int rlg = 0;
    while (rlg < 5 && (kern::kTailPre << rlg) < maxw) rlg++;
    if (single) rlg = std::max(rlg, 3);
    return rlg;
}
void build_tail_table(smg_hierarchy* h, const LevelPlan& lp, DLevel& L, int cs, int prec) {
    const int nc = (int)lp.colour_slice.size() - 1;
    const int rlg = tail_rlg(L.maxw, prec == 1), RL = 32 >> rlg;
    DLevel::TailTable& T = L.tt[prec];
    T.rlg = rlg;
    std::vector<std::vector<int32_t>> ent(cs);  // per CTA: 6 ints per unit
    std::vector<std::vector<int32_t>> cfirst(cs, std::vector<int32_t>(nc + 1, 0));
    std::vector<int> E(cs, 0), n_my(cs, 0);
    for (int c = 0; c < nc; c++) {
        for (int r = 0; r < cs; r++) cfirst[r][c] = n_my[r];
        int q = 0;  // unit counter of this colour
        for (int s = lp.colour_slice[c]; s < lp.colour_slice[c + 1]; s++) {
            const SliceMeta& m = lp.slices[s];
            for (int g = 0; g * RL < m.nrows; g++, q++) {
                const int r = q % cs;
                ent[r].insert(ent[r].end(), {(int32_t)m.off, m.width, m.row0 + g * RL, std::min(RL, m.nrows - g * RL),
                                             E[r], g});
                E[r] += m.width * RL;
                n_my[r]++;
            }
        }
    }
    // values a step barrier waits for: the colour's rows, plus one token from
    // each CTA that has no unit in the colour
    for (int r = 0; r < cs; r++) cfirst[r][nc] = n_my[r];
    std::vector<int32_t> wait_vals(nc);
    for (int c = 0; c < nc; c++) {
        int empty = 0;
        for (int r = 0; r < cs; r++) empty += cfirst[r][c + 1] == cfirst[r][c] ? 1 : 0;
        wait_vals[c] = lp.colour_row[c + 1] - lp.colour_row[c] + empty;
    }
    std::vector<int32_t> tab, off(cs + 1, 0);
    T.E_nmy.assign(cs, {0, 0});
    T.ints = 0;
    for (int r = 0; r < cs; r++) {
        off[r] = (int32_t)tab.size();
        const size_t head = tab.size();
        tab.push_back(n_my[r]);
        tab.push_back(E[r]);
        tab.insert(tab.end(), cfirst[r].begin(), cfirst[r].end());
        for (int c = 0; c < nc; c++) tab.push_back(wait_vals[c]);
        tab.insert(tab.end(), ent[r].begin(), ent[r].end());
        T.E_nmy[r] = {E[r], n_my[r]};
        T.ints = std::max(T.ints, (int)(tab.size() - head));
    }
    off[cs] = (int32_t)tab.size();
    T.tab = upload(h, tab);
    T.off = upload(h, off);
}
void build_tail_tables(smg_hierarchy* h, const Plan& P, int cs) {
    for (int l = 0; l < h->H; l++)
        for (int prec = 0; prec < 2; prec++) build_tail_table(h, P.L[l], h->L[l], cs, prec);
}

// Tail views of every level for one precision and a tail that starts at level
// t, with its shared-memory regions: levels packed from the coarsest upwards,
// each with its slice table and, while the staged copies still fit next to the
// arrays of one right-hand side, its staged entries (coarsest levels first).
// Returns H views; dbase = bytes of the regions of levels t..H-1.
template <typename T>
std::vector<TailLevel<T>> tail_table(smg_hierarchy* h, int t, int& dbase) {
    std::vector<TailLevel<T>> tab(h->H);
    const int cs = std::max(h->tail_cluster, 8);
    const bool single = sizeof(T) == 4;
    const int prec = single ? 1 : 0;
    int64_t budget = (int64_t)kTailSmemMax - (h->tail_cluster ? tail_slots(h, t, single) * (int64_t)sizeof(T) : 0);
    for (int l = t; l < h->H; l++) budget -= ((h->L[l].tt[prec].ints * 4 + 15) / 16) * 16;
    int64_t sbase = 0, rbase = 0;
    for (int l = h->H - 1; l >= 0; l--) {
        DLevel& L = h->L[l];
        DLevel& N = h->L[l + 1];
        LevelView<T> v = view<T>(L);
        LevelView<T> vn = view<T>(N);
        TailLevel<T>& e = tab[l];
        e.slices = L.slices;
        e.col = L.sell_col;
        e.sval = v.sval;
        e.dinv = v.dinv;
        e.diag = v.diag;
        e.colour_row = L.colour_row_dev;
        e.table = L.tt[prec].tab;
        e.table_off = L.tt[prec].off;
        e.x = v.x;
        e.b = v.b;
        e.nslices = L.nslices;
        e.ncolours = L.ncolours;
        e.n = (int)L.n;
        e.rlg = L.tt[prec].rlg;
        e.nloc = tail_nloc(L.n, cs);
        e.npad = tail_npad(L.n);
        e.nwork = tail_nwork(L, single);
        e.sbase = (int)sbase;
        sbase += e.npad + 2 * (int64_t)e.nloc + e.nwork;
        int stage = 0;
        for (const auto& en : L.tt[prec].E_nmy)
            stage = std::max(stage, StageLayout<T>(en.first, en.second << (5 - L.tt[prec].rlg)).bytes);
        e.tbytes = ((L.tt[prec].ints * 4 + 15) / 16) * 16;
        e.staged = (l >= t && stage <= budget) ? 1 : 0;
        if (e.staged) budget -= stage;
        e.rbase = (int)rbase;
        if (l >= t) rbase += e.tbytes + (e.staged ? stage : 0);
        e.pt_ptr = L.pt_ptr;
        e.pt_row = L.pt_row;
        e.pt_w = v.pt_w;
        e.n_next = (int)N.n;
        e.b_next = vn.b;
        e.x_next = vn.x;
        e.p_idx = L.p_idx;
        e.p_w = v.p_w;
        e.err = &h->state->tail_err;
    }
    dbase = (int)rbase;
    return tab;
}

// Views for every tail start, uploaded as one [t][l] array per precision.
template <typename T>
void* upload_tail_tables(smg_hierarchy* h, std::vector<int>& dbase) {
    const int H = h->H;
    dbase.assign(H + 1, 0);
    std::vector<TailLevel<T>> all;
    all.reserve((size_t)H * H);
    for (int t = 0; t < H; t++) {
        std::vector<TailLevel<T>> tab = tail_table<T>(h, t, dbase[t]);
        all.insert(all.end(), tab.begin(), tab.end());
    }
    TailLevel<T>* d = dalloc<TailLevel<T>>(h, (int64_t)H * H);
    ck(cudaMemcpy(d, all.data(), sizeof(TailLevel<T>) * all.size(), cudaMemcpyHostToDevice), "upload");
    return d;
}

template <typename T, int K>
bool allow_wide_clusters() {
    bool ok = cudaFuncSetAttribute(kern::tail_down<T, K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
              cudaSuccess;
    ok &= cudaFuncSetAttribute(kern::tail_up<T, K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    ok &= cudaFuncSetAttribute(kern::tail_down<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTailSmemMax) == cudaSuccess;
    ok &= cudaFuncSetAttribute(kern::tail_up<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax) ==
          cudaSuccess;
    return ok;
}

// CTAs per tail cluster: 16 (non-portable) when the device can schedule it, else
// the portable 8, else 0 (no tail).
int detect_tail_cluster() {
    bool ok = allow_wide_clusters<double, 1>() && allow_wide_clusters<double, 2>() &&
              allow_wide_clusters<double, 3>() && allow_wide_clusters<double, 4>() &&
              allow_wide_clusters<float, 1>() && allow_wide_clusters<float, 2>() && allow_wide_clusters<float, 3>() &&
              allow_wide_clusters<float, 4>();
    cudaGetLastError();
    if (!ok) return 0;  // the tail kernels cannot get their shared memory: no tail
    auto fits = [](auto kernel, int cs, int threads) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(threads);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        const bool ok = cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) == cudaSuccess && n >= 1;
        cudaGetLastError();
        return ok;
    };
    for (int cs : {16, 8})  // each kernel at its own block size (the largest register and thread demands)
        if (fits(kern::tail_down<double, 4>, cs, kern::TailThreads<double>::value) &&
            fits(kern::tail_down<float, 4>, cs, kern::TailThreads<float>::value))
            return cs;
    return 0;
}

float time_cycle(smg_hierarchy* h, bool mixed, cudaEvent_t e0, cudaEvent_t e1) {
    drop_graphs(h);
    cudaGraphExec_t g = cycle_graph(h, 1, mixed);
    ck(cudaGraphLaunch(g, h->cap), "tune launch");
    float best = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
        ck(cudaEventRecord(e0, h->cap), "event");
        ck(cudaGraphLaunch(g, h->cap), "tune launch");
        ck(cudaEventRecord(e1, h->cap), "event");
        ck(cudaEventSynchronize(e1), "event sync");
        float t = 0.f;
        ck(cudaEventElapsedTime(&t, e0, e1), "elapsed");
        best = std::min(best, t);
    }
    return best;
}

// First level handled by the cluster tail, per precision: the fastest cycle
// over the candidates (levels of at most 300k rows), or a size rule without tuning.
void choose_tail(smg_hierarchy* h, bool tune) {
    h->tail64 = h->tail32 = h->H;
    if (h->tail_cluster == 0 || h->H == 0) return;
    if (const char* env = std::getenv("SMG_TAIL_LEVEL")) {
        const int t = std::atoi(env);
        h->tail64 = h->tail32 = std::max(0, std::min(t, h->H));
        return;
    }
    if (!tune) {
        for (int l = h->H - 1; l >= 0 && h->L[l].nflat <= 2000000; l--) h->tail64 = l;
        for (int l = h->H - 1; l >= 1 && h->L[l].nflat <= 6000000; l--) h->tail32 = l;
        return;
    }
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0), "event");
    ck(cudaEventCreate(&e1), "event");
    const bool trace = std::getenv("SMG_TRACE_TUNE") != nullptr;
    for (int prec = 0; prec < 2; prec++) {
        int& t = prec == 0 ? h->tail64 : h->tail32;
        t = h->H;
        float best = time_cycle(h, prec == 1, e0, e1);
        if (trace) std::fprintf(stderr, "[smg tune] %s cycle, no tail: %.1f us\n", prec ? "f32" : "f64", best * 1e3f);
        int bestT = h->H;
        for (int cand = h->H - 1; cand >= 0 && h->L[cand].n <= 300000; cand--) {
            t = cand;
            if (tail_start(h, prec == 1, 1) != cand) break;  // does not fit in one CTA's shared memory
            const float ms = time_cycle(h, prec == 1, e0, e1);
            if (trace)
                std::fprintf(stderr, "[smg tune] %s cycle, tail from level %d: %.1f us\n", prec ? "f32" : "f64", cand,
                             ms * 1e3f);
            if (ms < best * 0.985f) {  // a larger tail must win by more than the timing noise
                best = ms;
                bestT = cand;
            }
        }
        t = bestT;
    }
    drop_graphs(h);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

// Galerkin stage 1 (Q = P^T A_l from the flat values `fine` into `rq`) and,
// with `coarse`, stage 2 (A_{l+1} = Q P).
void rec_galerkin(DLevel& L, DLevel& N, const double* fine, double* rq, double* coarse, cudaStream_t s) {
    kern::galerkin_q<<<blocks_for(L.rq_nq), kern::kThreads, 0, s>>>(L.rq_nq, L.q_dst, L.q_ptr, L.q_src, L.q_pw, fine,
                                                                    L.p_w, rq);
    if (coarse)
        kern::galerkin_qp<<<blocks_for(N.nflat), kern::kThreads, 0, s>>>(N.nflat, L.g_ptr, L.g_src, L.g_pw, rq, L.p_w,
                                                                         coarse);
}

// Reciprocal diagonals and binary32 copies of every level (operators and fused
// restriction operators).
void rec_prep_levels(smg_hierarchy* h, cudaStream_t s) {
    for (int l = 0; l < h->H; l++) {
        DLevel& L = h->L[l];
        kern::prep_level<<<blocks_for(L.nflat), kern::kThreads, 0, s>>>(L.nflat, L.n, L.vals, L.dinv, L.vals32,
                                                                      L.dinv32);
        kern::copy_f32<<<blocks_for(L.rq_nslots), kern::kThreads, 0, s>>>(L.rq_nslots, L.rq_val, L.rq_val32);
        if (L.bs == 1)
            kern::scale_sell<<<blocks_for((int64_t)L.nslices * 32), kern::kThreads, 0, s>>>(L.nslices, L.slices,
                                                                                         L.vals + L.sbase, L.dinv, L.gsv);
        if (L.bs == 3) {
            const int64_t nb = 9 * L.b_nslots, nd = 9 * (L.n / 3);
            kern::block_gather<<<blocks_for(nb), kern::kThreads, 0, s>>>(nb, L.b_src, L.vals, L.b_val, L.b_val32);
            kern::block_gather<<<blocks_for(nd), kern::kThreads, 0, s>>>(nd, L.d_src, L.vals, L.b_dblk, L.b_dblk32);
        }
    }
}

// The caller's right-hand side into level 0's colour-major order, and b / a_ii
// where level 0 is swept by binary64 Gauss-Seidel on scaled rows.
void gather_rhs(smg_hierarchy* h, int K, const double* b, cudaStream_t s) {
    DLevel& L0 = h->L[0];
    const int64_t m = L0.n * K;
    if (L0.bdi)
        kern::gather_rows_scaled<<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, K, h->perm0, b, L0.dinv, L0.b, L0.bdi);
    else
        kern::gather_rows<double><<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, K, h->perm0, b, L0.b);
}

// Galerkin chain, level preparation and the coarsest factor.
void rec_update(smg_hierarchy* h, cudaStream_t s, bool alone = true) {
    ck(cudaMemsetAsync(&h->state->chol_bad, 0, sizeof(int32_t), s), "memset");
    for (int l = 0; l < h->H; l++) rec_galerkin(h->L[l], h->L[l + 1], h->L[l].vals, h->L[l].rq_val, h->L[l + 1].vals, s);
    rec_prep_levels(h, s);
    record_coarsest_factor(h, s, alone);
}

// Galerkin products of L and M on their own, down the hierarchy (App. "Fast
// Data Smoothing": P^T A P = P^T M P + t P^T L P), computed once per positions.
void ensure_split(smg_hierarchy* h, cudaStream_t s) {
    if (h->split_valid) return;
    DLevel& L0 = h->L[0];
    if (!L0.Mg) {
        L0.Lg = h->Lflat0;
        L0.Mg = dalloc<double>(h, L0.nflat);
        for (int l = 1; l <= h->H; l++) {
            h->L[l].Lg = dalloc<double>(h, h->L[l].nflat);
            h->L[l].Mg = dalloc<double>(h, h->L[l].nflat);
        }
    }
    kern::mass_flat<<<blocks_for(L0.nflat), kern::kThreads, 0, s>>>(L0.nflat, L0.n, L0.coarsest ? L0.n : 0, h->Mdiag,
                                                                   L0.Mg);
    for (int l = 0; l < h->H; l++) {
        DLevel& L = h->L[l];
        DLevel& N = h->L[l + 1];
        if (!L.rq_L) {  // P^T L and P^T M in the fused restriction layout; the restriction
                        // segment of rq_M keeps -P^T (as rq_val does), rq_L holds 0 there,
                        // so rq_val = rq_M + t rq_L slot by slot
            L.rq_L = dalloc<double>(h, L.rq_nslots);
            L.rq_M = dalloc<double>(h, L.rq_nslots);
            ck(cudaMemsetAsync(L.rq_L, 0, sizeof(double) * L.rq_nslots, s), "memset");
            ck(cudaMemcpyAsync(L.rq_M, L.rq_val, sizeof(double) * L.rq_nslots, cudaMemcpyDeviceToDevice, s), "copy");
        }
        rec_galerkin(L, N, L.Lg, L.rq_L, N.Lg, s);
        rec_galerkin(L, N, L.Mg, L.rq_M, N.Mg, s);
    }
    ck(cudaGetLastError(), "split launches");
    h->split_valid = true;
}

// Every level's A = M + t L from the kept products (t in h->t_fast), the level
// preparation and the coarsest factor, as one graph.
void build_fast_t_graph(smg_hierarchy* h) {
    cudaStream_t s = h->cap;
    cudaGraph_t g = nullptr;
    ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture fast t");
    ck(cudaMemsetAsync(&h->state->chol_bad, 0, sizeof(int32_t), s), "memset");
    for (int l = 0; l <= h->H; l++) {
        DLevel& L = h->L[l];
        kern::axpy_devt<<<blocks_for(L.nflat), kern::kThreads, 0, s>>>(L.nflat, h->t_fast, L.Lg, L.Mg, L.vals);
    }
    for (int l = 0; l < h->H; l++) {
        DLevel& L = h->L[l];
        kern::axpy_devt<<<blocks_for(L.rq_nslots), kern::kThreads, 0, s>>>(L.rq_nslots, h->t_fast, L.rq_L, L.rq_M,
                                                                          L.rq_val);
    }
    rec_prep_levels(h, s);
    record_coarsest_factor(h, s);
    ck(cudaGetLastError(), "fast t launches");
    ck(cudaStreamEndCapture(s, &g), "end capture fast t");
    ck(cudaGraphInstantiate(&h->fast_t_exec, g, cudaGraphInstantiateFlagUseNodePriority), "instantiate fast t graph");
    cudaGraphDestroy(g);
}

// Level-0 assembly A = M + t L from positions V (t from device memory).
void rec_assembly(smg_hierarchy* h, const double* V, const double* t_dev, cudaStream_t s) {
    DLevel& L0 = h->L[0];
    const int64_t dense_n = L0.coarsest ? L0.n : 0;
    kern::face_geom<<<blocks_for(h->nf), kern::kThreads, 0, s>>>(h->nf, h->F, V, h->facegeom);
    kern::asm_diag<<<blocks_for(L0.n), kern::kThreads, 0, s>>>(L0.n, L0.coarsest ? L0.n + 1 : 1, h->inc_ptr,
                                                               h->inc_code, h->facegeom, h->Lflat0, h->Mdiag);
    const int64_t first = L0.coarsest ? 0 : L0.sbase;
    kern::asm_off<<<blocks_for(L0.nflat - first), kern::kThreads, 0, s>>>(L0.nflat, first, dense_n, h->opp0, h->opp1,
                                                                          h->facegeom, h->Lflat0);
    kern::combine_devt<<<blocks_for(L0.nflat), kern::kThreads, 0, s>>>(L0.nflat, L0.n, dense_n, t_dev, h->Lflat0,
                                                                       h->Mdiag, L0.vals);
}

void build_update_graph(smg_hierarchy* h) {
    cudaStream_t s = h->cap;
    cudaGraph_t g = nullptr;
    ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture update");
    rec_update(h, s);
    ck(cudaGetLastError(), "update launches");
    ck(cudaStreamEndCapture(s, &g), "end capture update");
    h->update_kernels = count_kernel_nodes(g);
    ck(cudaGraphInstantiate(&h->update_exec, g, cudaGraphInstantiateFlagUseNodePriority), "instantiate update graph");
    cudaGraphDestroy(g);
}

void drop_graphs(smg_hierarchy* h) {
    for (auto& kv : h->solve_exec) cudaGraphExecDestroy(kv.second);
    for (auto& kv : h->cycle_exec) cudaGraphExecDestroy(kv.second);
    h->solve_exec.clear();
    h->cycle_exec.clear();
}

void free_all(smg_hierarchy* h) {
    drop_graphs(h);
    if (h->update_exec) cudaGraphExecDestroy(h->update_exec);
    if (h->factor_exec) cudaGraphExecDestroy(h->factor_exec);
    if (h->fast_t_exec) cudaGraphExecDestroy(h->fast_t_exec);
    for (void* p : h->allocs) cudaFree(p);
    if (h->state_host) cudaFreeHost(h->state_host);
    for (auto e : h->ev_step)
        if (e) cudaEventDestroy(e);
    for (auto e : h->ev_col) cudaEventDestroy(e);
    for (auto e : h->ev_rest)
        if (e) cudaEventDestroy(e);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_join2) cudaEventDestroy(h->ev_join2);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->aux2) cudaStreamDestroy(h->aux2);
    h->allocs.clear();
}

void create_impl(const Plan& P, const smg_options& o, smg_hierarchy* h) {
    ck(cudaGetDevice(&h->device), "cudaGetDevice");
    h->opts = o;
    h->H = (int)P.L.size() - 1;
    ck(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaStreamCreateWithFlags(&h->aux2, cudaStreamNonBlocking), "cudaStreamCreate");
    h->L.resize(P.L.size());
    for (int l = 0; l <= h->H; l++) {
        const LevelPlan& lp = P.L[l];
        DLevel& L = h->L[l];
        L.n = lp.n;
        L.coarsest = lp.coarsest;
        L.sbase = lp.sbase;
        L.nflat = lp.nflat;
        L.nslots = lp.nslots;
        L.ncolours = lp.ncolours;
        L.R = 1;
        L.nslices = (int)lp.slices.size();
        L.colour_slice = lp.colour_slice;
        L.flat_to_csr = lp.flat_to_csr;
        L.nnz_csr = (int64_t)lp.col.size();
        L.vals = dalloc<double>(h, L.nflat);
        ck(cudaMemset(L.vals, 0, sizeof(double) * L.nflat), "memset");
        L.x = dalloc<double>(h, L.n * kMaxRhs);
        L.b = dalloc<double>(h, L.n * kMaxRhs);
        L.r = dalloc<double>(h, L.n * kMaxRhs);
        L.x32 = dalloc<float>(h, L.n * kMaxRhs);
        L.b32 = dalloc<float>(h, L.n * kMaxRhs);
        L.r32 = dalloc<float>(h, L.n * kMaxRhs);
        for (double* p : {L.x, L.b, L.r}) ck(cudaMemset(p, 0, sizeof(double) * L.n * kMaxRhs), "memset");
        for (float* p : {L.x32, L.b32, L.r32}) ck(cudaMemset(p, 0, sizeof(float) * L.n * kMaxRhs), "memset");
        if (L.coarsest) {
            L.np = (L.n + kDenseNB - 1) / kDenseNB * kDenseNB;
            L.chol = dalloc<double>(h, L.np * L.np);
            L.linv = dalloc<double>(h, L.np * L.np);
            L.linvT = dalloc<double>(h, L.np * L.np);
            L.dblk = dalloc<double>(h, L.np * kDenseNB);
            L.rinv = dalloc<double>(h, L.np);
            h->ev_step.assign(L.np / kDenseNB, nullptr);
            for (auto& e : h->ev_step) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
            h->ev_rest.assign(L.np / kDenseNB, nullptr);
            for (auto& e : h->ev_rest) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
            h->ev_col.assign(L.np / kDenseNB, nullptr);
            for (auto& e : h->ev_col) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
            ck(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "event");
            ck(cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming), "event");
            L.y = dalloc<double>(h, L.n * kMaxRhs);
            for (double* p : {L.chol, L.linv, L.linvT}) ck(cudaMemset(p, 0, sizeof(double) * L.np * L.np), "memset");
            continue;
        }
        L.slices = upload(h, lp.slices);
        L.sell_col = upload(h, lp.sell_col);
        L.colour_slice_dev = upload(h, lp.colour_slice);
        L.colour_row_dev = upload(h, lp.colour_row);
        L.seed_rows = (lp.colour_row.size() > 1 && lp.colour_row[0] == 0) ? lp.colour_row[1] : 0;
        if (!lp.b_slices.empty()) {  // 3|V| systems: 3 x 3 block layout; a launch class is not one
                                     // scalar colour, so no colour step is folded into the restriction
            L.bs = 3;
            L.seed_rows = 0;
            L.b_slices = upload(h, lp.b_slices);
            L.b_colour_slice = lp.b_colour_slice;
            L.b_col = upload(h, lp.b_col);
            L.b_src = upload(h, lp.b_src);
            L.d_src = upload(h, lp.d_src);
            L.b_nslots = lp.b_nslots;
            L.b_val = dalloc<double>(h, 9 * lp.b_nslots);
            L.b_val32 = dalloc<float>(h, 9 * lp.b_nslots);
            L.b_dblk = dalloc<double>(h, 9 * (L.n / 3));
            L.b_dblk32 = dalloc<float>(h, 9 * (L.n / 3));
        }
        for (const SliceMeta& m : lp.slices) L.maxw = std::max(L.maxw, (int)m.width);
        L.dinv = dalloc<double>(h, L.n);
        L.gsv = dalloc<double>(h, L.nflat - L.sbase);
        L.bdi = dalloc<double>(h, L.n * kMaxRhs);
        ck(cudaMemset(L.bdi, 0, sizeof(double) * L.n * kMaxRhs), "memset");
        L.vals32 = dalloc<float>(h, L.nflat);
        L.dinv32 = dalloc<float>(h, L.n);
        ck(cudaMemset(L.dinv, 0, sizeof(double) * L.n), "memset");
        ck(cudaMemset(L.vals32, 0, sizeof(float) * L.nflat), "memset");
        ck(cudaMemset(L.dinv32, 0, sizeof(float) * L.n), "memset");
        L.p_idx = upload(h, lp.p_idx);
        L.p_w = upload(h, lp.p_w);
        L.p_w32 = upload(h, to_f32(lp.p_w));
        L.pt_ptr = upload(h, lp.pt_ptr);
        L.pt_row = upload(h, lp.pt_row);
        L.pt_w = upload(h, lp.pt_w);
        L.pt_w32 = upload(h, to_f32(lp.pt_w));
        L.rq_slices = upload(h, lp.rq_slices);
        L.rq_nslices = (int)lp.rq_slices.size();
        L.rq_row = upload(h, lp.rq_row);
        L.rq_col = upload(h, lp.rq_col);
        L.rq_val = upload(h, lp.rq_w);
        L.rq_val32 = upload(h, to_f32(lp.rq_w));
        L.rq_nslots = (int64_t)lp.rq_col.size();
        L.rq_nq = (int64_t)lp.q_dst.size();
        L.rq_npt = (int64_t)lp.pt_row.size();
        L.q_dst = upload(h, lp.q_dst);
        L.q_ptr = upload(h, lp.q_ptr);
        L.q_src = upload(h, lp.q_src);
        L.q_pw = upload(h, lp.q_pw);
        L.q_nnz = (int64_t)lp.q_src.size();
        L.g_ptr = upload(h, lp.g_ptr);
        L.g_src = upload(h, lp.g_src);
        L.g_pw = upload(h, lp.g_pw);
        L.g_nnz = (int64_t)lp.g_src.size();
        {
            int R = 1;
            while (R < 16 && (lp.rq_maxw + R - 1) / R > 8) R *= 2;
            L.Rq = L.Rq32 = R;
        }
    }
    const AssemblyPlan& A = P.asmb;
    h->nv = A.nv;
    h->nf = A.nf;
    h->nu = P.L[0].n;
    h->F = upload(h, A.F);
    h->facegeom = dalloc<double>(h, 4 * A.nf);
    h->inc_ptr = upload(h, A.inc_ptr);
    h->inc_code = upload(h, A.inc_code);
    h->opp0 = upload(h, A.opp0);
    h->opp1 = upload(h, A.opp1);
    h->flat_to_user = upload(h, A.flat_to_user);
    h->nnz_user = (int64_t)P.L[0].col.size();
    h->Lflat0 = dalloc<double>(h, P.L[0].nflat);
    ck(cudaMemset(h->Lflat0, 0, sizeof(double) * P.L[0].nflat), "memset");
    h->Mdiag = dalloc<double>(h, P.L[0].n);
    h->perm0 = upload(h, P.L[0].perm);
    h->vinc_ptr = upload(h, A.vinc_ptr);
    h->vinc_code = upload(h, A.vinc_code);
    h->vert_unk = upload(h, A.vert_unk);
    h->state = dalloc<SolveState>(h, 1);
    ck(cudaMemset(h->state, 0, sizeof(SolveState)), "memset");
    h->partials = dalloc<double>(h, (int64_t)kern::kNormBlocks * 2 * kMaxRhs);
    h->part_rz = dalloc<double>(h, (int64_t)kern::kNormBlocks * kMaxRhs);
    h->part_pq = dalloc<double>(h, (int64_t)kern::kNormBlocks * kMaxRhs);
    {
        const int64_t m0 = P.L[0].n * kMaxRhs;
        h->cg_x = dalloc<double>(h, m0);
        h->cg_r = dalloc<double>(h, m0);
        h->cg_p = dalloc<double>(h, m0);
        h->cg_q = dalloc<double>(h, m0);
    }
    ck(cudaMallocHost((void**)&h->state_host, sizeof(SolveState)), "cudaMallocHost");
    h->tail_cluster = detect_tail_cluster();
    if (h->H > 0) {
        build_tail_tables(h, P, std::max(h->tail_cluster, 8));
        h->tail_lv64 = upload_tail_tables<double>(h, h->tail_dbase64);
        h->tail_lv32 = upload_tail_tables<float>(h, h->tail_dbase32);
    }
    ck(cudaDeviceSynchronize(), "upload");
    choose_lanes(h, P, o.autotune != 0);
    choose_tail(h, o.autotune != 0);
    build_update_graph(h);
    ck(cudaDeviceSynchronize(), "setup");
}

template <class T>
T* balloc(smg_batch* b, int64_t count) {
    if (count <= 0) count = 1;
    void* p = nullptr;
    ck(cudaMalloc(&p, sizeof(T) * (size_t)count), "cudaMalloc");
    b->allocs.push_back(p);
    return (T*)p;
}

void build_batch_update(smg_batch* B) {
    cudaGraph_t g = nullptr;
    ck(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    for (size_t i = 0; i < B->hs.size(); i++) {
        smg_hierarchy* h = B->hs[i];
        ck(cudaStreamBeginCaptureToGraph(B->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
           "capture batch update");
        rec_assembly(h, B->stage_V + 3 * B->voff[i], B->t_dev, B->cap);
        rec_update(h, B->cap, false);  // meshes updated together: no SM set aside per diagonal tile
        ck(cudaGetLastError(), "batch update launches");
        cudaGraph_t gg = g;
        ck(cudaStreamEndCapture(B->cap, &gg), "end capture batch update");
    }
    ck(cudaGraphInstantiate(&B->update_exec, g, cudaGraphInstantiateFlagUseNodePriority), "instantiate batch update");
    cudaGraphDestroy(g);
}

template <int K>
cudaGraphExec_t build_batch_solve(smg_batch* B, bool mixed) {
    cudaGraph_t g = nullptr;
    ck(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    for (size_t i = 0; i < B->hs.size(); i++) {
        smg_hierarchy* h = B->hs[i];
        DLevel& L0 = h->L[0];
        const int64_t m = L0.n * K;
        const double* bsrc = B->stage_b + B->uoff[i] * K;
        double* xsrc = B->stage_x + B->uoff[i] * K;
        smg::SolveState* dst = B->states + i;
        auto pro = [&](cudaStream_t s) {
            gather_rhs(h, K, bsrc, s);
            kern::gather_rows<double><<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, K, h->perm0, xsrc, L0.x);
        };
        auto epi = [&](cudaStream_t s) {
            kern::scatter_rows<double><<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, K, h->perm0, L0.x, xsrc);
            ck(cudaMemcpyAsync(dst, h->state, sizeof(smg::SolveState), cudaMemcpyDeviceToHost, s), "state copy");
        };
        add_solve_branch<K>(h, g, B->cap, mixed, pro, epi);
    }
    cudaGraphExec_t exec = nullptr;
    ck(cudaGraphInstantiate(&exec, g, 0), "instantiate batch solve");
    cudaGraphDestroy(g);
    return exec;
}

// The persistent solve as a graph: schedule reset, the engine, the states copy.
cudaGraphExec_t build_engine_graph(smg_batch* B, BatchEngine* E) {
    cudaGraph_t g = nullptr;
    ck(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "capture engine");
    ck(engine_record(E, B->cap), "engine launch");
    ck(cudaMemcpyAsync(B->states, engine_states(E), sizeof(SolveState) * B->hs.size(), cudaMemcpyDeviceToHost,
                       B->cap), "states copy");
    ck(cudaMemcpyAsync(B->engine_err, engine_error_flag(E), sizeof(int), cudaMemcpyDeviceToHost, B->cap),
       "error copy");
    ck(cudaStreamEndCapture(B->cap, &g), "end capture engine");
    cudaGraphExec_t exec = nullptr;
    ck(cudaGraphInstantiate(&exec, g, 0), "instantiate engine graph");
    cudaGraphDestroy(g);
    return exec;
}

void free_batch(smg_batch* B) {
    if (B->update_exec) cudaGraphExecDestroy(B->update_exec);
    for (auto& kv : B->solve_exec) cudaGraphExecDestroy(kv.second);
    for (auto& kv : B->engine_exec) cudaGraphExecDestroy(kv.second);
    for (auto& kv : B->engines) engine_destroy(kv.second);
    if (B->engine_err) cudaFreeHost(B->engine_err);
    for (void* p : B->allocs) cudaFree(p);
    if (B->t_host) cudaFreeHost(B->t_host);
    if (B->states) cudaFreeHost(B->states);
    if (B->cap) cudaStreamDestroy(B->cap);
}

int fail(const std::string& msg, int code) {
    set_error(msg);
    return code;
}

#define SMG_GUARD_BEGIN try {
#define SMG_GUARD_END                                      \
    }                                                      \
    catch (const CudaFail& e) {                            \
        return fail(e.what(), SMG_ERR_CUDA);               \
    }                                                      \
    catch (const std::runtime_error& e) {                  \
        cudaGetLastError();                                \
        return fail(e.what(), SMG_ERR_CUDA);               \
    }                                                      \
    catch (const std::bad_alloc&) {                        \
        return fail("host allocation failed", SMG_ERR_NO_MEMORY); \
    }

}  // namespace

extern "C" {

int smg_create(const smg_plan* plan, const smg_options* opts, smg_hierarchy** out) {
    if (!plan || !out) return fail("null plan or out", SMG_ERR_INVALID_ARG);
    *out = nullptr;
    smg_options o = plan->p.opts;
    if (opts) {  // solve-time fields from opts; decimation fields stay those of the plan
        o.mu_pre = opts->mu_pre;
        o.mu_post = opts->mu_post;
        o.max_cycles = opts->max_cycles;
        o.rtol = opts->rtol;
        o.precision = opts->precision;
        o.post_reverse = opts->post_reverse;
        o.autotune = opts->autotune;
        o.solver = opts->solver;
        o.smoother = opts->smoother;
        o.jacobi_omega = opts->jacobi_omega;
    }
    if (o.mu_pre < 0 || o.mu_post < 0 || o.max_cycles < 0 || !(o.rtol >= 0) ||
        (o.solver != SMG_SOLVER_VCYCLE && o.solver != SMG_SOLVER_PCG) ||
        (o.smoother != SMG_SMOOTHER_GS && o.smoother != SMG_SMOOTHER_JACOBI) ||
        !(o.jacobi_omega > 0.0 && o.jacobi_omega < 2.0))
        return fail("invalid solve options", SMG_ERR_INVALID_ARG);
    smg_hierarchy* h = new (std::nothrow) smg_hierarchy();
    if (!h) return SMG_ERR_NO_MEMORY;
    try {
        create_impl(plan->p, o, h);
    } catch (const CudaFail& e) {
        free_all(h);
        delete h;
        cudaGetLastError();
        return fail(e.what(), std::string(e.what()).find("out of memory") != std::string::npos ? SMG_ERR_NO_MEMORY
                                                                                                 : SMG_ERR_CUDA);
    } catch (const std::bad_alloc&) {
        free_all(h);
        delete h;
        return fail("host allocation failed", SMG_ERR_NO_MEMORY);
    }
    *out = h;
    return SMG_OK;
}

int smg_setup(const double* V, int64_t n, const int32_t* F, int64_t m, const uint8_t* mask, const smg_options* opts,
              smg_hierarchy** out) {
    smg_plan* p = nullptr;
    int st = smg_plan_build(V, n, F, m, mask, opts, &p);
    if (st != SMG_OK) return st;
    st = smg_create(p, opts, out);
    smg_plan_destroy(p);
    return st;
}

void smg_destroy(smg_hierarchy* h) {
    if (!h) return;
    cudaStreamSynchronize(h->cap);
    free_all(h);
    delete h;
}

int smg_set_options(smg_hierarchy* h, const smg_options* o) {
    if (!h || !o) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (o->mu_pre < 0 || o->mu_post < 0 || o->max_cycles < 0 || !(o->rtol >= 0) ||
        (o->precision != SMG_FP64 && o->precision != SMG_MIXED) ||
        (o->solver != SMG_SOLVER_VCYCLE && o->solver != SMG_SOLVER_PCG) ||
        (o->smoother != SMG_SMOOTHER_GS && o->smoother != SMG_SMOOTHER_JACOBI) ||
        !(o->jacobi_omega > 0.0 && o->jacobi_omega < 2.0))
        return fail("invalid solve options", SMG_ERR_INVALID_ARG);
    h->opts.mu_pre = o->mu_pre;
    h->opts.mu_post = o->mu_post;
    h->opts.max_cycles = o->max_cycles;
    h->opts.rtol = o->rtol;
    h->opts.precision = o->precision;
    h->opts.post_reverse = o->post_reverse;
    h->opts.solver = o->solver;
    h->opts.smoother = o->smoother;
    h->opts.jacobi_omega = o->jacobi_omega;
    drop_graphs(h);
    return SMG_OK;
}

int smg_update_positions(smg_hierarchy* h, const double* V, double t, smg_stream stream) {
    if (!h || !V) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (!std::isfinite(t)) return fail("t must be finite", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    DLevel& L0 = h->L[0];
    const int64_t dense_n = L0.coarsest ? L0.n : 0;
    kern::face_geom<<<blocks_for(h->nf), kern::kThreads, 0, s>>>(h->nf, h->F, V, h->facegeom);
    kern::asm_diag<<<blocks_for(L0.n), kern::kThreads, 0, s>>>(L0.n, L0.coarsest ? L0.n + 1 : 1, h->inc_ptr,
                                                               h->inc_code, h->facegeom, h->Lflat0, h->Mdiag);
    const int64_t first = L0.coarsest ? 0 : L0.sbase;
    kern::asm_off<<<blocks_for(L0.nflat - first), kern::kThreads, 0, s>>>(L0.nflat, first, dense_n, h->opp0, h->opp1,
                                                                          h->facegeom, h->Lflat0);
    kern::combine<<<blocks_for(L0.nflat), kern::kThreads, 0, s>>>(L0.nflat, L0.n, dense_n, t, h->Lflat0, h->Mdiag,
                                                                  L0.vals);
    ck(cudaGetLastError(), "assembly launches");
    ck(cudaGraphLaunch(h->update_exec, s), "update graph");
    h->have_positions = h->have_matrix = true;
    h->split_valid = false;
    return SMG_OK;
    SMG_GUARD_END
}

int smg_update_t(smg_hierarchy* h, double t, smg_stream stream) {
    if (!h) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (!h->have_positions) return fail("smg_update_t needs a previous smg_update_positions", SMG_ERR_STATE);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    // App. "Fast Data Smoothing": the first call after new positions keeps P^T L P
    // and P^T M P of every level; every call then only combines them with t
    if (!h->t_fast) h->t_fast = dalloc<double>(h, 1);
    ensure_split(h, s);
    if (!h->fast_t_exec) build_fast_t_graph(h);
    kern::set_scalar<<<1, 1, 0, s>>>(h->t_fast, t);
    ck(cudaGetLastError(), "set t");
    ck(cudaGraphLaunch(h->fast_t_exec, s), "fast t graph");
    h->have_matrix = true;
    return SMG_OK;
    SMG_GUARD_END
}

int smg_update_matrix(smg_hierarchy* h, const double* vals, smg_stream stream) {
    if (!h || !vals) return fail("null argument", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    DLevel& L0 = h->L[0];
    kern::scatter_user<<<blocks_for(L0.nflat), kern::kThreads, 0, s>>>(L0.nflat, h->flat_to_user, vals, L0.vals);
    ck(cudaGetLastError(), "scatter launch");
    ck(cudaGraphLaunch(h->update_exec, s), "update graph");
    h->have_matrix = true;
    return SMG_OK;
    SMG_GUARD_END
}

static int check_solve_args(smg_hierarchy* h, const double* b, double* x, int nrhs) {
    if (!h || !b || !x) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (nrhs < 1 || nrhs > kMaxRhs) return fail("nrhs must be 1..4", SMG_ERR_INVALID_ARG);
    if (!h->have_matrix) return fail("solve before any update", SMG_ERR_STATE);
    return SMG_OK;
}

int smg_solve_async(smg_hierarchy* h, const double* b, double* x, int nrhs, smg_stream stream) {
    int st = check_solve_args(h, b, x, nrhs);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    DLevel& L0 = h->L[0];
    const int64_t m = L0.n * nrhs;
    const bool mixed = h->opts.precision == SMG_MIXED;
    cudaGraphExec_t e = solve_graph(h, nrhs, mixed);
    gather_rhs(h, nrhs, b, s);
    kern::gather_rows<double><<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, nrhs, h->perm0, x, L0.x);
    ck(cudaGetLastError(), "gather");
    ck(cudaGraphLaunch(e, s), "solve graph");
    kern::scatter_rows<double><<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, nrhs, h->perm0, L0.x, x);
    ck(cudaGetLastError(), "scatter");
    ck(cudaMemcpyAsync(h->state_host, h->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s), "state copy");
    return SMG_OK;
    SMG_GUARD_END
}

int smg_solve_result(smg_hierarchy* h, smg_info* info) {
    if (!h) return fail("null argument", SMG_ERR_INVALID_ARG);
    const SolveState& ss = *h->state_host;
    if (info) {
        info->cycles = ss.cycles;
        info->status = ss.status;
        info->rel_residual0 = ss.rel0;
        info->rel_residual = ss.rel;
        info->rho = (ss.cycles > 0 && ss.rel0 > 0) ? std::pow(ss.rel / ss.rel0, 1.0 / ss.cycles) : 0.0;
    }
    if (ss.chol_bad) return fail("coarsest operator is not positive definite", SMG_ERR_NOT_SPD);
    if (ss.tail_err) return fail("cluster tail: a step barrier wait timed out", SMG_ERR_TIMEOUT);
    if (ss.bulk_err) return fail("Gauss-Seidel: a bulk copy of matrix entries did not complete", SMG_ERR_TIMEOUT);
    if (ss.status == SMG_ERR_NOT_CONVERGED) return fail("not converged within max_cycles", ss.status);
    if (ss.status == SMG_ERR_DIVERGED) return fail("residual became non-finite", ss.status);
    return SMG_OK;
}

int smg_solve(smg_hierarchy* h, const double* b, double* x, int nrhs, smg_info* info, smg_stream stream) {
    int st = smg_solve_async(h, b, x, nrhs, stream);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail(std::string("solve: ") + cudaGetErrorString(e), SMG_ERR_CUDA);
    return smg_solve_result(h, info);
}

int smg_vcycle(smg_hierarchy* h, const double* b, double* x, int nrhs, smg_stream stream) {
    int st = check_solve_args(h, b, x, nrhs);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    DLevel& L0 = h->L[0];
    const int64_t m = L0.n * nrhs;
    cudaGraphExec_t e = cycle_graph(h, nrhs, false);
    gather_rhs(h, nrhs, b, s);
    kern::gather_rows<double><<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, nrhs, h->perm0, x, L0.x);
    ck(cudaGetLastError(), "gather");
    ck(cudaGraphLaunch(e, s), "vcycle graph");
    kern::scatter_rows<double><<<blocks_for(m), kern::kThreads, 0, s>>>(L0.n, nrhs, h->perm0, L0.x, x);
    ck(cudaGetLastError(), "scatter");
    return SMG_OK;
    SMG_GUARD_END
}

int smg_mass(smg_hierarchy* h, double* m_dev, smg_stream stream) {
    if (!h || !m_dev) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (!h->have_positions) return fail("smg_mass needs smg_update_positions", SMG_ERR_STATE);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    kern::scatter_rows<double><<<blocks_for(h->nu), kern::kThreads, 0, s>>>(h->nu, 1, h->perm0, h->Mdiag, m_dev);
    ck(cudaGetLastError(), "mass");
    return SMG_OK;
    SMG_GUARD_END
}

int smg_apply_mass(smg_hierarchy* h, const double* x, double* y, int nrhs, smg_stream stream) {
    if (!h || !x || !y || nrhs < 1) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    if (!h->have_positions) return fail("smg_apply_mass needs smg_update_positions", SMG_ERR_STATE);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    kern::apply_mass<<<blocks_for(h->nu * nrhs), kern::kThreads, 0, s>>>(h->nu, nrhs, h->perm0, h->Mdiag, x, y);
    ck(cudaGetLastError(), "apply mass");
    return SMG_OK;
    SMG_GUARD_END
}

int smg_level_matrix(smg_hierarchy* h, int level, double* out, smg_stream stream) {
    if (!h || !out || level < 0 || level > h->H) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    DLevel& L = h->L[level];
    std::vector<double> flat(L.nflat);
    ck(cudaMemcpyAsync(flat.data(), L.vals, sizeof(double) * L.nflat, cudaMemcpyDeviceToHost, s), "copy");
    ck(cudaStreamSynchronize(s), "sync");
    for (int64_t k = 0; k < L.nnz_csr; k++) out[k] = 0.0;
    for (int64_t e = 0; e < L.nflat; e++)
        if (L.flat_to_csr[e] >= 0) out[L.flat_to_csr[e]] = flat[e];
    return SMG_OK;
    SMG_GUARD_END
}

int smg_run_stage(smg_hierarchy* h, int stage, int level, int nrhs, int precision, int count, smg_stream stream) {
    if (!h || nrhs < 1 || nrhs > kMaxRhs || count < 0 || level < 0 || level > h->H)
        return fail("invalid argument", SMG_ERR_INVALID_ARG);
    if (!h->have_matrix) return fail("stage before any update", SMG_ERR_STATE);
    const bool mixed = precision == SMG_MIXED;
    const bool needs_fine = stage == SMG_STAGE_SWEEP || stage == SMG_STAGE_RESIDUAL || stage == SMG_STAGE_GALERKIN;
    if (needs_fine && level >= h->H) return fail("level has no sparse operator", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    DLevel& L = h->L[level];
    cudaGraphExec_t e = nullptr;
    if (stage == SMG_STAGE_CYCLE) e = cycle_graph(h, nrhs, mixed);
    for (int it = 0; it < count; it++) {
        switch (stage) {
            case SMG_STAGE_CYCLE: ck(cudaGraphLaunch(e, s), "cycle graph"); break;
            case SMG_STAGE_SWEEP:
                if (mixed) {
                    LevelView<float> v = view<float>(L);
                    switch (nrhs) {
                        case 1: rec_sweep<float, 1>(L, v, v.b, v.x, false, s); break;
                        case 2: rec_sweep<float, 2>(L, v, v.b, v.x, false, s); break;
                        case 3: rec_sweep<float, 3>(L, v, v.b, v.x, false, s); break;
                        default: rec_sweep<float, 4>(L, v, v.b, v.x, false, s); break;
                    }
                } else {
                    LevelView<double> v = view<double>(L);
                    switch (nrhs) {
                        case 1: rec_sweep<double, 1>(L, v, v.b, v.x, false, s); break;
                        case 2: rec_sweep<double, 2>(L, v, v.b, v.x, false, s); break;
                        case 3: rec_sweep<double, 3>(L, v, v.b, v.x, false, s); break;
                        default: rec_sweep<double, 4>(L, v, v.b, v.x, false, s); break;
                    }
                }
                break;
            case SMG_STAGE_RESIDUAL: {
                LevelView<double> v = view<double>(L);
                rec_residual<double, 1>(L, v, s);
                break;
            }
            case SMG_STAGE_GALERKIN: {
                DLevel& N = h->L[level + 1];
                rec_galerkin(L, N, L.vals, L.rq_val, N.vals, s);
                break;
            }
            case SMG_STAGE_FACTOR:  // as the update graph runs it: captured once, launched as a graph
                if (!h->factor_exec) {
                    cudaGraph_t g = nullptr;
                    ck(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "capture factor");
                    record_coarsest_factor(h, h->cap);
                    ck(cudaGetLastError(), "factor launches");
                    ck(cudaStreamEndCapture(h->cap, &g), "end capture factor");
                    ck(cudaGraphInstantiate(&h->factor_exec, g, cudaGraphInstantiateFlagUseNodePriority), "instantiate factor graph");
                    cudaGraphDestroy(g);
                }
                ck(cudaGraphLaunch(h->factor_exec, s), "factor graph");
                break;
            case SMG_STAGE_UPDATE: ck(cudaGraphLaunch(h->update_exec, s), "update graph"); break;
            default: return fail("unknown stage", SMG_ERR_INVALID_ARG);
        }
    }
    ck(cudaGetLastError(), "stage launches");
    return SMG_OK;
    SMG_GUARD_END
}

int smg_level_restriction(const smg_hierarchy* h, int level, int64_t out[5]) {
    if (!h || !out || level < 0 || level >= h->H) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    const DLevel& L = h->L[level];
    out[0] = L.rq_nq;
    out[1] = L.rq_npt;
    out[2] = L.rq_nslots;
    out[3] = L.Rq;
    out[4] = L.Rq32;
    return SMG_OK;
}

int smg_level_config(const smg_hierarchy* h, int level, int32_t out[4]) {
    if (!h || !out || level < 0 || level > h->H) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    const DLevel& L = h->L[level];
    out[0] = L.R;
    out[1] = L.R32;
    out[2] = L.ncolours;
    out[3] = L.nslices;
    return SMG_OK;
}

int smg_level_staged(const smg_hierarchy* h, int level, int32_t out[2]) {
    if (!h || !out || level < 0 || level > h->H) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    const DLevel& L = h->L[level];
    out[0] = L.bulk ? 1 : 0;
    out[1] = L.bulk32 ? 1 : 0;
    return SMG_OK;
}

int smg_launch_counts(smg_hierarchy* h, int nrhs, int32_t out[3]) {
    if (!h || !out) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (nrhs < 1 || nrhs > kMaxRhs) return fail("nrhs must be 1..4", SMG_ERR_INVALID_ARG);
    SMG_GUARD_BEGIN
    const bool mixed = h->opts.precision == SMG_MIXED;
    solve_graph(h, nrhs, mixed);  // builds (and counts) it if needed
    const int key = (h->opts.solver == SMG_SOLVER_PCG ? 32 : 0) + (mixed ? 16 : 0) + nrhs;
    const auto it = h->solve_kernels.find(key);
    // smg_update_positions launches four assembly kernels before its graph;
    // smg_solve_async two gathers before and one scatter after its graph
    out[0] = 4 + h->update_kernels;
    out[1] = it == h->solve_kernels.end() ? -1 : 3 + it->second.first;
    out[2] = it == h->solve_kernels.end() ? -1 : it->second.second;
    return SMG_OK;
    SMG_GUARD_END
}

int smg_cycle_config(const smg_hierarchy* h, int32_t out[4]) {
    if (!h || !out) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    out[0] = h->H;
    out[1] = h->tail64;
    out[2] = h->tail32;
    out[3] = h->tail_cluster;
    return SMG_OK;
}

int smg_batch_create(smg_hierarchy* const* hs, int count, smg_batch** out) {
    if (!hs || count < 1 || !out) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail("no current device", SMG_ERR_CUDA);
    for (int i = 0; i < count; i++)
        if (!hs[i] || hs[i]->device != dev) return fail("null hierarchy or one of another device", SMG_ERR_INVALID_ARG);
    smg_batch* B = new (std::nothrow) smg_batch();
    if (!B) return SMG_ERR_NO_MEMORY;
    try {
        B->device = dev;
        B->hs.assign(hs, hs + count);
        B->uoff.assign(count + 1, 0);
        B->voff.assign(count + 1, 0);
        for (int i = 0; i < count; i++) {
            B->uoff[i + 1] = B->uoff[i] + hs[i]->nu;
            B->voff[i + 1] = B->voff[i] + hs[i]->nv;
        }
        ck(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking), "cudaStreamCreate");
        B->stage_b = balloc<double>(B, B->uoff[count] * kMaxRhs);
        B->stage_x = balloc<double>(B, B->uoff[count] * kMaxRhs);
        B->stage_V = balloc<double>(B, B->voff[count] * 3);
        B->t_dev = balloc<double>(B, 1);
        ck(cudaMallocHost((void**)&B->t_host, sizeof(double)), "cudaMallocHost");
        ck(cudaMallocHost((void**)&B->states, sizeof(SolveState) * count), "cudaMallocHost");
        ck(cudaMallocHost((void**)&B->engine_err, sizeof(int)), "cudaMallocHost");
        *B->engine_err = 0;
        build_batch_update(B);
    } catch (const CudaFail& e) {
        free_batch(B);
        delete B;
        cudaGetLastError();
        return fail(e.what(), SMG_ERR_CUDA);
    } catch (const std::bad_alloc&) {
        free_batch(B);
        delete B;
        return fail("host allocation failed", SMG_ERR_NO_MEMORY);
    }
    *out = B;
    return SMG_OK;
}

void smg_batch_destroy(smg_batch* B) {
    if (!B) return;
    cudaStreamSynchronize(B->cap);
    free_batch(B);
    delete B;
}

int smg_batch_offsets(const smg_batch* B, int64_t* u, int64_t* v) {
    if (!B) return fail("null batch", SMG_ERR_INVALID_ARG);
    for (size_t i = 0; i < B->uoff.size(); i++) {
        if (u) u[i] = B->uoff[i];
        if (v) v[i] = B->voff[i];
    }
    return SMG_OK;
}

int smg_batch_update_positions(smg_batch* B, const double* V, double t, smg_stream stream) {
    if (!B || !V) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (!std::isfinite(t)) return fail("t must be finite", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    ck(cudaMemcpyAsync(B->stage_V, V, sizeof(double) * 3 * B->voff.back(), cudaMemcpyDeviceToDevice, s), "copy V");
    ck(cudaStreamSynchronize(s), "sync");  // t_host is reused by the next call
    *B->t_host = t;
    ck(cudaMemcpyAsync(B->t_dev, B->t_host, sizeof(double), cudaMemcpyHostToDevice, s), "copy t");
    ck(cudaGraphLaunch(B->update_exec, s), "batch update");
    for (smg_hierarchy* h : B->hs) {
        h->have_positions = h->have_matrix = true;
        h->split_valid = false;
    }
    return SMG_OK;
    SMG_GUARD_END
}

int smg_batch_solve(smg_batch* B, const double* b, double* x, int nrhs, smg_info* infos, smg_stream stream) {
    if (!B || !b || !x) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (nrhs < 1 || nrhs > kMaxRhs) return fail("nrhs must be 1..4", SMG_ERR_INVALID_ARG);
    for (smg_hierarchy* h : B->hs)
        if (!h->have_matrix) return fail("batch solve before any update", SMG_ERR_STATE);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    const bool mixed = B->hs[0]->opts.precision == SMG_MIXED;
    const int key = (mixed ? 16 : 0) + nrhs;
    const bool persistent = B->mode == SMG_BATCH_PERSISTENT && engine_supported(B);
    auto it = persistent ? B->engine_exec.find(key) : B->solve_exec.find(key);
    cudaGraphExec_t e;
    if (persistent && it != B->engine_exec.end()) e = it->second;
    else if (persistent) {
        BatchEngine* E = engine_create(B, nrhs, mixed);
        B->engines[key] = E;
        e = build_engine_graph(B, E);
        B->engine_exec[key] = e;
    } else if (it != B->solve_exec.end()) e = it->second;
    else {
        switch (nrhs) {
            case 1: e = build_batch_solve<1>(B, mixed); break;
            case 2: e = build_batch_solve<2>(B, mixed); break;
            case 3: e = build_batch_solve<3>(B, mixed); break;
            default: e = build_batch_solve<4>(B, mixed); break;
        }
        B->solve_exec[key] = e;
    }
    const size_t bytes = sizeof(double) * (size_t)(B->uoff.back() * nrhs);
    ck(cudaMemcpyAsync(B->stage_b, b, bytes, cudaMemcpyDeviceToDevice, s), "copy b");
    ck(cudaMemcpyAsync(B->stage_x, x, bytes, cudaMemcpyDeviceToDevice, s), "copy x");
    ck(cudaGraphLaunch(e, s), "batch solve");
    ck(cudaMemcpyAsync(x, B->stage_x, bytes, cudaMemcpyDeviceToDevice, s), "copy x back");
    ck(cudaStreamSynchronize(s), "sync");
    if (persistent && *B->engine_err)
        return fail("persistent batch solve: no work unit could be taken for the idle limit", SMG_ERR_TIMEOUT);
    if (persistent) engine_trace(B->engines[key], B->states);
    int worst = SMG_OK;
    for (size_t i = 0; i < B->hs.size(); i++) {
        const SolveState& ss = B->states[i];
        if (infos) {
            infos[i].cycles = ss.cycles;
            infos[i].status = ss.status;
            infos[i].rel_residual0 = ss.rel0;
            infos[i].rel_residual = ss.rel;
            infos[i].rho = (ss.cycles > 0 && ss.rel0 > 0) ? std::pow(ss.rel / ss.rel0, 1.0 / ss.cycles) : 0.0;
        }
        int st = ss.chol_bad ? SMG_ERR_NOT_SPD : (ss.status < 0 ? SMG_OK : ss.status);
        if (worst == SMG_OK && st != SMG_OK) worst = st;
    }
    if (worst != SMG_OK) return fail("a mesh of the batch did not converge or was not SPD", worst);
    return SMG_OK;
    SMG_GUARD_END
}

int smg_batch_set_wait_limit(smg_batch* B, double seconds) {
    if (!B || !(seconds >= 0.0) || seconds > 60.0) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    B->wait_ns = (long long)(seconds * 1e9);
    for (auto& kv : B->engine_exec) cudaGraphExecDestroy(kv.second);  // rebuilt with the new limit
    for (auto& kv : B->engines) engine_destroy(kv.second);
    B->engine_exec.clear();
    B->engines.clear();
    return SMG_OK;
}

int smg_batch_set_mode(smg_batch* B, int mode) {
    if (!B || (mode != SMG_BATCH_PERSISTENT && mode != SMG_BATCH_GRAPH)) return fail("invalid argument", SMG_ERR_INVALID_ARG);
    B->mode = mode;
    return SMG_OK;
}

int smg_lumped_mass(smg_hierarchy* h, const double* V, double* m, smg_stream stream) {
    if (!h || !V || !m) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (h->opts.block_size != 1) return fail("position derivatives need one unknown per vertex", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    kern::face_geom<<<blocks_for(h->nf), kern::kThreads, 0, s>>>(h->nf, h->F, V, h->facegeom);
    kern::mass_from_faces<<<blocks_for(h->nv), kern::kThreads, 0, s>>>(h->nv, h->vinc_ptr, h->vinc_code, h->vert_unk,
                                                                       h->facegeom, m);
    ck(cudaGetLastError(), "mass");
    return SMG_OK;
    SMG_GUARD_END
}

static void ensure_face_scratch(smg_hierarchy* h) {
    if (!h->facegrad) {
        h->facegrad = dalloc<double>(h, 9 * h->nf);
        h->dt_face = dalloc<double>(h, h->nf);
    }
}

int smg_mass_grad(smg_hierarchy* h, const double* V, const double* w, double* gradV, smg_stream stream) {
    if (!h || !V || !w || !gradV) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (h->opts.block_size != 1) return fail("position derivatives need one unknown per vertex", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    ensure_face_scratch(h);
    kern::face_grad<1><<<blocks_for(h->nf), kern::kThreads, 0, s>>>(h->nf, h->F, V, h->vert_unk, nullptr, nullptr, w,
                                                                   1, 0.0, 1.0, h->facegrad, h->dt_face);
    kern::vertex_gather<<<blocks_for(h->nv), kern::kThreads, 0, s>>>(h->nv, h->vinc_ptr, h->vinc_code, h->facegrad,
                                                                     gradV);
    ck(cudaGetLastError(), "mass grad");
    return SMG_OK;
    SMG_GUARD_END
}

int smg_operator_grad(smg_hierarchy* h, const double* V, double t, const double* lam, const double* x, int nrhs,
                      double* gradV, double* dt, smg_stream stream) {
    if (!h || !V || !lam || !x || !gradV) return fail("null argument", SMG_ERR_INVALID_ARG);
    if (h->opts.block_size != 1) return fail("position derivatives need one unknown per vertex", SMG_ERR_INVALID_ARG);
    if (nrhs < 1 || nrhs > kMaxRhs) return fail("nrhs must be 1..4", SMG_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    SMG_GUARD_BEGIN
    ensure_face_scratch(h);
    const dim3 grid(blocks_for(h->nf)), block(kern::kThreads);
    switch (nrhs) {
        case 1: kern::face_grad<1><<<grid, block, 0, s>>>(h->nf, h->F, V, h->vert_unk, lam, x, nullptr, 0, t, -1.0, h->facegrad, h->dt_face); break;
        case 2: kern::face_grad<2><<<grid, block, 0, s>>>(h->nf, h->F, V, h->vert_unk, lam, x, nullptr, 0, t, -1.0, h->facegrad, h->dt_face); break;
        case 3: kern::face_grad<3><<<grid, block, 0, s>>>(h->nf, h->F, V, h->vert_unk, lam, x, nullptr, 0, t, -1.0, h->facegrad, h->dt_face); break;
        default: kern::face_grad<4><<<grid, block, 0, s>>>(h->nf, h->F, V, h->vert_unk, lam, x, nullptr, 0, t, -1.0, h->facegrad, h->dt_face); break;
    }
    kern::vertex_gather<<<blocks_for(h->nv), kern::kThreads, 0, s>>>(h->nv, h->vinc_ptr, h->vinc_code, h->facegrad,
                                                                     gradV);
    if (dt) kern::sum_fixed<<<1, kern::kThreads, 0, s>>>(h->nf, h->dt_face, dt);
    ck(cudaGetLastError(), "operator grad");
    return SMG_OK;
    SMG_GUARD_END
}

int64_t smg_device_bytes(const smg_hierarchy* h) { return h ? h->bytes : 0; }

}  // extern "C"
