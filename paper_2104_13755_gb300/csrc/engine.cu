// Persistent batched solve: one kernel launch runs every V-cycle (Alg. 2) of
// every mesh of a batch, with the stopping test of Alg. 1 on the device.
//
// Each mesh's solve is compiled on the host into a program: a list of phases
// (gather of the caller's vectors, level-0 residual norm, stopping test, the
// Gauss-Seidel colour steps of every level, the fused residual-restriction,
// the two products of the coarsest direct solve, prolongation with
// correction, the refinement update of the mixed form, scatter of the
// result).  A phase is a set of independent warp-sized work units (a SELL-32
// slice's rows for the sparse phases, a dense row for the coarsest products).
// The resident warps of the launch take units from a per-mesh ticket word
// (phase << 32 | next unit), so units of different meshes -- and of the many
// small coarse-level phases of one mesh and another -- run side by side; the
// warp that completes the last unit of a phase advances that mesh to the next
// phase (or, after the stopping test, back to the first phase of a cycle).
// Dependencies exist only inside a mesh, between consecutive phases, so no
// warp ever waits for a particular other warp: a warp without work polls the
// tickets again after a short sleep, and gives up (setting an error flag
// reported as SMG_ERR_TIMEOUT) only when no unit anywhere could be taken for a
// bounded time.  Data written inside the launch is read through L2
// (ld.global.cg); units publish with a device-scope fence before their
// completion count, the phase advance with a fence before the new ticket.
//
// Every row of every unit computes exactly what the launched kernels compute
// (the same SELL slices, lanes per row and summation order), so the iterates
// equal those of a single-mesh solve without the cluster tail.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <stdexcept>
#include <string>
#include <vector>

#include "rowslice.cuh"

namespace smg {
namespace eng {

enum : int32_t {
    kGatherIn = 0,
    kResnorm,
    kNormFinal,
    kGs,
    kRestrict,
    kCoarseLo,
    kCoarseUp,
    kProlong,
    kIrUpdate,
    kScatterOut
};

constexpr int kUnitsPerResnorm = 4;  // warp slices summed by one residual-norm unit
constexpr int kElemsPerUnit = 256;   // vector elements of one gather / scatter / update unit

struct Phase {
    int32_t type, level, units, prec;  // prec: 0 binary64, 1 binary32
    // kGs: a first slice, b slices, c lanes per row; kRestrict: a rows seeded, c lanes;
    // kResnorm: a init, b binary32 residual, c lanes; kNormFinal: a init, b cycle start, c exit
    int32_t a, b, c, d;  // kNormFinal: d partials to sum
};

struct ELevel {
    const SliceMeta* slices;
    const int32_t* col;
    const double* sval;
    const float* sval32;
    const double* diag;
    const double* dinv;
    const float* dinv32;
    double *x, *b;
    float *x32, *b32;
    const RQSlice* rq;
    const int32_t* rq_row;
    const int32_t* rq_col;
    const double* rq_val;
    const float* rq_val32;
    const int32_t* p_idx;
    const double* p_w;
    const float* p_w32;
    const double *linv, *linvT;
    double* y;
    int64_t np;
    int32_t n, nslices;
};

struct EMesh {
    const Phase* prog;
    const ELevel* lv;
    const double* b_user;
    double* x_user;
    const int32_t* perm0;
    SolveState* st;
    double* part;  // [units of the residual-norm phase][2 K]
    double rtol;
    int32_t nphase, H, n0, max_cycles;
    long long* trace;  // [0] launch start, [1 + mesh] finish time (globaltimer ns)
};

// Scheduling words of one mesh, each on its own 128-byte line (meshes' words
// in different L2 lines, the polled ticket apart from the completion count).
struct alignas(128) ECtl {
    unsigned long long ticket;  // phase << 32 | next unit
    char pad0[120];
    unsigned int done;          // units of the current phase completed
    char pad1[124];
};

template <typename T>
__device__ __forceinline__ T ldc(const T* p) {
    return __ldcg(p);
}

// ---------------------------------------------------------------- units
template <typename T, int K, int R>
__device__ __noinline__ void gs_unit(const ELevel& L, const Phase& ph, int u, int lane) {
    const int s = ph.a + u / R;
    const SliceMeta m = L.slices[s];
    const T* sval = sizeof(T) == 4 ? (const T*)L.sval32 : (const T*)L.sval;
    const T* dinv = sizeof(T) == 4 ? (const T*)L.dinv32 : (const T*)L.dinv;
    T* x = sizeof(T) == 4 ? (T*)L.x32 : (T*)L.x;
    const T* b = sizeof(T) == 4 ? (const T*)L.b32 : (const T*)L.b;
    kern::RowSlice<T, K, R, kern::Pre<T, K, R>::value> rs;
    rs.load(m, u % R, lane, L.col, sval);
    const bool valid = rs.r < m.nrows;
    const int row = m.row0 + (valid ? rs.r : 0);
    const T d = __ldg(dinv + row);
    T bv[K], acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) bv[q] = ldc(b + (int64_t)row * K + q);
    rs.template dot_from<true>(m, L.col, sval, x, bv, acc);
    if (valid && rs.sub == 0)
#pragma unroll
        for (int q = 0; q < K; q++) x[(int64_t)row * K + q] = acc[q] * d;
}

template <typename T, int K, int R>
__device__ __noinline__ void restrict_unit(const ELevel& L, const ELevel& N, const Phase& ph, int u, int lane) {
    constexpr int RL = 32 / R;
    const RQSlice m = L.rq[u / R];
    const int sub = lane / RL;
    const int r = (u % R) * RL + (lane % RL);
    const int W = m.wb + m.wq;
    const bool valid = r < m.nrows;
    const int I = valid ? L.rq_row[m.pos0 + r] : 0;
    const T* val = sizeof(T) == 4 ? (const T*)L.rq_val32 : (const T*)L.rq_val;
    const T* b = sizeof(T) == 4 ? (const T*)L.b32 : (const T*)L.b;
    const T* x = sizeof(T) == 4 ? (const T*)L.x32 : (const T*)L.x;
    T* bc = sizeof(T) == 4 ? (T*)N.b32 : (T*)N.b;
    T* xc = sizeof(T) == 4 ? (T*)N.x32 : (T*)N.x;
    const T* dinv_c = sizeof(T) == 4 ? (const T*)N.dinv32 : (const T*)N.dinv;
    const int nseed = ph.a;
    T acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = T(0);
    for (int k = sub; k < W; k += R) {
        const int cc = __ldg(L.rq_col + m.off + k * 32 + r);
        const T vv = __ldg(val + m.off + k * 32 + r);
        const T* src = k < m.wb ? b : x;
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] -= vv * ldc(src + (int64_t)cc * K + q);
    }
#pragma unroll
    for (int o = 16; o >= RL; o >>= 1)
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (valid && sub == 0) {
        const T ds = I < nseed ? __ldg(dinv_c + I) : T(0);
#pragma unroll
        for (int q = 0; q < K; q++) {
            bc[(int64_t)I * K + q] = acc[q];
            xc[(int64_t)I * K + q] = I < nseed ? acc[q] * ds : T(0);
        }
    }
}

template <typename T, int K>
__device__ __noinline__ void prolong_unit(const ELevel& L, const ELevel& N, int u, int lane) {
    const int p = u * 32 + lane;
    if (p >= L.n) return;
    const int n = L.n;
    const T* w = sizeof(T) == 4 ? (const T*)L.p_w32 : (const T*)L.p_w;
    const T* xc = sizeof(T) == 4 ? (const T*)N.x32 : (const T*)N.x;
    T* x = sizeof(T) == 4 ? (T*)L.x32 : (T*)L.x;
    int c[3];
    T wa[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        c[a] = __ldg(L.p_idx + (int64_t)a * n + p);
        wa[a] = __ldg(w + (int64_t)a * n + p);
    }
#pragma unroll
    for (int q = 0; q < K; q++) {
        const T acc = wa[0] * ldc(xc + (int64_t)c[0] * K + q) + wa[1] * ldc(xc + (int64_t)c[1] * K + q) +
                      wa[2] * ldc(xc + (int64_t)c[2] * K + q);
        x[(int64_t)p * K + q] = ldc(x + (int64_t)p * K + q) + acc;
    }
}

// y = L^-1 b at the coarsest level (one row per unit), b binary64 or binary32.
template <int K>
__device__ __noinline__ void coarse_lo_unit(const ELevel& C, bool in32, int i, int lane) {
    const double* row = C.linv + (int64_t)i * C.np;
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
    for (int j = lane; j <= i; j += 32) {
        const double xv = __ldg(row + j);
#pragma unroll
        for (int q = 0; q < K; q++) {
            const double bv = in32 ? (double)ldc(C.b32 + (int64_t)j * K + q) : ldc(C.b + (int64_t)j * K + q);
            acc[q] += xv * bv;
        }
    }
#pragma unroll
    for (int q = 0; q < K; q++)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) C.y[(int64_t)i * K + q] = acc[q];
}

// x = L^-T y (one row per unit), x binary64 or binary32.
template <int K>
__device__ __noinline__ void coarse_up_unit(const ELevel& C, bool out32, int j, int lane) {
    const double* row = C.linvT + (int64_t)j * C.np;
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
    for (int i = j + lane; i < C.n; i += 32) {
        const double xv = __ldg(row + i);
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] += xv * ldc(C.y + (int64_t)i * K + q);
    }
#pragma unroll
    for (int q = 0; q < K; q++)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) {
            if (out32) C.x32[(int64_t)j * K + q] = (float)acc[q];
            else C.x[(int64_t)j * K + q] = acc[q];
        }
}

// Level-0 residual rows of kUnitsPerResnorm warp slices: partial sums of
// ||b - A x||^2 (and ||b||^2 when init) for this unit, and with r32 the
// binary32 residual (next inner right-hand side) and a zero binary32 iterate.
template <int K, int R>
__device__ __noinline__ void resnorm_unit(const ELevel& L, const Phase& ph, double* part, int u, int lane) {
    double rr[K], bb[K];
#pragma unroll
    for (int q = 0; q < K; q++) rr[q] = bb[q] = 0.0;
    const int w0 = u * kUnitsPerResnorm;
    for (int w = w0; w < w0 + kUnitsPerResnorm && w < L.nslices * R; w++) {
        const SliceMeta m = L.slices[w / R];
        kern::RowSlice<double, K, R, kern::Pre<double, K, R>::value> rs;
        rs.load(m, w % R, lane, L.col, L.sval);
        const bool valid = rs.r < m.nrows;
        const int row = m.row0 + (valid ? rs.r : 0);
        const double d = __ldg(L.diag + row);
        double bv[K], own[K], acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) {
            bv[q] = ldc(L.b + (int64_t)row * K + q);
            own[q] = bv[q] - d * ldc(L.x + (int64_t)row * K + q);
        }
        rs.template dot_from<true>(m, L.col, L.sval, L.x, own, acc);
        if (valid && rs.sub == 0)
#pragma unroll
            for (int q = 0; q < K; q++) {
                rr[q] += acc[q] * acc[q];
                if (ph.a) bb[q] += bv[q] * bv[q];
                if (ph.b) {
                    L.b32[(int64_t)row * K + q] = (float)acc[q];
                    L.x32[(int64_t)row * K + q] = 0.0f;
                }
            }
    }
#pragma unroll
    for (int q = 0; q < K; q++)
        for (int o = 16; o > 0; o >>= 1) {
            rr[q] += __shfl_xor_sync(0xffffffffu, rr[q], o);
            bb[q] += __shfl_xor_sync(0xffffffffu, bb[q], o);
        }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) {
            part[(int64_t)u * 2 * K + q] = rr[q];
            part[(int64_t)u * 2 * K + K + q] = bb[q];
        }
}

// Stopping test of Alg. 1 over the residual-norm partials (fixed order);
// returns the next phase.
template <int K>
__device__ __noinline__ int norm_final_unit(const EMesh& M, const Phase& ph, int nparts, int lane) {
    double acc[2 * K];
#pragma unroll
    for (int q = 0; q < 2 * K; q++) acc[q] = 0.0;
    for (int u = lane; u < nparts; u += 32)
#pragma unroll
        for (int q = 0; q < 2 * K; q++) acc[q] += ldc(M.part + (int64_t)u * 2 * K + q);
#pragma unroll
    for (int q = 0; q < 2 * K; q++)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    int next = ph.c;
    if (lane == 0) {
        SolveState* st = M.st;
        if (ph.a)
            for (int q = 0; q < K; q++) st->bnorm2[q] = acc[K + q];
        double rel = 0.0;
        for (int q = 0; q < K; q++) {
            const double bn = ph.a ? acc[K + q] : ldc(&st->bnorm2[q]);
            const double rq = bn > 0.0 ? sqrt(acc[q] / bn) : sqrt(acc[q]);
            rel = (rq > rel || rq != rq) ? rq : rel;
        }
        const int cycles = ph.a ? 0 : ldc(&st->cycles) + 1;
        if (ph.a) st->rel0 = rel;
        st->cycles = cycles;
        st->rel = rel;
        const bool finite = isfinite(rel);
        const bool converged = finite && rel <= M.rtol;
        const bool more = finite && !converged && cycles < M.max_cycles;
        st->status = converged ? SMG_OK : (!finite ? SMG_ERR_DIVERGED : (more ? -1 : SMG_ERR_NOT_CONVERGED));
        next = more ? ph.b : ph.c;
    }
    return __shfl_sync(0xffffffffu, next, 0);
}

#define SMG_ENG_R(R, CALL)                                   \
    do {                                                     \
        switch (R) {                                         \
            case 1: { constexpr int RR = 1; CALL; } break;   \
            case 2: { constexpr int RR = 2; CALL; } break;   \
            case 4: { constexpr int RR = 4; CALL; } break;   \
            case 8: { constexpr int RR = 8; CALL; } break;   \
            default: { constexpr int RR = 16; CALL; } break; \
        }                                                    \
    } while (0)

// One unit of phase p of mesh m; returns the phase that follows when this unit
// is the phase's last (-1: the phase's default successor p + 1).
template <int K>
__device__ int run_unit(const EMesh& M, const Phase& ph, int u, int lane) {
    const ELevel& L = M.lv[ph.level];
    switch (ph.type) {
        case kGatherIn:
        case kScatterOut: {
            const int64_t m = (int64_t)M.n0 * K;
            for (int64_t e = (int64_t)u * kElemsPerUnit + lane; e < m && e < (int64_t)(u + 1) * kElemsPerUnit; e += 32) {
                const int64_t p = e / K, q = e - p * K;
                const int64_t src = (int64_t)__ldg(M.perm0 + p) * K + q;
                if (ph.type == kGatherIn) {
                    L.b[e] = ldc(M.b_user + src);
                    L.x[e] = ldc(M.x_user + src);
                } else {
                    M.x_user[src] = ldc(L.x + e);
                }
            }
            break;
        }
        case kResnorm: SMG_ENG_R(ph.c, (resnorm_unit<K, RR>(L, ph, M.part, u, lane))); break;
        case kNormFinal: return norm_final_unit<K>(M, ph, ph.d, lane);
        case kGs:
            if (ph.prec) SMG_ENG_R(ph.c, (gs_unit<float, K, RR>(L, ph, u, lane)));
            else SMG_ENG_R(ph.c, (gs_unit<double, K, RR>(L, ph, u, lane)));
            break;
        case kRestrict:
            if (ph.prec) SMG_ENG_R(ph.c, (restrict_unit<float, K, RR>(L, M.lv[ph.level + 1], ph, u, lane)));
            else SMG_ENG_R(ph.c, (restrict_unit<double, K, RR>(L, M.lv[ph.level + 1], ph, u, lane)));
            break;
        case kCoarseLo: coarse_lo_unit<K>(L, ph.prec != 0, u, lane); break;
        case kCoarseUp: coarse_up_unit<K>(L, ph.prec != 0, u, lane); break;
        case kProlong:
            if (ph.prec) prolong_unit<float, K>(L, M.lv[ph.level + 1], u, lane);
            else prolong_unit<double, K>(L, M.lv[ph.level + 1], u, lane);
            break;
        case kIrUpdate: {
            const int64_t m = (int64_t)M.n0 * K;
            for (int64_t e = (int64_t)u * kElemsPerUnit + lane; e < m && e < (int64_t)(u + 1) * kElemsPerUnit; e += 32)
                L.x[e] = ldc(L.x + e) + (double)ldc(L.x32 + e);
            break;
        }
        default: break;
    }
    return -1;
}

// Acquire-release fence at device scope: orders this thread's (and, through
// the warp barriers around it, its warp's) memory operations against the
// scheduling atomics; lighter than a sequentially consistent fence.
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ long long globaltimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int K, int MINB>
__global__ void __launch_bounds__(256, MINB) engine(const EMesh* __restrict__ meshes, int nmesh,
                                                   const int32_t* __restrict__ home, ECtl* ctl, int* finished,
                                                   int* err, long long idle_limit_ns) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (gw == 0 && lane == 0) meshes[0].trace[0] = globaltimer();
    // every warp serves one mesh (warps dealt to meshes in proportion to their
    // unknowns, so polling is spread over the meshes' control words); when
    // that mesh is done it moves on to the next mesh that is not
    int m = home[gw];
    int visit = (m + 1 + gw % max(nmesh - 1, 1)) % nmesh;  // mesh to help while the own one has nothing to hand out
    long long idle_since = 0;
    int backoff = 32;
    for (;;) {
        int p = 0, u = 0, got = 0, moved = 0, stop = 0, cur = m;
        if (lane == 0) {
            // take a unit of mesh c if its current phase has one left
            auto take = [&](int c) {
                const EMesh& M = meshes[c];
                const unsigned long long tw = *(volatile unsigned long long*)&ctl[c].ticket;
                const int pp = (int)(tw >> 32), uu = (int)(tw & 0xffffffffu);
                if (pp >= M.nphase || uu >= M.prog[pp].units) return pp >= M.nphase ? 2 : 0;
                const unsigned long long old = atomicAdd(&ctl[c].ticket, 1ull);
                const int p2 = (int)(old >> 32), u2 = (int)(old & 0xffffffffu);
                if (p2 < M.nphase && u2 < M.prog[p2].units) {
                    p = p2;
                    u = u2;
                    cur = c;
                    fence_acq_rel();  // acquire: the phase's inputs, published before the ticket
                    return 1;
                }
                return 0;
            };
            const int r = take(m);
            if (r == 1) {
                got = 1;
            } else if (r == 2) {  // this mesh is done
                if (*(volatile int*)finished >= nmesh || *(volatile int*)err) stop = 1;
                else {
                    m = (m + 1) % nmesh;
                    moved = 1;
                }
            } else if (nmesh > 1) {  // help another mesh for one unit
                if (visit == m) visit = (visit + 1) % nmesh;
                got = take(visit) == 1;
                visit = (visit + 1) % nmesh;
            }
            if (!got && !moved && !stop) {
                if (*(volatile int*)err) stop = 1;
                const long long now = globaltimer();
                if (idle_since == 0) idle_since = now;
                else if (now - idle_since > idle_limit_ns) atomicExch(err, 1);
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return;
        m = __shfl_sync(0xffffffffu, m, 0);
        cur = __shfl_sync(0xffffffffu, cur, 0);
        if (__shfl_sync(0xffffffffu, moved, 0)) continue;
        if (!__shfl_sync(0xffffffffu, got, 0)) {
            __nanosleep(backoff);
            backoff = min(backoff * 2, 512);
            continue;
        }
        p = __shfl_sync(0xffffffffu, p, 0);
        u = __shfl_sync(0xffffffffu, u, 0);
        __syncwarp();  // order the lanes' reads after lane 0's acquire
        idle_since = 0;
        backoff = 32;
        const EMesh& M = meshes[cur];
        const Phase ph = M.prog[p];
        const int next = run_unit<K>(M, ph, u, lane);
        fence_acq_rel();  // release: this unit's results before its completion count
        __syncwarp();
        if (lane == 0) {
            const unsigned int d = atomicAdd(&ctl[cur].done, 1u);
            if (d + 1 == (unsigned int)ph.units) {  // last unit: advance the mesh
                fence_acq_rel();
                const int np = next >= 0 ? next : p + 1;
                atomicExch(&ctl[cur].done, 0u);
                fence_acq_rel();
                atomicExch(&ctl[cur].ticket, (unsigned long long)np << 32);
                if (np >= M.nphase) {
                    M.trace[1 + cur] = globaltimer();
                    atomicAdd(finished, 1);
                }
            }
        }
        __syncwarp();
    }
}

}  // namespace eng

// ---------------------------------------------------------------- host side
// Dispatch on the right-hand-side count and the blocks per SM of the engine.
#define SMG_ENG_K(K, MINB, CALL)                                                             \
    do {                                                                                     \
        if ((MINB) >= 4) {                                                                   \
            constexpr int MB = 4;                                                            \
            switch (K) {                                                                     \
                case 1: { constexpr int KK = 1; CALL; } break;                               \
                case 2: { constexpr int KK = 2; CALL; } break;                               \
                case 3: { constexpr int KK = 3; CALL; } break;                               \
                default: { constexpr int KK = 4; CALL; } break;                              \
            }                                                                                \
        } else {                                                                             \
            constexpr int MB = 2;                                                            \
            switch (K) {                                                                     \
                case 1: { constexpr int KK = 1; CALL; } break;                               \
                case 2: { constexpr int KK = 2; CALL; } break;                               \
                case 3: { constexpr int KK = 3; CALL; } break;                               \
                default: { constexpr int KK = 4; CALL; } break;                              \
            }                                                                                \
        }                                                                                    \
    } while (0)

constexpr int kEngineBlocksPerSm = 4;

struct BatchEngine {
    std::vector<void*> allocs;
    eng::EMesh* meshes = nullptr;
    eng::ECtl* ctl = nullptr;
    int* counters = nullptr;      // finished meshes at [0], error flag at [32]
    SolveState* states = nullptr;  // every mesh's solve state after the launch, contiguous
    long long* trace = nullptr;    // launch start and every mesh's finish time (globaltimer)
    int32_t* home = nullptr;       // mesh served by each warp of the launch
    int nmesh = 0, K = 1, grid = 0, minb = 2;
    long long idle_ns = 0;         // a warp that finds no unit for this long reports a timeout
};

namespace {

template <class T>
T* eng_alloc(BatchEngine* E, int64_t count) {
    if (count <= 0) count = 1;
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (size_t)count) != cudaSuccess) throw std::runtime_error("cudaMalloc");
    E->allocs.push_back(p);
    return (T*)p;
}

template <class T>
T* eng_upload(BatchEngine* E, const std::vector<T>& v) {
    T* p = eng_alloc<T>(E, (int64_t)v.size());
    if (!v.empty() && cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        throw std::runtime_error("cudaMemcpy");
    return p;
}

// The solve of one mesh as a phase list (Alg. 1 loop around Alg. 2).
std::vector<eng::Phase> mesh_program(const smg_hierarchy* h, int K, bool mixed) {
    using namespace eng;
    std::vector<Phase> prog;
    const int H = h->H;
    const int prec = mixed ? 1 : 0;
    const DLevel& L0 = h->L[0];
    auto add = [&](int type, int level, int64_t units, int a = 0, int b = 0, int c = 0) {
        Phase ph{};
        ph.type = type;
        ph.level = level;
        ph.units = (int32_t)units;
        ph.prec = prec;
        ph.a = a;
        ph.b = b;
        ph.c = c;

        if (units > 0) prog.push_back(ph);
        return (int)prog.size() - 1;
    };
    const int64_t vec_units = (L0.n * K + kElemsPerUnit - 1) / kElemsPerUnit;
    const int64_t rn_units = ((int64_t)L0.nslices * L0.R + kUnitsPerResnorm - 1) / kUnitsPerResnorm;
    add(kGatherIn, 0, vec_units);
    add(kResnorm, 0, rn_units, 1, mixed ? 1 : 0, L0.R);
    const int init_final = add(kNormFinal, 0, 1, 1);
    const int cycle0 = (int)prog.size();
    auto lanes = [&](const DLevel& L) { return mixed ? L.R32 : L.R; };
    auto rq_lanes = [&](const DLevel& L) { return mixed ? L.Rq32 : L.Rq; };
    auto seeded = [&](int l) { return h->opts.mu_pre > 0 && l >= 1 && l < H && h->L[l].seed_rows > 0; };
    auto sweep = [&](int l, bool reverse, int first) {
        const DLevel& L = h->L[l];
        const int R = lanes(L);
        for (int cc = first; cc < L.ncolours; cc++) {
            const int c = reverse ? L.ncolours - 1 - cc : cc;
            const int s0 = L.colour_slice[c], s1 = L.colour_slice[c + 1];
            add(kGs, l, (int64_t)(s1 - s0) * R, s0, s1 - s0, R);
        }
    };
    for (int l = 0; l < H; l++) {
        for (int it = 0; it < h->opts.mu_pre; it++) sweep(l, false, (it == 0 && seeded(l)) ? 1 : 0);
        const DLevel& L = h->L[l];
        add(kRestrict, l, (int64_t)L.rq_nslices * rq_lanes(L), seeded(l + 1) ? h->L[l + 1].seed_rows : 0, 0,
            rq_lanes(L));
    }
    add(kCoarseLo, H, h->L[H].n);
    add(kCoarseUp, H, h->L[H].n);
    for (int l = H - 1; l >= 0; l--) {
        add(kProlong, l, (h->L[l].n + 31) / 32);
        for (int it = 0; it < h->opts.mu_post; it++) sweep(l, h->opts.post_reverse != 0, 0);
    }
    if (mixed) add(kIrUpdate, 0, vec_units);
    add(kResnorm, 0, rn_units, 0, mixed ? 1 : 0, L0.R);
    const int final_ = add(kNormFinal, 0, 1, 0);
    const int exit_ = add(kScatterOut, 0, vec_units);
    for (int f : {init_final, final_}) {
        prog[f].b = cycle0;
        prog[f].c = exit_;
        prog[f].d = (int32_t)rn_units;  // partials the stopping test sums
    }
    return prog;
}

__global__ void copy_states(const eng::EMesh* __restrict__ meshes, int nmesh, SolveState* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nmesh) out[i] = *meshes[i].st;
}

}  // namespace

bool engine_supported(const smg_batch* B) {
    for (const smg_hierarchy* h : B->hs)
        if (h->H < 1 || h->opts.smoother != SMG_SMOOTHER_GS || h->opts.solver != SMG_SOLVER_VCYCLE ||
            h->opts.block_size != 1)
            return false;
    return true;
}

BatchEngine* engine_create(smg_batch* B, int K, bool mixed) {
    BatchEngine* E = new BatchEngine();
    try {
        E->nmesh = (int)B->hs.size();
        E->K = K;
        E->idle_ns = B->wait_ns;
        std::vector<eng::EMesh> meshes(E->nmesh);
        for (int i = 0; i < E->nmesh; i++) {
            smg_hierarchy* h = B->hs[i];
            std::vector<eng::Phase> prog = mesh_program(h, K, mixed);
            std::vector<eng::ELevel> lv(h->H + 1);
            for (int l = 0; l <= h->H; l++) {
                DLevel& L = h->L[l];
                eng::ELevel& e = lv[l];
                e = eng::ELevel{};
                e.slices = L.slices;
                e.col = L.sell_col;
                e.sval = L.vals ? L.vals + L.sbase : nullptr;
                e.sval32 = L.vals32 ? L.vals32 + L.sbase : nullptr;
                e.diag = L.vals;
                e.dinv = L.dinv;
                e.dinv32 = L.dinv32;
                e.x = L.x;
                e.b = L.b;
                e.x32 = L.x32;
                e.b32 = L.b32;
                e.rq = L.rq_slices;
                e.rq_row = L.rq_row;
                e.rq_col = L.rq_col;
                e.rq_val = L.rq_val;
                e.rq_val32 = L.rq_val32;
                e.p_idx = L.p_idx;
                e.p_w = L.p_w;
                e.p_w32 = L.p_w32;
                e.linv = L.linv;
                e.linvT = L.linvT;
                e.y = L.y;
                e.np = L.np;
                e.n = (int32_t)L.n;
                e.nslices = L.nslices;
            }
            eng::EMesh& M = meshes[i];
            M.prog = eng_upload(E, prog);
            M.lv = eng_upload(E, lv);
            M.b_user = B->stage_b + B->uoff[i] * K;
            M.x_user = B->stage_x + B->uoff[i] * K;
            M.perm0 = h->perm0;
            M.st = h->state;
            int32_t nparts = 1;
            for (const eng::Phase& ph : prog)
                if (ph.type == eng::kNormFinal) nparts = ph.d;
            M.part = eng_alloc<double>(E, (int64_t)nparts * 2 * K);
            M.rtol = h->opts.rtol;
            M.nphase = (int32_t)prog.size();
            M.H = h->H;
            M.n0 = (int32_t)h->L[0].n;
            M.max_cycles = h->opts.max_cycles;
        }
        E->trace = eng_alloc<long long>(E, 1 + E->nmesh);
        for (auto& M : meshes) M.trace = E->trace;
        E->meshes = eng_upload(E, meshes);
        E->ctl = eng_alloc<eng::ECtl>(E, E->nmesh);
        E->counters = eng_alloc<int>(E, 64);  // finished at [0], error flag at [32]: separate lines
        E->states = eng_alloc<SolveState>(E, E->nmesh);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // blocks of 8 warps per SM: 4 (64 registers a thread; 85 ms for the 64-mesh
        // batch against 95 ms with 2 blocks of 128 registers); SMG_ENGINE_BLOCKS_PER_SM
        // overrides (a measurement aid)
        E->minb = kEngineBlocksPerSm;
        if (const char* env = std::getenv("SMG_ENGINE_BLOCKS_PER_SM")) E->minb = std::atoi(env) >= 4 ? 4 : 2;
        cudaError_t occ = cudaSuccess;
        SMG_ENG_K(E->K, E->minb, occ = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eng::engine<KK, MB>, 256, 0));
        if (occ != cudaSuccess || per_sm < 1) throw std::runtime_error("engine occupancy");
        E->grid = sms * std::min(per_sm, E->minb);
        // warps dealt to meshes in proportion to their unknowns (at least one each)
        const int W = E->grid * 8;
        std::vector<double> w(E->nmesh);
        double tot = 0.0;
        for (int i = 0; i < E->nmesh; i++) tot += (w[i] = (double)B->hs[i]->L[0].n);
        std::vector<int32_t> home(W, 0);
        std::vector<int> share(E->nmesh, 1);
        int left = W - E->nmesh;
        if (left < 0) left = 0;
        std::vector<double> frac(E->nmesh);
        int given = 0;
        for (int i = 0; i < E->nmesh; i++) {
            const double want = left * w[i] / tot;
            share[i] += (int)want;
            given += (int)want;
            frac[i] = want - (int)want;
        }
        std::vector<int> order(E->nmesh);
        for (int i = 0; i < E->nmesh; i++) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return frac[a] > frac[b]; });
        for (int k = 0; k < left - given; k++) share[order[k % E->nmesh]]++;
        for (int i = 0, g = 0; i < E->nmesh; i++)  // interleaved: warp g of the launch serves mesh home[g]
            for (int k = 0; k < share[i] && g < W; k++) home[g++] = i;
        std::vector<int32_t> dealt(W);
        for (int g = 0; g < W; g++) dealt[g] = home[(int64_t)g * 7919 % W];  // spread a mesh's warps over SMs
        E->home = eng_upload(E, W % 7919 == 0 ? home : dealt);
    } catch (...) {
        engine_destroy(E);
        throw;
    }
    return E;
}

void engine_destroy(BatchEngine* E) {
    if (!E) return;
    for (void* p : E->allocs) cudaFree(p);
    delete E;
}


cudaError_t engine_record(BatchEngine* E, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(E->ctl, 0, sizeof(eng::ECtl) * E->nmesh, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(E->counters, 0, sizeof(int) * 64, s);
    if (e != cudaSuccess) return e;
    const dim3 grid(E->grid), block(256);
    SMG_ENG_K(E->K, E->minb,
              (eng::engine<KK, MB><<<grid, block, 0, s>>>(E->meshes, E->nmesh, E->home, E->ctl, E->counters,
                                                           E->counters + 32, E->idle_ns)));
    copy_states<<<(E->nmesh + 127) / 128, 128, 0, s>>>(E->meshes, E->nmesh, E->states);
    return cudaGetLastError();
}

const int* engine_error_flag(const BatchEngine* E) { return E->counters + 32; }
const SolveState* engine_states(const BatchEngine* E) { return E->states; }

// With SMG_TRACE_ENGINE set: the finish time of every mesh after the launch
// start, and the solve's cycles per mesh (stderr).  Synchronous; a tracing aid.
void engine_trace(const BatchEngine* E, const SolveState* host_states) {
    if (!std::getenv("SMG_TRACE_ENGINE")) return;
    std::vector<long long> t(1 + E->nmesh);
    if (cudaMemcpy(t.data(), E->trace, sizeof(long long) * t.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return;
    std::vector<double> us(E->nmesh);
    for (int i = 0; i < E->nmesh; i++) us[i] = (t[1 + i] - t[0]) * 1e-3;
    for (int i = 0; i < E->nmesh; i++)
        std::fprintf(stderr, "[smg engine] mesh %d finished at %.1f us (%d cycles)\n", i, us[i], host_states[i].cycles);
}
int engine_grid(const BatchEngine* E) { return E->grid; }

}  // namespace smg
