// Coarsest level of Alg. 2 ("solve A x = b", direct): a dense binary64
// Cholesky factor A_H = L L^T computed once per update, then the inverse factor
// X = L^{-1} and its transpose, so that each cycle's direct solve
// x = L^{-T} (L^{-1} b) is two dense triangular products spread over the whole
// GPU instead of two serial substitutions.
//
// Blocked right-looking algorithms with 32 x 32 tiles; the matrix is padded to
// a multiple of 32 with an identity block.
#include <algorithm>
#include <stdexcept>
#include <string>

#include "device.hpp"

namespace smg {
namespace {

constexpr int NB = kDenseNB;

__global__ void k_pad_copy(const double* __restrict__ A, int64_t n, double* __restrict__ C, double* __restrict__ X,
                           int64_t np) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np * np) return;
    int64_t i = e / np, j = e % np;
    double v = (i < n && j < n) ? A[i * n + j] : (i == j ? 1.0 : 0.0);
    C[e] = v;
    X[e] = (i == j) ? 1.0 : 0.0;
}

// Reciprocal square root on the pivot chain (a positive binary64 pivot): a
// binary32 estimate y0 (the leading bits of a moved into a float by integer
// operations, one rsqrtf), then one second-order correction from the binomial
// series of (1 - e)^(-1/2): y = y0 (1 + e/2 + 3 e^2 / 8) with e = 1 - a y0^2,
// whose truncation error (~5 e^3 / 16, e < 2^-20) is far below binary64
// rounding.  Four dependent binary64 operations: on this part a dependent
// chain through it takes ~430 clocks against ~890 through rsqrt(), within one
// unit in the last place of the exact value (measured against a quad-precision
// reference over 2^20 arguments).  Outside the range a float holds (and for a
// non-positive or non-finite pivot) it returns rsqrt(a).
__device__ __forceinline__ double rsqrt_pivot(double a) {
    const int hi = __double2hiint(a);
    const unsigned lo = (unsigned)__double2loint(a);
    const int ex = (hi >> 20) & 0x7ff;  // biased binary64 exponent; binary32 exponent = ex - 896
    if (hi < 0 || ex < 898 || ex > 1149) return rsqrt(a);
    const unsigned fb = ((unsigned)(ex - 896) << 23) | (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
    const int yhi = (int)(((((yb >> 23) & 0xffu) + 896u) << 20) | ((yb & 0x7fffffu) >> 3));
    const double y0 = __hiloint2double(yhi, (int)(yb << 29));
    const double e = fma(-(a * y0), y0, 1.0);
    return fma(y0 * e, fma(0.375, e, 0.5), y0);
}

// Factor diagonal tile j.  A binary64 instruction holds its warp for about 64
// clocks on this part (dependent or not), so the pivot chain (shuffle,
// rsqrt_pivot, scale) sets the time and everything else is kept off it:
// warp w holds columns c = w, w + 8, ... of the tile in registers (lane = row);
// in step k the owner of column k + 1 applies pivot k to that column only,
// factors it (pivot k + 1) and publishes it in shared memory, while every other
// warp applies pivot k to its columns right of k + 1 (lower triangle).  The
// owner catches up on pivot k in step k + 1, so the published columns rotate
// over three buffers and one barrier per pivot suffices.
constexpr int kDiagWarps = 8;
// Dynamic shared memory the diagonal-tile kernel requests beyond its own
// arrays, so that no other block fits beside it: the kernel is bound by its
// dependent binary64 chain, and a trailing-update block on the same SM would
// take the SM's binary64 issue from it.
constexpr int kDiagExclusiveSmem = 212 * 1024;
constexpr int kDiagCols = NB / kDiagWarps;
__global__ void __launch_bounds__(32 * kDiagWarps) k_chol_diag(double* __restrict__ C, int64_t np, int j,
                                                                double* __restrict__ rinv_out,
                                                                int32_t* __restrict__ bad) {
    __shared__ double a[NB][NB + 1];
    __shared__ double lk[3][NB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double* T = C + (int64_t)j * NB * np + (int64_t)j * NB;
    for (int e = threadIdx.x; e < NB * NB; e += 32 * kDiagWarps) a[e / NB][e % NB] = T[(int64_t)(e / NB) * np + e % NB];
    __syncthreads();
    double col[kDiagCols];  // col[m] = a[lane][m * kDiagWarps + w]
#pragma unroll
    for (int m = 0; m < kDiagCols; m++) col[m] = a[lane][m * kDiagWarps + w];
    // column p (owned by this warp) becomes column p of L: l = a / sqrt(a_pp),
    // on lane p itself sqrt(a_pp).  No test on the pivot chain: a pivot that is
    // not positive gives a NaN or an infinity that the check of the diagonal
    // after the loop reports.
    auto pivot = [&](double& cp, int p) {
        const double y = rsqrt_pivot(__shfl_sync(0xffffffffu, cp, p));
        const double l = cp * y;
        if (lane >= p) cp = l;
        lk[p % 3][lane] = l;
        if (lane == p) rinv_out[(int64_t)j * NB + p] = y;
    };
    if (w == 0) pivot(col[0], 0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k + 1 < NB; k++) {
        const double lr = lk[k % 3][lane];
        if (w == (k + 1) % kDiagWarps) {
            const int m1 = (k + 1) / kDiagWarps;
            if (lane >= k + 1) col[m1] -= lr * lk[k % 3][k + 1];
            pivot(col[m1], k + 1);
        } else {
            const bool late = k > 0 && w == k % kDiagWarps;  // owner of column k: pivot k - 1 still to apply
            const double lp = late ? lk[(k + 2) % 3][lane] : 0.0;
#pragma unroll
            for (int m = 0; m < kDiagCols; m++) {
                const int c = m * kDiagWarps + w;
                if (c > k + 1 && lane >= c) {
                    if (late) col[m] -= lp * lk[(k + 2) % 3][c];
                    col[m] -= lr * lk[k % 3][c];
                }
            }
        }
        __syncthreads();
    }
    bool flagged = false;  // not SPD: a diagonal entry of L that is not positive and finite
#pragma unroll
    for (int m = 0; m < kDiagCols; m++) {
        const int c = m * kDiagWarps + w;
        if (lane == c && !(col[m] > 0.0 && isfinite(col[m]))) flagged = true;
        T[(int64_t)lane * np + c] = (c <= lane) ? col[m] : 0.0;
    }
    if (flagged) atomicExch(bad, 1);
}

// Inverse of diagonal tile j (X = L_jj^{-1}, forward elimination of L X = I):
// columns are independent, so eight blocks of four warps take one column per
// warp (each binary64 instruction holds its warp, so one column per warp is
// the shortest chain); lane = row, the row-k value arrives by shuffle.
constexpr int kInvBlocks = NB / 4;
__global__ void __launch_bounds__(128) k_tile_inv(const double* __restrict__ C, int64_t np, int j,
                                                  const double* __restrict__ rinv, double* __restrict__ dblk) {
    __shared__ double l[NB][NB + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double* T = C + (int64_t)j * NB * np + (int64_t)j * NB;
    for (int e = threadIdx.x; e < NB * NB; e += 128) l[e / NB][e % NB] = T[(int64_t)(e / NB) * np + e % NB];
    __syncthreads();
    const int c0 = blockIdx.x * 4 + w;  // this warp's column
    double x0 = (lane == c0) ? 1.0 : 0.0;
    const double ri = rinv[(int64_t)j * NB + lane];
    for (int k = c0; k < NB; k++) {
        // row k of the column is final after scaling; broadcast it
        const double k0 = __shfl_sync(0xffffffffu, x0 * ri, k);
        if (lane == k) x0 = k0;
        else if (lane > k) x0 -= l[lane][k] * k0;
    }
    dblk[(int64_t)j * NB * NB + lane * NB + c0] = (lane >= c0) ? x0 : 0.0;
}

// Work units of the tile kernels: a 32 x 32 output tile split into kQ blocks of
// 32 / kQ rows (binary64 throughput is per SM, so more SMs per tile).
constexpr int kQ = 4;
constexpr int kQR = NB / kQ;

// L_ij = A_ij L_jj^{-T} for the tiles below the diagonal tile j.
__global__ void __launch_bounds__(kQR * NB) k_chol_panel(double* __restrict__ C, int64_t np, int j,
                                                         const double* __restrict__ dblk) {
    __shared__ double a[kQR][NB + 1];
    __shared__ double d[NB][NB + 1];
    const int i = j + 1 + blockIdx.x / kQ, q0 = (blockIdx.x % kQ) * kQR;
    const int rl = threadIdx.x / NB, c = threadIdx.x % NB;
    double* T = C + ((int64_t)i * NB + q0) * np + (int64_t)j * NB;
    a[rl][c] = T[(int64_t)rl * np + c];
#pragma unroll
    for (int q = 0; q < kQ; q++) d[rl + kQR * q][c] = dblk[(int64_t)j * NB * NB + (rl + kQR * q) * NB + c];
    __syncthreads();
    double s[4] = {0.0, 0.0, 0.0, 0.0};  // four independent partial sums
    for (int k = 0; k <= c; k++) s[k & 3] += a[rl][k] * d[c][k];
    T[(int64_t)rl * np + c] = (s[0] + s[1]) + (s[2] + s[3]);
}

__device__ __forceinline__ void tri_index(int b, int& ii, int& kk) {
    int t = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
    while ((t + 1) * (t + 2) / 2 <= b) t++;
    while (t * (t + 1) / 2 > b) t--;
    ii = t;
    kk = b - t * (t + 1) / 2;
}

// Trailing update A_ik -= L_ij L_kj^T for first <= k <= i (tiles of the
// triangle from block `first` on; first = j + 1 is the whole trailing matrix).
__global__ void __launch_bounds__(kQR * NB) k_chol_update(double* __restrict__ C, int64_t np, int j, int first) {
    __shared__ double li[kQR][NB + 1];
    __shared__ double lk[NB][NB + 1];
    int ii, kk;
    tri_index(blockIdx.x / kQ, ii, kk);
    const int q0 = (blockIdx.x % kQ) * kQR;
    const int i = first + ii, k = first + kk;
    const int rl = threadIdx.x / NB, c = threadIdx.x % NB;
    li[rl][c] = C[((int64_t)i * NB + q0 + rl) * np + (int64_t)j * NB + c];
#pragma unroll
    for (int q = 0; q < kQ; q++) lk[rl + kQR * q][c] = C[((int64_t)k * NB + rl + kQR * q) * np + (int64_t)j * NB + c];
    __syncthreads();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < NB; q++) s[q & 3] += li[rl][q] * lk[c][q];
    C[((int64_t)i * NB + q0 + rl) * np + (int64_t)k * NB + c] -= (s[0] + s[1]) + (s[2] + s[3]);
}

// Look-ahead part of the trailing update: block column k = j + 1 only
// (A_i,j+1 -= L_ij L_j+1,j^T for i >= j + 1), which is all the next diagonal
// tile and panel need.
__global__ void __launch_bounds__(kQR * NB) k_chol_update_col(double* __restrict__ C, int64_t np, int j) {
    __shared__ double li[kQR][NB + 1];
    __shared__ double lk[NB][NB + 1];
    const int i = j + 1 + blockIdx.x / kQ, k = j + 1;
    const int q0 = (blockIdx.x % kQ) * kQR;
    const int rl = threadIdx.x / NB, c = threadIdx.x % NB;
    li[rl][c] = C[((int64_t)i * NB + q0 + rl) * np + (int64_t)j * NB + c];
#pragma unroll
    for (int q = 0; q < kQ; q++) lk[rl + kQR * q][c] = C[((int64_t)k * NB + rl + kQR * q) * np + (int64_t)j * NB + c];
    __syncthreads();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < NB; q++) s[q & 3] += li[rl][q] * lk[c][q];
    C[((int64_t)i * NB + q0 + rl) * np + (int64_t)k * NB + c] -= (s[0] + s[1]) + (s[2] + s[3]);
}

// Block row i of X = L^{-1}: X_i,jb = L_ii^{-1} B_i,jb for jb <= i (B accumulates
// I - sum L X).  In place, so one block per tile (rows depend on earlier rows).
__global__ void __launch_bounds__(NB * NB) k_trinv_row(double* __restrict__ X, int64_t np, int i,
                                                       const double* __restrict__ dblk) {
    __shared__ double bs[NB][NB + 1];
    __shared__ double d[NB][NB + 1];
    const int jb = blockIdx.x;
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    double* T = X + (int64_t)i * NB * np + (int64_t)jb * NB;
    bs[r][c] = T[(int64_t)r * np + c];
    d[r][c] = dblk[(int64_t)i * NB * NB + r * NB + c];
    __syncthreads();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q <= r; q++) s[q & 3] += d[r][q] * bs[q][c];
    T[(int64_t)r * np + c] = (s[0] + s[1]) + (s[2] + s[3]);
}

// B_k,jb -= L_k,i X_i,jb for k > i, jb <= i (output rows split over kQ blocks;
// the tiles read are not written by this kernel).
// The inverse factor is off the critical path of the factorisation, so its
// products run on at most kInvCtas blocks (grid-stride over the work units):
// fewer SMs then share their binary64 unit with the diagonal-tile kernel.
constexpr int kInvCtas = 128;  // measured on the 1M torus: 64 leaves the inverse last, uncapped slows the diagonal tiles
__global__ void __launch_bounds__(kQR * NB) k_trinv_update(double* __restrict__ X, const double* __restrict__ C,
                                                           int64_t np, int i, int nunits) {
    __shared__ double l[kQR][NB + 1];
    __shared__ double xs[NB][NB + 1];
    const int rl = threadIdx.x / NB, c = threadIdx.x % NB;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int t = u / kQ, q0 = (u % kQ) * kQR;
        const int k = i + 1 + t / (i + 1);
        const int jb = t % (i + 1);
        l[rl][c] = C[((int64_t)k * NB + q0 + rl) * np + (int64_t)i * NB + c];
#pragma unroll
        for (int q = 0; q < kQ; q++)
            xs[rl + kQR * q][c] = X[((int64_t)i * NB + rl + kQR * q) * np + (int64_t)jb * NB + c];
        __syncthreads();
        double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < NB; q++) s[q & 3] += l[rl][q] * xs[q][c];
        X[((int64_t)k * NB + q0 + rl) * np + (int64_t)jb * NB + c] -= (s[0] + s[1]) + (s[2] + s[3]);
        __syncthreads();  // the tiles in shared memory are reloaded for the next unit
    }
}

__global__ void k_transpose(const double* __restrict__ X, double* __restrict__ XT, int64_t np) {
    __shared__ double t[NB][NB + 1];
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    t[r][c] = X[((int64_t)bi * NB + r) * np + (int64_t)bj * NB + c];
    __syncthreads();
    XT[((int64_t)bj * NB + r) * np + (int64_t)bi * NB + c] = t[c][r];
}

template <int K, bool IN32>
__global__ void k_coarse_lower(const double* __restrict__ X, int64_t np, int n, const void* __restrict__ in,
                               double* __restrict__ y) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const double* row = X + (int64_t)i * np;
    // the factor does not change within a cycle: pull the row into L2 while the
    // grid waits for its predecessor (launched early, it waits through the
    // whole down-sweep below)
    for (int c = lane * 16; c <= i; c += 32 * 16) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + c));
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
#pragma unroll 8
    for (int j = lane; j <= i; j += 32) {
        double xv = row[j];
#pragma unroll
        for (int q = 0; q < K; q++) {
            double bv = IN32 ? (double)((const float*)in)[j * K + q] : ((const double*)in)[j * K + q];
            acc[q] += xv * bv;
        }
    }
#pragma unroll
    for (int q = 0; q < K; q++)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) y[i * K + q] = acc[q];
}

template <int K, bool OUT32>
__global__ void k_coarse_upper(const double* __restrict__ XT, int64_t np, int n, const double* __restrict__ y,
                               void* __restrict__ out) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const double* row = XT + (int64_t)j * np;
    for (int c = (j & ~15) + lane * 16; c < n; c += 32 * 16) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + c));
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
#pragma unroll 8
    for (int i = j + lane; i < n; i += 32) {
        double xv = row[i];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] += xv * y[i * K + q];
    }
#pragma unroll
    for (int q = 0; q < K; q++)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) {
            if (OUT32) ((float*)out)[j * K + q] = (float)acc[q];
            else ((double*)out)[j * K + q] = acc[q];
        }
}

template <int K>
void coarse_solve_k(DLevel& C, const void* in, bool in32, void* out, bool out32, cudaStream_t s) {
    const int n = (int)C.n;
    const dim3 grid((n + 7) / 8), block(256);
    const double* linv = C.linv;
    const double* linvT = C.linvT;
    const double* y = C.y;
    const int64_t np = C.np;
    if (in32) launch_pdl(k_coarse_lower<K, true>, grid, block, s, linv, np, n, in, C.y);
    else launch_pdl(k_coarse_lower<K, false>, grid, block, s, linv, np, n, in, C.y);
    if (out32) launch_pdl(k_coarse_upper<K, true>, grid, block, s, linvT, np, n, y, out);
    else launch_pdl(k_coarse_upper<K, false>, grid, block, s, linvT, np, n, y, out);
}

void ck_dense(cudaError_t e, const char* what) {
    if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
}

// Launch on the critical path of the factorisation, with the greatest stream
// priority (graphs holding it are instantiated to honour node priorities): the
// block scheduler then dispatches its blocks ahead of pending blocks of the
// trailing updates and inverse products.
template <typename... Params, typename... Args>
void launch_crit(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int prio,
                 Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ck_dense(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...), "factor launch");
}

}  // namespace

void record_coarsest_factor(smg_hierarchy* h, cudaStream_t s, bool alone) {
    DLevel& C = h->L[h->H];
    const int64_t np = C.np;
    const int nb = (int)(np / NB);
    // Cholesky steps on `s`; block row j of the inverse factor needs only diagonal
    // tile j and panel j, so the inverse runs on a second stream one step behind
    cudaStream_t s2 = h->aux, s3 = h->aux2;
    k_pad_copy<<<(unsigned)((np * np + 255) / 256), 256, 0, s>>>(C.vals, C.n, C.chol, C.linv, np);
    // look-ahead: after panel j the main stream updates only block column j + 1
    // (what diagonal tile j + 1 and panel j + 1 need); the rest of the trailing
    // update runs on s3, one step behind, and the main stream waits for it only
    // before it next touches those tiles
    bool forked3 = false;  // s3 joins the captured work only once it has some
    int lo = 0, prio = 0;
    ck_dense(cudaDeviceGetStreamPriorityRange(&lo, &prio), "priority range");
    ck_dense(cudaFuncSetAttribute(k_chol_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, kDiagExclusiveSmem),
             "diagonal kernel attribute");
    for (int j = 0; j < nb; j++) {
        launch_crit(k_chol_diag, dim3(1), dim3(32 * kDiagWarps), alone ? (size_t)kDiagExclusiveSmem : 0, s, prio,
                    C.chol, np, j, C.rinv, &h->state->chol_bad);
        launch_crit(k_tile_inv, dim3(kInvBlocks), dim3(128), 0, s, prio, (const double*)C.chol, np, j,
                    (const double*)C.rinv, C.dblk);
        const int T = nb - j - 1;
        if (T > 0)
            launch_crit(k_chol_panel, dim3(T * kQ), dim3(kQR * NB), 0, s, prio, C.chol, np, j, (const double*)C.dblk);
        cudaEventRecord(h->ev_step[j], s);
        if (T > 0) {
            if (j > 0 && nb - j > 1) cudaStreamWaitEvent(s, h->ev_rest[j - 1], 0);  // columns >= j + 1 of step j - 1
            launch_crit(k_chol_update_col, dim3(T * kQ), dim3(kQR * NB), 0, s, prio, C.chol, np, j);
        }
        // block columns j + 2 .. on s3, after the look-ahead column: started beside it, the trailing
        // update's blocks fill the GPU first and the look-ahead column waits behind them
        if (T > 1) {
            forked3 = true;
            cudaEventRecord(h->ev_col[j], s);
            cudaStreamWaitEvent(s3, h->ev_col[j], 0);
            k_chol_update<<<(T - 1) * T / 2 * kQ, kQR * NB, 0, s3>>>(C.chol, np, j, j + 2);
            cudaEventRecord(h->ev_rest[j], s3);
        }
        cudaStreamWaitEvent(s2, h->ev_step[j], 0);
        k_trinv_row<<<j + 1, NB * NB, 0, s2>>>(C.linv, np, j, C.dblk);
        if (j + 1 < nb) {
            const int units = (nb - j - 1) * (j + 1) * kQ;
            k_trinv_update<<<std::min(units, kInvCtas), kQR * NB, 0, s2>>>(C.linv, C.chol, np, j, units);
        }
    }
    cudaEventRecord(h->ev_join, s2);
    cudaStreamWaitEvent(s, h->ev_join, 0);
    if (forked3) {
        cudaEventRecord(h->ev_join2, s3);
        cudaStreamWaitEvent(s, h->ev_join2, 0);
    }
    k_transpose<<<dim3(nb, nb), NB * NB, 0, s>>>(C.linv, C.linvT, np);
}

void record_coarsest_solve(smg_hierarchy* h, int K, const void* in, bool in32, void* out, bool out32,
                           cudaStream_t s) {
    DLevel& C = h->L[h->H];
    switch (K) {
        case 1: coarse_solve_k<1>(C, in, in32, out, out32, s); break;
        case 2: coarse_solve_k<2>(C, in, in32, out, out32, s); break;
        case 3: coarse_solve_k<3>(C, in, in32, out, out32, s); break;
        default: coarse_solve_k<4>(C, in, in32, out, out32, s); break;
    }
}

}  // namespace smg
