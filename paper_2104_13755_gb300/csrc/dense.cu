// Coarsest level of Alg. 2 ("solve A x = b", direct): a dense binary64
// Cholesky factor A_H = L L^T computed once per update, then the inverse factor
// X = L^{-1} and its transpose, so that each cycle's direct solve
// x = L^{-T} (L^{-1} b) is two dense triangular products spread over the whole
// GPU instead of two serial substitutions.
//
// Blocked right-looking algorithms with 32 x 32 tiles; the matrix is padded to
// a multiple of 32 with an identity block.
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

// Factor diagonal tile j in shared memory and store its triangular inverse.
__global__ void __launch_bounds__(NB * NB) k_chol_diag(double* __restrict__ C, int64_t np, int j,
                                                       double* __restrict__ dblk, int32_t* __restrict__ bad) {
    __shared__ double a[NB][NB + 1];
    __shared__ double inv[NB][NB + 1];
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    double* T = C + (int64_t)j * NB * np + (int64_t)j * NB;
    a[r][c] = T[(int64_t)r * np + c];
    __syncthreads();
    for (int k = 0; k < NB; k++) {
        if (r == k && c == k) {
            double d = a[k][k];
            if (!(d > 0.0) || !isfinite(d)) {  // not SPD: flag it, keep the arithmetic finite
                atomicExch(bad, 1);
                d = 1.0;
            }
            a[k][k] = sqrt(d);
        }
        __syncthreads();
        if (c == k && r > k) a[r][k] = a[r][k] / a[k][k];
        __syncthreads();
        if (c > k && r >= c) a[r][c] -= a[r][k] * a[c][k];
        __syncthreads();
    }
    T[(int64_t)r * np + c] = (c <= r) ? a[r][c] : 0.0;
    if (r == 0) {  // column c of the inverse of the lower-triangular tile
        for (int i = 0; i < NB; i++) {
            double v;
            if (i < c) v = 0.0;
            else if (i == c) v = 1.0 / a[c][c];
            else {
                double s = 0.0;
                for (int k = c; k < i; k++) s += a[i][k] * inv[k][c];
                v = -s / a[i][i];
            }
            inv[i][c] = v;
        }
    }
    __syncthreads();
    dblk[(int64_t)j * NB * NB + r * NB + c] = inv[r][c];
}

// L_ij = A_ij L_jj^{-T} for the tiles below the diagonal tile j.
__global__ void __launch_bounds__(NB * NB) k_chol_panel(double* __restrict__ C, int64_t np, int j,
                                                        const double* __restrict__ dblk) {
    __shared__ double a[NB][NB + 1];
    __shared__ double d[NB][NB + 1];
    const int i = j + 1 + blockIdx.x;
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    double* T = C + (int64_t)i * NB * np + (int64_t)j * NB;
    a[r][c] = T[(int64_t)r * np + c];
    d[r][c] = dblk[(int64_t)j * NB * NB + r * NB + c];
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k <= c; k++) s += a[r][k] * d[c][k];
    T[(int64_t)r * np + c] = s;
}

__device__ __forceinline__ void tri_index(int b, int& ii, int& kk) {
    int t = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
    while ((t + 1) * (t + 2) / 2 <= b) t++;
    while (t * (t + 1) / 2 > b) t--;
    ii = t;
    kk = b - t * (t + 1) / 2;
}

// Trailing update A_ik -= L_ij L_kj^T for j < k <= i.
__global__ void __launch_bounds__(NB * NB) k_chol_update(double* __restrict__ C, int64_t np, int j) {
    __shared__ double li[NB][NB + 1];
    __shared__ double lk[NB][NB + 1];
    int ii, kk;
    tri_index(blockIdx.x, ii, kk);
    const int i = j + 1 + ii, k = j + 1 + kk;
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    li[r][c] = C[((int64_t)i * NB + r) * np + (int64_t)j * NB + c];
    lk[r][c] = C[((int64_t)k * NB + r) * np + (int64_t)j * NB + c];
    __syncthreads();
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < NB; q++) s += li[r][q] * lk[c][q];
    C[((int64_t)i * NB + r) * np + (int64_t)k * NB + c] -= s;
}

// Block row i of X = L^{-1}: X_i,jb = L_ii^{-1} B_i,jb for jb <= i (B accumulates I - sum L X).
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
    double s = 0.0;
    for (int q = 0; q <= r; q++) s += d[r][q] * bs[q][c];
    T[(int64_t)r * np + c] = s;
}

// B_k,jb -= L_k,i X_i,jb for k > i, jb <= i.
__global__ void __launch_bounds__(NB * NB) k_trinv_update(double* __restrict__ X, const double* __restrict__ C,
                                                          int64_t np, int i) {
    __shared__ double l[NB][NB + 1];
    __shared__ double xs[NB][NB + 1];
    const int k = i + 1 + blockIdx.x / (i + 1);
    const int jb = blockIdx.x % (i + 1);
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;
    l[r][c] = C[((int64_t)k * NB + r) * np + (int64_t)i * NB + c];
    xs[r][c] = X[((int64_t)i * NB + r) * np + (int64_t)jb * NB + c];
    __syncthreads();
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < NB; q++) s += l[r][q] * xs[q][c];
    X[((int64_t)k * NB + r) * np + (int64_t)jb * NB + c] -= s;
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
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
    const double* row = X + (int64_t)i * np;
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
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
    const double* row = XT + (int64_t)j * np;
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
    const int grid = (n + 7) / 8;
    if (in32) k_coarse_lower<K, true><<<grid, 256, 0, s>>>(C.linv, C.np, n, in, C.y);
    else k_coarse_lower<K, false><<<grid, 256, 0, s>>>(C.linv, C.np, n, in, C.y);
    if (out32) k_coarse_upper<K, true><<<grid, 256, 0, s>>>(C.linvT, C.np, n, C.y, out);
    else k_coarse_upper<K, false><<<grid, 256, 0, s>>>(C.linvT, C.np, n, C.y, out);
}

}  // namespace

void record_coarsest_factor(smg_hierarchy* h, cudaStream_t s) {
    DLevel& C = h->L[h->H];
    const int64_t np = C.np;
    const int nb = (int)(np / NB);
    k_pad_copy<<<(unsigned)((np * np + 255) / 256), 256, 0, s>>>(C.vals, C.n, C.chol, C.linv, np);
    for (int j = 0; j < nb; j++) {
        k_chol_diag<<<1, NB * NB, 0, s>>>(C.chol, np, j, C.dblk, &h->state->chol_bad);
        const int T = nb - j - 1;
        if (T > 0) {
            k_chol_panel<<<T, NB * NB, 0, s>>>(C.chol, np, j, C.dblk);
            k_chol_update<<<T * (T + 1) / 2, NB * NB, 0, s>>>(C.chol, np, j);
        }
    }
    for (int i = 0; i < nb; i++) {
        k_trinv_row<<<i + 1, NB * NB, 0, s>>>(C.linv, np, i, C.dblk);
        if (i + 1 < nb) k_trinv_update<<<(nb - i - 1) * (i + 1), NB * NB, 0, s>>>(C.linv, C.chol, np, i);
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
