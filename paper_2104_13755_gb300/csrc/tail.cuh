// Cluster tail of the V-cycle: the levels below a tuned size run inside one
// thread-block cluster (up to 16 CTAs, one per SM), one launch for the whole
// down-sweep (pre-relaxation, residual, restriction of every tail level) and one
// for the up-sweep (prolongation with correction, post-relaxation).  Colour
// classes and level transfers are separated by the cluster barrier (release /
// acquire at cluster scope) instead of kernel boundaries; values written inside
// the launch are read through L2 (ld.global.cg).  The arithmetic per row is the
// same as the full-GPU kernels (Alg. 2 with the multicolour Gauss-Seidel of
// App. "Multi-Color Gauss Seidel").
#pragma once

#include "kernels.cuh"

namespace smg {

// Device view of one level for the tail kernels (one precision).
template <typename T>
struct TailLevel {
    const SliceMeta* slices;
    const int32_t* col;
    const T* sval;
    const T* dinv;
    const T* diag;
    const int32_t* colour_slice;  // ncolours + 1 slice offsets
    T* x;
    T* b;
    T* r;
    int nslices, ncolours, n;
    // restriction into level + 1
    const int32_t* pt_ptr;
    const int32_t* pt_row;
    const T* pt_w;
    int n_next;
    T* b_next;
    T* x_next;
    // prolongation from level + 1
    const int32_t* p_idx;
    const T* p_w;
};

namespace kern {

constexpr int kTailThreads = 512;
constexpr int kTailR = 8;  // lanes per row inside the tail

// Cluster-wide barrier with release / acquire ordering of memory at cluster
// scope.  The non-.aligned form: a warp may reach it after divergent loops.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

template <typename T, int K>
__device__ __forceinline__ void tail_gs(const TailLevel<T>& L, int c, int gwarp, int nwarps, int lane) {
    const int s0 = L.colour_slice[c], s1 = L.colour_slice[c + 1];
    const int need = (s1 - s0) * kTailR;
    for (int w = gwarp; w < need; w += nwarps) {
        const SliceMeta m = L.slices[s0 + w / kTailR];
        RowSlice<T, K, kTailR, Pre<T, K>::value> rs;
        rs.load(m, w % kTailR, lane, L.col, L.sval);
        const bool valid = rs.r < m.nrows;
        const int row = m.row0 + (valid ? rs.r : 0);
        const T d = L.dinv[row];
        T acc[K];
        rs.template dot<true>(m, L.col, L.sval, L.x, acc);
        if (valid && rs.sub == 0)
#pragma unroll
            for (int q = 0; q < K; q++) L.x[(int64_t)row * K + q] = (__ldcg(L.b + (int64_t)row * K + q) + acc[q]) * d;
    }
}

template <typename T, int K>
__device__ __forceinline__ void tail_residual(const TailLevel<T>& L, int gwarp, int nwarps, int lane) {
    const int need = L.nslices * kTailR;
    for (int w = gwarp; w < need; w += nwarps) {
        const SliceMeta m = L.slices[w / kTailR];
        RowSlice<T, K, kTailR, Pre<T, K>::value> rs;
        rs.load(m, w % kTailR, lane, L.col, L.sval);
        const bool valid = rs.r < m.nrows;
        const int row = m.row0 + (valid ? rs.r : 0);
        const T d = L.diag[row];
        T acc[K];
        rs.template dot<true>(m, L.col, L.sval, L.x, acc);
        if (valid && rs.sub == 0)
#pragma unroll
            for (int q = 0; q < K; q++)
                L.r[(int64_t)row * K + q] =
                    (__ldcg(L.b + (int64_t)row * K + q) - d * __ldcg(L.x + (int64_t)row * K + q)) + acc[q];
    }
}

// b_{l+1} = P^T r_l (four lanes per coarse row) and the zero start x_{l+1} = 0.
// Every thread makes the same number of passes (the shuffles need whole warps).
template <typename T, int K>
__device__ __forceinline__ void tail_restrict(const TailLevel<T>& L, int gthread, int nthreads) {
    constexpr int RR = 4;
    const int sub = gthread % RR;
    const int per_pass = nthreads / RR;
    const int passes = (L.n_next + per_pass - 1) / per_pass;
    for (int pass = 0; pass < passes; pass++) {
        const int g = pass * per_pass + gthread / RR;
        const bool ok = g < L.n_next;
        const int I = ok ? g : L.n_next - 1;
        T acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = T(0);
        for (int k = L.pt_ptr[I] + sub; k < L.pt_ptr[I + 1]; k += RR) {
            const int i = L.pt_row[k];
            const T wk = L.pt_w[k];
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += wk * __ldcg(L.r + (int64_t)i * K + q);
        }
#pragma unroll
        for (int o = RR / 2; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        if (ok && sub == 0)
#pragma unroll
            for (int q = 0; q < K; q++) {
                L.b_next[(int64_t)I * K + q] = acc[q];
                L.x_next[(int64_t)I * K + q] = T(0);
            }
    }
}

// x_l += P x_{l+1}
template <typename T, int K>
__device__ __forceinline__ void tail_prolong(const TailLevel<T>& L, int gthread, int nthreads) {
    for (int p = gthread; p < L.n; p += nthreads) {
        T acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = T(0);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int c = L.p_idx[(int64_t)a * L.n + p];
            const T wa = L.p_w[(int64_t)a * L.n + p];
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += wa * __ldcg(L.x_next + (int64_t)c * K + q);
        }
#pragma unroll
        for (int q = 0; q < K; q++) L.x[(int64_t)p * K + q] = __ldcg(L.x + (int64_t)p * K + q) + acc[q];
    }
}

// Down-sweep of levels [l0, l1): pre-relaxation, residual, restriction.
template <typename T, int K>
__global__ void __launch_bounds__(kTailThreads) tail_down(const TailLevel<T>* __restrict__ lv, int l0, int l1,
                                                          int mu_pre) {
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (kTailThreads / 32);
    const int gwarp = blockIdx.x * (kTailThreads / 32) + (threadIdx.x >> 5);
    const int nthreads = gridDim.x * kTailThreads;
    const int gthread = blockIdx.x * kTailThreads + threadIdx.x;
    pdl_wait();
    pdl_trigger();
    for (int l = l0; l < l1; l++) {
        const TailLevel<T> L = lv[l];
        for (int it = 0; it < mu_pre; it++)
            for (int c = 0; c < L.ncolours; c++) {
                tail_gs<T, K>(L, c, gwarp, nwarps, lane);
                cluster_sync();
            }
        tail_residual<T, K>(L, gwarp, nwarps, lane);
        cluster_sync();
        tail_restrict<T, K>(L, gthread, nthreads);
        cluster_sync();
    }
}

// Up-sweep of levels [l0, l1) from level l1 - 1 upwards: prolongation with the
// correction add, then post-relaxation (colour classes reversed if asked).
template <typename T, int K>
__global__ void __launch_bounds__(kTailThreads) tail_up(const TailLevel<T>* __restrict__ lv, int l0, int l1,
                                                        int mu_post, int reverse) {
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (kTailThreads / 32);
    const int gwarp = blockIdx.x * (kTailThreads / 32) + (threadIdx.x >> 5);
    const int nthreads = gridDim.x * kTailThreads;
    const int gthread = blockIdx.x * kTailThreads + threadIdx.x;
    pdl_wait();
    pdl_trigger();
    for (int l = l1 - 1; l >= l0; l--) {
        const TailLevel<T> L = lv[l];
        tail_prolong<T, K>(L, gthread, nthreads);
        cluster_sync();
        for (int it = 0; it < mu_post; it++)
            for (int cc = 0; cc < L.ncolours; cc++) {
                tail_gs<T, K>(L, reverse ? L.ncolours - 1 - cc : cc, gwarp, nwarps, lane);
                cluster_sync();
            }
    }
}

}  // namespace kern
}  // namespace smg
