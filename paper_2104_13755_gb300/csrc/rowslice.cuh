// Shared row machinery of the sparse kernels: loads, programmatic dependent
// launch, and the SELL-32 row walk with R lanes per row (RowSlice), used by the
// launched kernels and by the persistent batched solve alike.
#pragma once

#include "device.hpp"

namespace smg {
namespace kern {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kNormBlocks = 608;  // fixed grid of the deterministic norm reduction

template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
    return __ldg(p);
}

// Loads of data that other CTAs of the same launch write (cluster tail kernels):
// served by L2, the coherence point, never by the non-coherent read-only path.
template <bool COHERENT, typename T>
__device__ __forceinline__ T ldx(const T* p) {
    if (COHERENT) return __ldcg(p);
    return __ldg(p);
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Kernels of a cycle are launched so that the
// next kernel may start while the previous one drains: everything a kernel
// reads that no kernel of the cycle writes (matrix entries, slice headers,
// prolongation weights) is loaded before pdl_wait(); everything produced by an
// earlier kernel is read after it.  pdl_wait() returns once the preceding grid
// has completed and its writes are visible (immediately when launched
// without the attribute); pdl_trigger() lets the following grid start.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Entries per lane loaded ahead of the dependency wait.  With one lane per row
// (the finest level, valence ~6) six entries cover a typical row and keep the
// kernel at 48 registers, five resident blocks per SM; with two lanes per row
// (the first coarse level, rows of 15-25 entries) twelve per lane keep rows
// out of the path that loads entries after the wait.
template <typename T, int K, int R>
struct Pre {
    static constexpr int value = R == 1 ? 6 : (R == 2 && K == 1) ? 12 : ((K <= 2 || sizeof(T) == 4) ? 8 : 4);
};
// The launched Gauss-Seidel colour step of a coarse level: a colour class
// there fills fewer than one block per SM, so registers are not what limits
// residency, while any entry past the prefetched ones costs a dependent load
// after the wait that the whole step waits for.  Binary64 with one right-hand
// side prefetches enough to cover rows of 36 (two lanes) and 44 (four lanes)
// entries, the widest rows of the first coarse levels of the test meshes.
template <typename T, int K, int R>
struct PreGS {
    static constexpr int value =
        (sizeof(T) == 8 && K == 1 && R == 2) ? 18 : (sizeof(T) == 8 && K == 1 && R == 4) ? 11 : Pre<T, K, R>::value;
};
template <int K, int R>
struct MinBlocks {
    static constexpr int value = (R == 1 && K == 1) ? 5 : 1;
};

// A warp covers 32 / R rows of a SELL-32 slice (sub-slice g of R), R lanes per
// row: lane = sub * (32 / R) + rl holds entries k = sub, sub + R, ... of row
// g * (32 / R) + rl, so the lanes of one `sub` read contiguous slots.  acc gets
// -sum_k a_k x_{c_k}, summed over the R lanes of a row by a fixed xor tree.
template <typename T, int K, int R, int PRE>
struct RowSlice {
    static constexpr int RL = 32 / R;  // rows per warp
    int c[PRE];
    T v[PRE];
    int W, sub, r;
    __device__ __forceinline__ void load(const SliceMeta& m, int g, int lane, const int32_t* __restrict__ col,
                                         const T* __restrict__ sval) {
        W = m.width;
        sub = lane / RL;
        r = g * RL + (lane % RL);
#pragma unroll
        for (int u = 0; u < PRE; u++) {
            const int k = sub + R * u;
            if (k < W) {
                c[u] = ldg(col + m.off + k * 32 + r);
                v[u] = ldg(sval + m.off + k * 32 + r);
            }
        }
    }
    // COHERENT = false: x is read-only in this launch except at rows this warp
    // owns; true: other CTAs of this launch write x between cluster barriers
    template <bool COHERENT = false>
    __device__ __forceinline__ void dot(const SliceMeta& m, const int32_t* __restrict__ col,
                                        const T* __restrict__ sval, const T* x, T (&acc)[K]) const {
        T zero[K];
#pragma unroll
        for (int q = 0; q < K; q++) zero[q] = T(0);
        dot_from<COHERENT>(m, col, sval, x, zero, acc);
    }
    // acc = init - sum_k a_k x_{c_k}: the row's first lane starts its chain
    // from init, so the caller's own term costs no separate add.
    template <bool COHERENT = false>
    __device__ __forceinline__ void dot_from(const SliceMeta& m, const int32_t* __restrict__ col,
                                             const T* __restrict__ sval, const T* x, const T (&init)[K],
                                             T (&acc)[K]) const {
        T xv[PRE][K];
#pragma unroll
        for (int u = 0; u < PRE; u++)
            if (sub + R * u < W)
#pragma unroll
                for (int q = 0; q < K; q++) xv[u][q] = ldx<COHERENT>(x + (int64_t)c[u] * K + q);
        // Binary64: one chain.  A binary64 instruction holds its warp for the
        // same ~64 clocks whether or not it depends on the one before, so the
        // count of instructions, not the chain depth, sets the time; a second
        // chain would only add the final add.  Binary32 with several lanes per
        // row: two chains for instruction-level parallelism.
        constexpr bool SPLIT = R > 1 && sizeof(T) == 4;
        T a1[K];
#pragma unroll
        for (int q = 0; q < K; q++) {
            acc[q] = sub == 0 ? init[q] : T(0);
            a1[q] = T(0);
        }
#pragma unroll
        for (int u = 0; u < PRE; u++)
            if (sub + R * u < W)
#pragma unroll
                for (int q = 0; q < K; q++) {
                    if (SPLIT && (u & 1)) a1[q] -= v[u] * xv[u][q];
                    else acc[q] -= v[u] * xv[u][q];
                }
        for (int k = sub + R * PRE; k < W; k += R) {  // rows longer than PRE * R: the rare tail
            const int cc = ldg(col + m.off + k * 32 + r);
            const T vv = ldg(sval + m.off + k * 32 + r);
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] -= vv * ldx<COHERENT>(x + (int64_t)cc * K + q);
        }
        if (SPLIT)
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += a1[q];
#pragma unroll
        for (int o = 16; o >= RL; o >>= 1)
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
};

}  // namespace kern
}  // namespace smg
