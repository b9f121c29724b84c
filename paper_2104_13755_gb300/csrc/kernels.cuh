// Sparse kernels of the V-cycle (Alg. 2) and the per-frame update.
//
// Layout (per level, rows permuted colour-major): the off-diagonal entries sit in
// warp-sized slices of one colour class with R lanes per row (R chosen per level
// so a lane holds few entries; see SliceMeta), so every warp-wide load of values
// or column indices is one contiguous, aligned 128/256-byte segment and all
// gathers of a row are in flight together.  The diagonal is stored apart (and
// its reciprocal for the Gauss-Seidel update).  Vectors with K right-hand sides
// are row-major n x K, so a neighbour gather reads K adjacent values.
#pragma once

#include "rowslice.cuh"

namespace smg {
namespace kern {

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy (TMA) primitives on shared::cta addresses.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// This thread's arrival on the barrier, announcing `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Wait (CTA scope, acquire) for phase `parity` of the barrier, at most `limit`
// polls; false when the polls ran out.
__device__ __forceinline__ bool mbar_wait_cta(uint32_t bar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
constexpr int kBulkWaitPolls = 1 << 22;  // far beyond any copy of a few KB; each poll may suspend the thread

// Binary64 Gauss-Seidel runs on the operator with each row scaled by its
// reciprocal diagonal (values a_ij / a_ii, right-hand side b_i / a_ii, both
// formed outside the colour steps: the values at each update, b / a_ii where b
// is written), so a row's update x_i = b_i / a_ii - sum_{j != i} (a_ij / a_ii) x_j
// is one FMA chain without the final product by the reciprocal diagonal: that
// product sat on the dependent chain of every colour step.  Binary32 keeps the
// unscaled form.
template <typename T>
struct ScaledGS {
    static constexpr bool value = sizeof(T) == 8;
};

// ---------------------------------------------------------------------------
// Multicolour Gauss-Seidel (App. "Multi-Color Gauss Seidel"): one colour class,
// x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii for every row i of the class.
// No row of a class is coupled to another row of the same class, so the rows
// update in parallel and the x values gathered here are not written by this
// launch (padding entries point at the row itself with value 0).
template <typename T, int K, int R>
__global__ void __launch_bounds__(kThreads, MinBlocks<K, R>::value) gs_colour(const SliceMeta* __restrict__ slices, int s0, int s1,
                                                      const int32_t* __restrict__ col, const T* __restrict__ sval,
                                                      const T* __restrict__ dinv, const T* __restrict__ b,
                                                      T* __restrict__ x) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int s = s0 + w / R;
    const int lane = threadIdx.x & 31;
    if (s >= s1) return;
    const SliceMeta m = slices[s];
    RowSlice<T, K, R, PreGS<T, K, R>::value> rs;
    rs.load(m, w % R, lane, col, sval);
    const bool valid = rs.r < m.nrows;
    const int row = m.row0 + (valid ? rs.r : 0);
    const T d = ScaledGS<T>::value ? T(1) : dinv[row];
    pdl_wait();
    pdl_trigger();
    T bv[K], acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) bv[q] = b[(int64_t)row * K + q];
    rs.dot_from(m, col, sval, x, bv, acc);  // b_i - sum_{j != i} a_ij x_j (scaled rows: the new x_i)
    if (valid && rs.sub == 0)
#pragma unroll
        for (int q = 0; q < K; q++) x[(int64_t)row * K + q] = ScaledGS<T>::value ? acc[q] : acc[q] * d;
}

// One lane per row with the slice's entries staged by TMA: the form of
// gs_colour<T, K, 1> for the finest level, where a colour class is ~10^5-10^6
// short rows.  Each warp's slice of column indices and values (its first WC
// entries per row) comes into shared memory by two bulk copies that complete
// on a warp-private mbarrier, issued before the dependency wait.  No entry is
// held in registers across the wait, so eight 256-thread blocks stay resident
// per SM and a ~250k-row class is in flight in one wave, where the
// register-prefetching kernel (five blocks per SM) runs it in two.  The
// arithmetic is that of gs_colour<T, K, 1>: one FMA chain from b in slot order
// (binary32: then the product with the reciprocal diagonal).  Entries past WC (rare wide
// rows) are read from global memory.  A copy that never completes leaves the
// warp after kBulkWaitPolls polls with *err set and its rows unchanged.
template <typename T, int K, int WC>
struct BulkCfg {
    static constexpr int col_bytes = WC * 32 * 4;
    static constexpr int warp_bytes = WC * 32 * (4 + (int)sizeof(T));  // indices, then values
    static constexpr int block_bytes = kWarps * warp_bytes + kWarps * 8;  // entries, then one mbarrier per warp
    static constexpr int min_blocks = K == 1 ? 8 : (K == 2 ? 4 : 2);    // 32 / 64 / 128 registers per thread
};
template <typename T, int K, int WC>
__global__ void __launch_bounds__(kThreads, (BulkCfg<T, K, WC>::min_blocks))
    gs_colour_bulk(const SliceMeta* __restrict__ slices, int s0, int s1, const int32_t* __restrict__ col,
                   const T* __restrict__ sval, const T* __restrict__ dinv, const T* __restrict__ b,
                   T* __restrict__ x, int* __restrict__ err) {
    using C = BulkCfg<T, K, WC>;
    extern __shared__ __align__(16) unsigned char bulk_smem[];
    const int wib = threadIdx.x >> 5;
    const int s = s0 + (int)blockIdx.x * kWarps + wib;
    const int lane = threadIdx.x & 31;
    if (s >= s1) return;
    const SliceMeta m = slices[s];
    const int32_t* scol = reinterpret_cast<const int32_t*>(bulk_smem + wib * C::warp_bytes);
    const T* sv = reinterpret_cast<const T*>(bulk_smem + wib * C::warp_bytes + C::col_bytes);
    const uint32_t bar = smem_u32(bulk_smem) + (uint32_t)(kWarps * C::warp_bytes + 8 * wib);
    const int Wc = m.width < WC ? m.width : WC;
    if (lane == 0 && Wc > 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect(bar, (uint32_t)(Wc * 32 * (4 + (int)sizeof(T))));
        bulk_g2s(smem_u32(scol), col + m.off, (uint32_t)(Wc * 32 * 4), bar);
        bulk_g2s(smem_u32(sv), sval + m.off, (uint32_t)(Wc * 32 * (int)sizeof(T)), bar);
    }
    __syncwarp();
    const bool valid = lane < m.nrows;
    const int row = m.row0 + (valid ? lane : 0);
    const T d = ScaledGS<T>::value ? T(1) : dinv[row];
    pdl_wait();
    pdl_trigger();
    T acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = b[(int64_t)row * K + q];
    if (Wc > 0 && !mbar_wait_cta(bar, 0, kBulkWaitPolls)) {
        atomicExch(err, 1);
        mbar_wait_cta(bar, 0, kBulkWaitPolls);  // the copies land before the block's shared memory is released
        return;
    }
    T xv[WC][K];
#pragma unroll
    for (int u = 0; u < WC; u++)
        if (u < Wc) {
            const int c = scol[u * 32 + lane];
#pragma unroll
            for (int q = 0; q < K; q++) xv[u][q] = ldg(x + (int64_t)c * K + q);
        }
#pragma unroll
    for (int u = 0; u < WC; u++)
        if (u < Wc) {
            const T v = sv[u * 32 + lane];
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] -= v * xv[u][q];
        }
    for (int k = WC; k < m.width; k++) {  // rows wider than the staged part
        const int cc = ldg(col + m.off + k * 32 + lane);
        const T vv = ldg(sval + m.off + k * 32 + lane);
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] -= vv * ldg(x + (int64_t)cc * K + q);
    }
    if (valid)
#pragma unroll
        for (int q = 0; q < K; q++) x[(int64_t)row * K + q] = ScaledGS<T>::value ? acc[q] : acc[q] * d;
}

// 3|V| systems: one launch class (a vertex colour class) of the sweep in 3 x 3
// blocks.  Unknown (v, c) has colour 3 C(v) + c, so scalar Gauss-Seidel in
// colour order updates, for each vertex of class C, component 0, then 1, then
// 2 (reverse sweep: 2, 1, 0), each from the newest values: neighbours of other
// classes are not updated inside the class, and the vertex's own other
// components enter through its diagonal block.  R lanes per vertex (32 / R
// vertices per warp, a slice of 32 vertices over R warps), lane `sub` taking
// neighbour blocks sub, sub + R, ..., summed over the R lanes by a fixed xor
// tree; each neighbour block costs one column index and one 24-byte gather of
// the neighbour's three values.
template <typename T, int K, int R>
__global__ void __launch_bounds__(kThreads) gs_block3(const SliceMeta* __restrict__ slices, int s0, int s1,
                                                      const int32_t* __restrict__ bcol, const T* __restrict__ bval,
                                                      const T* __restrict__ dblk, int64_t nv,
                                                      const T* __restrict__ dinv, const T* __restrict__ b,
                                                      T* __restrict__ x, int reverse) {
    constexpr int RL = 32 / R;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int s = s0 + w / R;
    const int lane = threadIdx.x & 31;
    if (s >= s1) return;
    const SliceMeta m = slices[s];
    const int sub = lane / RL;
    const int r = (w % R) * RL + (lane % RL);
    const bool valid = r < m.nrows;
    const int64_t pv = m.row0 + (valid ? r : 0);
    T D[9], di[3];
    if (sub == 0) {
#pragma unroll
        for (int q = 0; q < 9; q++) D[q] = ldg(dblk + q * nv + pv);
#pragma unroll
        for (int a = 0; a < 3; a++) di[a] = ldg(dinv + 3 * pv + a);
    }
    const int32_t* cb = bcol + m.off + r;
    const T* vb = bval + 9 * (int64_t)m.off + r;
    int c0 = sub < m.width ? ldg(cb + sub * 32) : 0;
    pdl_wait();
    pdl_trigger();
    T acc[3][K];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int q = 0; q < K; q++) acc[a][q] = (sub == 0) ? b[(3 * pv + a) * K + q] : T(0);
    for (int k = sub; k < m.width; k += R) {
        const int c = c0;
        if (k + R < m.width) c0 = ldg(cb + (k + R) * 32);
        T xw[3][K];
#pragma unroll
        for (int e = 0; e < 3; e++)
#pragma unroll
            for (int q = 0; q < K; q++) xw[e][q] = x[(3 * (int64_t)c + e) * K + q];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int e = 0; e < 3; e++) {
                const T v = ldg(vb + (9 * k + 3 * a + e) * 32);
#pragma unroll
                for (int q = 0; q < K; q++) acc[a][q] -= v * xw[e][q];
            }
    }
#pragma unroll
    for (int o = 16; o >= RL; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int q = 0; q < K; q++) acc[a][q] += __shfl_xor_sync(0xffffffffu, acc[a][q], o);
    if (sub != 0 || !valid) return;
    T xo[3][K], xn[3][K];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int q = 0; q < K; q++) xo[a][q] = x[(3 * pv + a) * K + q];
#pragma unroll
    for (int q = 0; q < K; q++) {
        if (!reverse) {
            xn[0][q] = (acc[0][q] - D[1] * xo[1][q] - D[2] * xo[2][q]) * di[0];
            xn[1][q] = (acc[1][q] - D[3] * xn[0][q] - D[5] * xo[2][q]) * di[1];
            xn[2][q] = (acc[2][q] - D[6] * xn[0][q] - D[7] * xn[1][q]) * di[2];
        } else {
            xn[2][q] = (acc[2][q] - D[6] * xo[0][q] - D[7] * xo[1][q]) * di[2];
            xn[1][q] = (acc[1][q] - D[3] * xo[0][q] - D[5] * xn[2][q]) * di[1];
            xn[0][q] = (acc[0][q] - D[1] * xn[1][q] - D[2] * xn[2][q]) * di[0];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int q = 0; q < K; q++) x[(3 * pv + a) * K + q] = xn[a][q];
}

// Values of the 3 x 3 block layout from the flat values (src -1: zero), binary64
// and binary32.
__global__ void block_gather(int64_t m, const int32_t* __restrict__ src, const double* __restrict__ vals,
                             double* __restrict__ out, float* __restrict__ out32) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t k = src[e];
    const double v = k >= 0 ? vals[k] : 0.0;
    out[e] = v;
    out32[e] = (float)v;
}

// Damped Jacobi update x <- x + omega D^{-1} r after r = b - A x (App.
// "Ablation Study": the smoother compared with Gauss-Seidel).
template <typename T, int K>
__global__ void jacobi_update(int64_t n, T omega, const T* __restrict__ dinv, const T* __restrict__ r,
                              T* __restrict__ x) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const T w = omega * dinv[e / K];
    pdl_wait();
    pdl_trigger();
    x[e] += w * r[e];
}

// r = b - A x over all rows of a level.
template <typename T, int K, int R>
__global__ void __launch_bounds__(kThreads, MinBlocks<K, R>::value) residual(const SliceMeta* __restrict__ slices, int nslices,
                                                     const int32_t* __restrict__ col, const T* __restrict__ sval,
                                                     const T* __restrict__ diag, const T* __restrict__ b,
                                                     const T* __restrict__ x, T* __restrict__ r) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int s = w / R;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const SliceMeta m = slices[s];
    RowSlice<T, K, R, Pre<T, K, R>::value> rs;
    rs.load(m, w % R, lane, col, sval);
    const bool valid = rs.r < m.nrows;
    const int row = m.row0 + (valid ? rs.r : 0);
    const T d = diag[row];
    pdl_wait();
    pdl_trigger();
    T own[K], acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) own[q] = b[(int64_t)row * K + q] - d * x[(int64_t)row * K + q];
    rs.dot_from(m, col, sval, x, own, acc);  // b_i - a_ii x_i - sum_{j != i} a_ij x_j
    if (valid && rs.sub == 0)
#pragma unroll
        for (int q = 0; q < K; q++) r[(int64_t)row * K + q] = acc[q];
}

// Residual fused with restriction (Alg. 2 "compute residual", "restrict
// residual"): b_{h+1} = P^T (b_h - A_h x_h) computed as P^T b_h - Q x_h with
// Q = P^T A_h from the Galerkin stage 1, so one gather per coarse row replaces
// the residual pass, its round trip through memory and the restriction pass.
// Rows are coarse rows in the RQSlice layout (R lanes per row; entries k < wb
// hold -P[i,I] against b_h, the rest Q[I,j] against x_h), so acc = init - sum
// over all entries of value * vector.  The kernel also starts the coarse
// iterate, x_{h+1} = 0, and the first Gauss-Seidel colour step from that zero
// gives each row of colour class 0 (rows [0, nseed)) exactly b_i / a_ii (its
// neighbours are all zero, and fma(-a, 0, b) = b), so with nseed > 0 it writes
// that value and the caller skips that colour step.
template <typename T, int K, int R>
__global__ void __launch_bounds__(kThreads) restrict_fused(const RQSlice* __restrict__ slices, int nslices,
                                                           const int32_t* __restrict__ rq_row,
                                                           const int32_t* __restrict__ col, const T* __restrict__ val,
                                                           const T* __restrict__ b, const T* __restrict__ x,
                                                           T* __restrict__ bc, T* __restrict__ xc,
                                                           const T* __restrict__ dinv_c, int nseed,
                                                           T* __restrict__ bdi_c) {
    constexpr int RL = 32 / R, PRE = 8;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int s = w / R;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const RQSlice m = slices[s];
    const int sub = lane / RL;
    const int r = (w % R) * RL + (lane % RL);
    const int W = m.wb + m.wq;
    const bool valid = r < m.nrows;
    const int I = valid ? rq_row[m.pos0 + r] : 0;
    int c[PRE];
    T v[PRE];
#pragma unroll
    for (int u = 0; u < PRE; u++) {
        const int k = sub + R * u;
        if (k < W) {
            c[u] = ldg(col + m.off + k * 32 + r);
            v[u] = ldg(val + m.off + k * 32 + r);
        }
    }
    const T dc = (valid && (I < nseed || bdi_c != nullptr)) ? dinv_c[I] : T(0);
    pdl_wait();
    pdl_trigger();
    T acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = T(0);
    T g[PRE][K];
#pragma unroll
    for (int u = 0; u < PRE; u++) {
        const int k = sub + R * u;
        if (k < W) {
            const T* src = k < m.wb ? b : x;
#pragma unroll
            for (int q = 0; q < K; q++) g[u][q] = ldg(src + (int64_t)c[u] * K + q);
        }
    }
#pragma unroll
    for (int u = 0; u < PRE; u++)
        if (sub + R * u < W)
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] -= v[u] * g[u][q];
    for (int k = sub + R * PRE; k < W; k += R) {
        const int cc = ldg(col + m.off + k * 32 + r);
        const T vv = ldg(val + m.off + k * 32 + r);
        const T* src = k < m.wb ? b : x;
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] -= vv * ldg(src + (int64_t)cc * K + q);
    }
#pragma unroll
    for (int o = 16; o >= RL; o >>= 1)
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (valid && sub == 0)
#pragma unroll
        for (int q = 0; q < K; q++) {
            bc[(int64_t)I * K + q] = acc[q];
            if (bdi_c) bdi_c[(int64_t)I * K + q] = acc[q] * dc;
            xc[(int64_t)I * K + q] = I < nseed ? acc[q] * dc : T(0);
        }
}

// Prolongation with the correction add, x_h <- x_h + P c (Alg. 2 "prolong
// correction", "update solution"): three barycentric weights per fine row.
template <typename T, int K>
__global__ void __launch_bounds__(kThreads) prolong_add(int n, const int32_t* __restrict__ idx,
                                                        const T* __restrict__ w, const T* __restrict__ xc,
                                                        T* __restrict__ x) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c[3];
    T wa[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        c[a] = idx[(int64_t)a * n + p];
        wa[a] = w[(int64_t)a * n + p];
    }
    pdl_wait();
    pdl_trigger();
    T xv[3][K];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int q = 0; q < K; q++) xv[a][q] = ldg(xc + (int64_t)c[a] * K + q);
#pragma unroll
    for (int q = 0; q < K; q++) {
        T acc = wa[0] * xv[0][q] + wa[1] * xv[1][q] + wa[2] * xv[2][q];
        x[(int64_t)p * K + q] += acc;
    }
}

// ---------------------------------------------------------------------------
// Level-0 residual norms for the stopping test of Alg. 1, reduced in a fixed
// order (fixed grid, fixed tree) so the result is bitwise reproducible.
// INIT also accumulates ||b||^2; R32 also stores the residual in binary32 (the
// right-hand side of the next inner cycle of the mixed-precision form) and
// zeroes that cycle's binary32 iterate.
template <int K, int R, bool INIT, bool R32>
__global__ void __launch_bounds__(kThreads) resnorm(const SliceMeta* __restrict__ slices, int nslices,
                                                    const int32_t* __restrict__ col, const double* __restrict__ sval,
                                                    const double* __restrict__ diag, const double* __restrict__ b,
                                                    const double* __restrict__ x, double* __restrict__ partials,
                                                    float* __restrict__ r32, float* __restrict__ x32,
                                                    double* __restrict__ r64) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    pdl_wait();
    pdl_trigger();
    double rr[K], bb[K];
#pragma unroll
    for (int q = 0; q < K; q++) rr[q] = bb[q] = 0.0;
    for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < nslices * R; w += gridDim.x * kWarps) {
        const SliceMeta m = slices[w / R];
        RowSlice<double, K, R, Pre<double, K, R>::value> rs;
        rs.load(m, w % R, lane, col, sval);
        const bool valid = rs.r < m.nrows;
        const int row = m.row0 + (valid ? rs.r : 0);
        const double d = diag[row];
        double bv[K], own[K], acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) {
            bv[q] = b[(int64_t)row * K + q];
            own[q] = bv[q] - d * x[(int64_t)row * K + q];
        }
        rs.dot_from(m, col, sval, x, own, acc);  // the residual of the row
        if (valid && rs.sub == 0) {
#pragma unroll
            for (int q = 0; q < K; q++) {
                const double rv = acc[q];
                rr[q] += rv * rv;
                if (r64) r64[(int64_t)row * K + q] = rv;
                if (INIT) bb[q] += bv[q] * bv[q];
                if (R32) {
                    r32[(int64_t)row * K + q] = (float)rv;
                    x32[(int64_t)row * K + q] = 0.0f;
                }
            }
        }
    }
    __shared__ double red[kWarps][2 * K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        for (int o = 16; o > 0; o >>= 1) {
            rr[q] += __shfl_xor_sync(0xffffffffu, rr[q], o);
            bb[q] += __shfl_xor_sync(0xffffffffu, bb[q], o);
        }
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) {
            red[wid][q] = rr[q];
            red[wid][K + q] = bb[q];
        }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double s = 0.0;
        for (int w = 0; w < kWarps; w++) s += red[w][threadIdx.x];
        partials[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = s;
    }
}

// The same for a dense level-0 matrix (single-level hierarchy): a warp per row.
template <int K, bool INIT, bool R32>
__global__ void __launch_bounds__(kThreads) resnorm_dense(int n, const double* __restrict__ A,
                                                          const double* __restrict__ b, const double* __restrict__ x,
                                                          double* __restrict__ partials, float* __restrict__ r32,
                                                          float* __restrict__ x32, double* __restrict__ r64) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    pdl_wait();
    pdl_trigger();
    double rr[K], bb[K];
#pragma unroll
    for (int q = 0; q < K; q++) rr[q] = bb[q] = 0.0;
    for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < n; i += gridDim.x * kWarps) {
        double acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double a = A[(int64_t)i * n + j];
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += a * x[(int64_t)j * K + q];
        }
#pragma unroll
        for (int q = 0; q < K; q++) {
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            const double bv = b[(int64_t)i * K + q];
            const double rv = bv - acc[q];
            if (lane == 0) {
                rr[q] += rv * rv;
                if (r64) r64[(int64_t)i * K + q] = rv;
                if (INIT) bb[q] += bv * bv;
                if (R32) {
                    r32[(int64_t)i * K + q] = (float)rv;
                    x32[(int64_t)i * K + q] = 0.0f;
                }
            }
        }
    }
    __shared__ double red[kWarps][2 * K];
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) {
            red[wid][q] = rr[q];
            red[wid][K + q] = bb[q];
        }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double s = 0.0;
        for (int w = 0; w < kWarps; w++) s += red[w][threadIdx.x];
        partials[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = s;
    }
}

// Final reduction and stopping test.  `init`: before the first cycle (records
// ||b|| and rel0); otherwise after a cycle.  Sets the WHILE condition of the
// solve graph: continue while rel > rtol, finite, and cycles < max_cycles.
template <int K>
__global__ void norm_final(const double* __restrict__ partials, int nblocks, SolveState* __restrict__ st,
                           cudaGraphConditionalHandle hnd, int init, double rtol, int max_cycles, int use_cond) {
    __shared__ double red[kThreads][2 * K];
    pdl_wait();
    pdl_trigger();
    double acc[2 * K];
#pragma unroll
    for (int q = 0; q < 2 * K; q++) acc[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 2 * K; q++) acc[q] += partials[(int64_t)b * 2 * K + q];
#pragma unroll
    for (int q = 0; q < 2 * K; q++) red[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 2 * K; q++) red[threadIdx.x][q] += red[threadIdx.x + w][q];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if (init)
        for (int q = 0; q < K; q++) st->bnorm2[q] = red[0][K + q];
    double rel = 0.0;
    for (int q = 0; q < K; q++) {
        const double bn = st->bnorm2[q];
        const double rq = bn > 0.0 ? sqrt(red[0][q] / bn) : sqrt(red[0][q]);
        rel = (rq > rel || rq != rq) ? rq : rel;
    }
    if (init) {
        st->rel0 = rel;
        st->cycles = 0;
    } else {
        st->cycles += 1;
    }
    st->rel = rel;
    const bool finite = isfinite(rel);
    const bool converged = finite && rel <= rtol;
    const bool more = finite && !converged && st->cycles < max_cycles;
    st->status = converged ? SMG_OK : (!finite ? SMG_ERR_DIVERGED : (more ? -1 : SMG_ERR_NOT_CONVERGED));
    if (use_cond) cudaGraphSetConditional(hnd, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Conjugate gradients preconditioned by one V-cycle from a zero start (Sec.
// "Limitations & Future Work" names the multigrid cycle as a CG
// preconditioner).  Each right-hand side is its own CG.  Every reduction uses
// the fixed grid of kNormBlocks blocks and a fixed order, and the scalars
// (alpha, beta) are recomputed identically by every block from the partials,
// so the iteration is bitwise reproducible and needs no extra launches.

// Sum of the K-column block partials (stride doubles per block) in a fixed
// order; every thread of the block gets the totals.
template <int K>
__device__ __forceinline__ void sum_partials(const double* __restrict__ part, int nblocks, int stride,
                                             double (&out)[K]) {
    __shared__ double red[kThreads][K];
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] += part[(int64_t)b * stride + q];
#pragma unroll
    for (int q = 0; q < K; q++) red[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < K; q++) red[threadIdx.x][q] += red[threadIdx.x + w][q];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < K; q++) out[q] = red[0][q];
    __syncthreads();
}

// Block reduction of per-thread column sums into part[block * stride + q].
template <int K>
__device__ __forceinline__ void block_partials(double (&v)[K], double* __restrict__ part, int stride) {
    __shared__ double red[kWarps][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < K; q++)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) red[wid][q] = v[q];
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int w = 0; w < kWarps; w++) t += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * stride + threadIdx.x] = t;
    }
}

__global__ void cg_copy(int64_t m, const double* __restrict__ src, double* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    pdl_wait();
    pdl_trigger();
    dst[e] = src[e];
}

// Right-hand side and zero start of the preconditioner cycle: b_0 <- r, x_0 <- 0
// (and, for a binary64 cycle, b_0 / a_ii into bdi0 when given; K columns).
template <typename T>
__global__ void cg_precond_in(int64_t m, int K, const double* __restrict__ r, T* __restrict__ b0, T* __restrict__ x0,
                              const double* __restrict__ dinv0, double* __restrict__ bdi0) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    pdl_wait();
    pdl_trigger();
    b0[e] = (T)r[e];
    x0[e] = T(0);
    if (bdi0) bdi0[e] = r[e] * dinv0[e / K];
}

// Partials of rho = r . z per column (z in the cycle's precision).
template <int K, typename TZ>
__global__ void __launch_bounds__(kThreads) cg_dot(int64_t n, const double* __restrict__ r, const TZ* __restrict__ z,
                                                   double* __restrict__ part) {
    pdl_wait();
    pdl_trigger();
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; q++) acc[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] += r[i * K + q] * (double)z[i * K + q];
    block_partials<K>(acc, part, K);
}

// p <- z + beta p, beta = rho / rho_previous (p <- z in the first iteration).
// rho goes to slot (iteration & 1) of the state; the previous one is read from
// the other slot, so block 0's store cannot race the other blocks' loads.
template <int K, typename TZ>
__global__ void __launch_bounds__(kThreads) cg_p_update(int64_t n, const double* __restrict__ part_rz,
                                                        const TZ* __restrict__ z, double* __restrict__ p,
                                                        SolveState* __restrict__ st) {
    pdl_wait();
    pdl_trigger();
    double rho[K];
    sum_partials<K>(part_rz, kNormBlocks, K, rho);
    const int it = st->cycles;
    double beta[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        const double old = st->cg_rho[(it + 1) & 1][q];
        beta[q] = (it == 0 || old == 0.0) ? 0.0 : rho[q] / old;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < K; q++) st->cg_rho[it & 1][q] = rho[q];
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
#pragma unroll
        for (int q = 0; q < K; q++) {
            const double zv = (double)z[i * K + q];
            p[i * K + q] = it == 0 ? zv : zv + beta[q] * p[i * K + q];
        }
}

// q <- A p and the partials of p . q (SELL level 0, diagonal apart).
template <int K, int R>
__global__ void __launch_bounds__(kThreads) cg_spmv(const SliceMeta* __restrict__ slices, int nslices,
                                                    const int32_t* __restrict__ col, const double* __restrict__ sval,
                                                    const double* __restrict__ diag, const double* __restrict__ p,
                                                    double* __restrict__ qv, double* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    pdl_wait();
    pdl_trigger();
    double pq[K];
#pragma unroll
    for (int q = 0; q < K; q++) pq[q] = 0.0;
    for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < nslices * R; w += gridDim.x * kWarps) {
        const SliceMeta m = slices[w / R];
        RowSlice<double, K, R, Pre<double, K, R>::value> rs;
        rs.load(m, w % R, lane, col, sval);
        double acc[K];
        rs.dot(m, col, sval, p, acc);  // acc = -(sum of the off-diagonal products)
        if (rs.r < m.nrows && rs.sub == 0) {
            const int row = m.row0 + rs.r;
            const double d = diag[row];
#pragma unroll
            for (int q = 0; q < K; q++) {
                const double pv = p[(int64_t)row * K + q];
                const double v = d * pv - acc[q];
                qv[(int64_t)row * K + q] = v;
                pq[q] += pv * v;
            }
        }
    }
    block_partials<K>(pq, part, K);
}

// The same for a dense level-0 matrix (single-level hierarchy): a warp per row.
template <int K>
__global__ void __launch_bounds__(kThreads) cg_spmv_dense(int n, const double* __restrict__ A,
                                                          const double* __restrict__ p, double* __restrict__ qv,
                                                          double* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    pdl_wait();
    pdl_trigger();
    double pq[K];
#pragma unroll
    for (int q = 0; q < K; q++) pq[q] = 0.0;
    for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < n; i += gridDim.x * kWarps) {
        double acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = 0.0;
        for (int j = lane; j < n; j += 32)
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += A[(int64_t)i * n + j] * p[(int64_t)j * K + q];
#pragma unroll
        for (int q = 0; q < K; q++) {
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (lane == 0) {
                qv[(int64_t)i * K + q] = acc[q];
                pq[q] += p[(int64_t)i * K + q] * acc[q];
            }
        }
    }
    block_partials<K>(pq, part, K);
}

// x <- x + alpha p, r <- r - alpha q with alpha = rho / (p . q), and the
// partials of ||r||^2 in the layout of the stopping test (2K per block).
template <int K>
__global__ void __launch_bounds__(kThreads) cg_xr_update(int64_t n, const double* __restrict__ part_pq,
                                                         const double* __restrict__ p, const double* __restrict__ qv,
                                                         double* __restrict__ x, double* __restrict__ r,
                                                         const SolveState* __restrict__ st, double* __restrict__ part_rr) {
    pdl_wait();
    pdl_trigger();
    double pq[K];
    sum_partials<K>(part_pq, kNormBlocks, K, pq);
    const int it = st->cycles;
    double alpha[K], rr[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        alpha[q] = pq[q] != 0.0 ? st->cg_rho[it & 1][q] / pq[q] : 0.0;
        rr[q] = 0.0;
    }
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
#pragma unroll
        for (int q = 0; q < K; q++) {
            x[i * K + q] += alpha[q] * p[i * K + q];
            const double rv = r[i * K + q] - alpha[q] * qv[i * K + q];
            r[i * K + q] = rv;
            rr[q] += rv * rv;
        }
    block_partials<K>(rr, part_rr, 2 * K);
    if (threadIdx.x < K) part_rr[(int64_t)blockIdx.x * 2 * K + K + threadIdx.x] = 0.0;
}

// ---------------------------------------------------------------------------
// Per-frame update kernels

// Per face: cotangent of the angle at each corner and the area.
__global__ void face_geom(int64_t nf, const int32_t* __restrict__ F, const double* __restrict__ V,
                          double* __restrict__ fg) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    double p[3][3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int64_t v = F[3 * f + c];
#pragma unroll
        for (int d = 0; d < 3; d++) p[c][d] = V[3 * v + d];
    }
    double e1[3], e2[3], cr[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        e1[d] = p[1][d] - p[0][d];
        e2[d] = p[2][d] - p[0][d];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double dbl = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);  // twice the area
    const double inv = 1.0 / dbl;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double* a = p[c];
        const double* u = p[(c + 1) % 3];
        const double* w = p[(c + 2) % 3];
        const double dot = (u[0] - a[0]) * (w[0] - a[0]) + (u[1] - a[1]) * (w[1] - a[1]) + (u[2] - a[2]) * (w[2] - a[2]);
        fg[4 * f + c] = dot * inv;  // |e1 x e2| is the same at every corner
    }
    fg[4 * f + 3] = 0.5 * dbl;
}

// Diagonal of the cotan Laplacian (positive semi-definite sign) and the lumped
// mass: L_ii = sum over incident faces of (cot of the two other corners) / 2,
// M_ii = sum of incident face areas / 3.
__global__ void asm_diag(int64_t n, int64_t dstride, const int32_t* __restrict__ inc_ptr,
                         const int32_t* __restrict__ inc_code, const double* __restrict__ fg,
                         double* __restrict__ Lflat, double* __restrict__ M) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double ld = 0.0, m = 0.0;
    for (int k = inc_ptr[p]; k < inc_ptr[p + 1]; k++) {
        const int code = inc_code[k];
        const int64_t f = code / 3;
        const int c = code - 3 * (code / 3);
        ld += 0.5 * (fg[4 * f + (c + 1) % 3] + fg[4 * f + (c + 2) % 3]);
        m += fg[4 * f + 3] / 3.0;
    }
    Lflat[p * dstride] = ld;
    M[p] = m;
}

// Off-diagonal cotan weights: L_ij = -(cot a + cot b) / 2 over the corners
// opposite the edge ij (one corner on a boundary edge).
__global__ void asm_off(int64_t nflat, int64_t first, int64_t dense_n, const int32_t* __restrict__ opp0,
                        const int32_t* __restrict__ opp1, const double* __restrict__ fg, double* __restrict__ Lflat) {
    const int64_t e = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nflat) return;
    if (dense_n > 0 && e / dense_n == e % dense_n) return;
    const int a = opp0[e], b = opp1[e];
    double s = 0.0;
    if (a >= 0) s += fg[4 * (int64_t)(a / 3) + a % 3];
    if (b >= 0) s += fg[4 * (int64_t)(b / 3) + b % 3];
    Lflat[e] = -0.5 * s;
}

// A = t L + M on the flat layout.
__global__ void combine(int64_t nflat, int64_t n, int64_t dense_n, double t, const double* __restrict__ Lflat,
                        const double* __restrict__ M, double* __restrict__ vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nflat) return;
    double v = t * Lflat[e];
    if (dense_n > 0) {
        if (e / dense_n == e % dense_n) v += M[e / dense_n];
    } else if (e < n) {
        v += M[e];
    }
    vals[e] = v;
}

// The same with t read from device memory (graph-captured batch updates).
__global__ void combine_devt(int64_t nflat, int64_t n, int64_t dense_n, const double* __restrict__ t,
                             const double* __restrict__ Lflat, const double* __restrict__ M,
                             double* __restrict__ vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nflat) return;
    double v = t[0] * Lflat[e];
    if (dense_n > 0) {
        if (e / dense_n == e % dense_n) v += M[e / dense_n];
    } else if (e < n) {
        v += M[e];
    }
    vals[e] = v;
}

// Fast parameter update (App. "Fast Data Smoothing"): with P^T L P and P^T M P
// of every level kept, A_l(t) = P^T M P + t P^T L P is one pass per level.
__global__ void axpy_devt(int64_t nflat, const double* __restrict__ t, const double* __restrict__ Lv,
                          const double* __restrict__ Mv, double* __restrict__ vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nflat) return;
    vals[e] = Mv[e] + t[0] * Lv[e];
}

// Flat level-0 values of the lumped mass: the diagonal entries, zero elsewhere.
__global__ void mass_flat(int64_t nflat, int64_t n, int64_t dense_n, const double* __restrict__ M,
                          double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nflat) return;
    double v = 0.0;
    if (dense_n > 0) {
        if (e / dense_n == e % dense_n) v = M[e / dense_n];
    } else if (e < n) {
        v = M[e];
    }
    out[e] = v;
}

__global__ void set_scalar(double* __restrict__ d, double v) { d[0] = v; }

// User-supplied level-0 values (natural CSR) scattered to the flat layout.
__global__ void scatter_user(int64_t nflat, const int64_t* __restrict__ map, const double* __restrict__ user,
                             double* __restrict__ vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nflat) return;
    const int64_t k = map[e];
    vals[e] = k >= 0 ? user[k] : 0.0;
}

// Numeric Galerkin product A_{h+1} = P^T A_h P (Eq. gca) on the precomputed
// patterns, in two stages that are both fixed-order gathers (no atomics):
// stage 1 forms Q = P^T A_h, one thread per entry of Q, each summing its
// products P[i,I] A_h[i,j] over the fine rows i of P^T row I; stage 2 forms
// A_{h+1} = Q P, one thread per coarse entry, summing Q[I,j] P[j,J] over the
// columns j of Q row I.  Q stays in the slots of the fused residual-restriction
// operator, which uses it in every cycle.
__global__ void galerkin_q(int64_t nq, const int32_t* __restrict__ dst, const int32_t* __restrict__ ptr,
                           const int32_t* __restrict__ src, const int32_t* __restrict__ pw,
                           const double* __restrict__ fine, const double* __restrict__ p_w, double* __restrict__ rq) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nq) return;
    double acc = 0.0;
    for (int32_t k = ptr[e]; k < ptr[e + 1]; k++) acc = fma(ldg(p_w + pw[k]), ldg(fine + src[k]), acc);
    rq[dst[e]] = acc;
}

__global__ void galerkin_qp(int64_t nflat_c, const int32_t* __restrict__ ptr, const int32_t* __restrict__ src,
                            const int32_t* __restrict__ pw, const double* __restrict__ rq,
                            const double* __restrict__ p_w, double* __restrict__ coarse) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nflat_c) return;
    double acc = 0.0;
    for (int32_t k = ptr[d]; k < ptr[d + 1]; k++) acc = fma(ldg(rq + src[k]), ldg(p_w + pw[k]), acc);
    coarse[d] = acc;
}

// Binary32 copy of an array (the fused restriction operator of the mixed form).
__global__ void copy_f32(int64_t m, const double* __restrict__ a, float* __restrict__ o) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) o[e] = (float)a[e];
}

// Reciprocal diagonal and the binary32 copies used by the mixed-precision cycle.
__global__ void prep_level(int64_t nflat, int64_t n, const double* __restrict__ vals, double* __restrict__ dinv,
                           float* __restrict__ vals32, float* __restrict__ dinv32) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nflat) return;
    vals32[e] = (float)vals[e];
    if (e < n) {
        const double di = 1.0 / vals[e];
        dinv[e] = di;
        dinv32[e] = (float)di;
    }
}

// Off-diagonal SELL values scaled by their row's reciprocal diagonal (one warp
// per slice, lane = row of the slice; padding rows hold zeros).
__global__ void scale_sell(int nslices, const SliceMeta* __restrict__ slices, const double* __restrict__ sval,
                           const double* __restrict__ dinv, double* __restrict__ out) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= nslices) return;
    const SliceMeta m = slices[w];
    const double d = lane < m.nrows ? dinv[m.row0 + lane] : 0.0;
    for (int k = 0; k < m.width; k++) {
        const int64_t e = (int64_t)m.off + k * 32 + lane;
        out[e] = sval[e] * d;
    }
}

// ---------------------------------------------------------------------------
// Permutation between the caller's unknown order and the colour-major order.
template <typename T>
__global__ void gather_rows(int64_t n, int K, const int32_t* __restrict__ perm, const T* __restrict__ src,
                            T* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const int64_t p = e / K, q = e - p * K;
    dst[e] = src[(int64_t)perm[p] * K + q];
}
// The same for the level-0 right-hand side, also writing b_i / a_ii (binary64
// Gauss-Seidel's scaled rows).
__global__ void gather_rows_scaled(int64_t n, int K, const int32_t* __restrict__ perm, const double* __restrict__ src,
                                   const double* __restrict__ dinv, double* __restrict__ dst,
                                   double* __restrict__ dst_scaled) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const int64_t p = e / K, q = e - p * K;
    const double v = src[(int64_t)perm[p] * K + q];
    dst[e] = v;
    dst_scaled[e] = v * dinv[p];
}
template <typename T>
__global__ void scatter_rows(int64_t n, int K, const int32_t* __restrict__ perm, const T* __restrict__ src,
                             T* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const int64_t p = e / K, q = e - p * K;
    dst[(int64_t)perm[p] * K + q] = src[e];
}

// Iterative refinement update x <- x + d (binary32 correction, binary64 iterate).
__global__ void ir_update(int64_t m, const float* __restrict__ d, double* __restrict__ x) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    pdl_wait();
    pdl_trigger();
    x[e] += (double)d[e];
}

// y = M x with the lumped mass (permuted rows) written in the caller's order.
__global__ void apply_mass(int64_t n, int K, const int32_t* __restrict__ perm, const double* __restrict__ M,
                           const double* __restrict__ x, double* __restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const int64_t p = e / K, q = e - p * K;
    const int64_t u = perm[p];
    y[u * K + q] = M[p] * x[u * K + q];
}

}  // namespace kern
}  // namespace smg
