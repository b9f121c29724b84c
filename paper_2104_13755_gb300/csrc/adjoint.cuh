// Derivatives of the level-0 operator with respect to vertex positions and t,
// for the differentiable solve x = A(V, t)^{-1} b (A = M + t L, lumped mass M,
// positive semi-definite cotangent Laplacian L).
//
// With lambda = A^{-1} g for an upstream gradient g, the chain rule needs
// d/dV [lambda^T A(V) x] and lambda^T L x.  Both are sums over faces f of
//   (area_f / 3) sum_{c in f} lambda_c x_c  +  t sum_k (cot_k / 2) (lambda_i - lambda_j)(x_i - x_j)
// (edge (i, j) opposite corner k), because x^T L y = sum over edges of the
// cotangent weight times the edge differences.  Known (Dirichlet) vertices
// carry zero.  Per face the analytic derivatives are
//   d area / d p_i = n^ x (p_{i+2} - p_{i+1}) / 2
//   d cot_k / d u = v / |n| - (u.v / |n|^2) (v x n^),  d cot_k / d v = u / |n| - (u.v / |n|^2) (n^ x u)
// with u = p_{k+1} - p_k, v = p_{k+2} - p_k, n = u x v; the per-face pieces are
// gathered per vertex in a fixed order (deterministic, no atomics).
#pragma once

#include "kernels.cuh"

namespace smg {
namespace kern {

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 add(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 mul(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Per face: g[c] = scale * (cm * d area / d p_c + t * sum_k wk_k * d cot_k / d p_c).
//   mode 0 (operator): cm = sum over corners and right-hand sides of lambda x / 3,
//                      wk_k = sum_q (dlambda)(dx) / 2 on the edge opposite k; the
//                      face's sum_k wk_k cot_k goes to dt_face
//   mode 1 (mass):     cm = (w_0 + w_1 + w_2) / 3, no cotangent part
template <int K>
__global__ void face_grad(int64_t nf, const int32_t* __restrict__ F, const double* __restrict__ V,
                          const int32_t* __restrict__ vert_unk, const double* __restrict__ lam,
                          const double* __restrict__ x, const double* __restrict__ w, int mode, double t,
                          double scale, double* __restrict__ facegrad, double* __restrict__ dt_face) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int u[3];
    D3 p[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int v = F[3 * f + c];
        u[c] = vert_unk[v];
        p[c] = d3(V + 3 * (int64_t)v);
    }
    double cm = 0.0, wk[3] = {0.0, 0.0, 0.0};
    if (mode == 0) {
        double lv[3][K], xv[3][K];
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int q = 0; q < K; q++) {
                lv[c][q] = u[c] >= 0 ? lam[(int64_t)u[c] * K + q] : 0.0;
                xv[c][q] = u[c] >= 0 ? x[(int64_t)u[c] * K + q] : 0.0;
                cm += lv[c][q] * xv[c][q];
            }
        cm /= 3.0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int i = (k + 1) % 3, j = (k + 2) % 3;
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < K; q++) s += (lv[i][q] - lv[j][q]) * (xv[i][q] - xv[j][q]);
            wk[k] = 0.5 * s;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; c++) cm += u[c] >= 0 ? w[u[c]] : 0.0;
        cm /= 3.0;
    }
    const D3 n = cross(sub(p[1], p[0]), sub(p[2], p[0]));
    const double A2 = sqrt(dot(n, n));
    const D3 nh = mul(1.0 / A2, n);
    D3 g[3];
#pragma unroll
    for (int c = 0; c < 3; c++) g[c] = mul(0.5 * cm, cross(nh, sub(p[(c + 2) % 3], p[(c + 1) % 3])));
    double dtf = 0.0;
    if (mode == 0) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const D3 uu = sub(p[(k + 1) % 3], p[k]);
            const D3 vv = sub(p[(k + 2) % 3], p[k]);
            const double d = dot(uu, vv);
            dtf += wk[k] * d / A2;
            const double a = t * wk[k] / A2, bcoef = t * wk[k] * d / (A2 * A2);
            const D3 du = sub(mul(a, vv), mul(bcoef, cross(vv, nh)));
            const D3 dv = sub(mul(a, uu), mul(bcoef, cross(nh, uu)));
            g[(k + 1) % 3] = add(g[(k + 1) % 3], du);
            g[(k + 2) % 3] = add(g[(k + 2) % 3], dv);
            g[k] = sub(g[k], add(du, dv));
        }
        dt_face[f] = scale * dtf;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        facegrad[9 * f + 3 * c + 0] = scale * g[c].x;
        facegrad[9 * f + 3 * c + 1] = scale * g[c].y;
        facegrad[9 * f + 3 * c + 2] = scale * g[c].z;
    }
}

// gradV[v] = sum over the face corners at v of their per-face pieces (fixed order).
__global__ void vertex_gather(int64_t nv, const int32_t* __restrict__ ptr, const int32_t* __restrict__ code,
                              const double* __restrict__ facegrad, double* __restrict__ gradV) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int k = ptr[v]; k < ptr[v + 1]; k++) {
        const int64_t cc = code[k];  // face * 3 + corner
        g0 += facegrad[3 * cc + 0];
        g1 += facegrad[3 * cc + 1];
        g2 += facegrad[3 * cc + 2];
    }
    gradV[3 * v + 0] = g0;
    gradV[3 * v + 1] = g1;
    gradV[3 * v + 2] = g2;
}

// Fixed-order sum of per-face values into out[0] (one block).
__global__ void sum_fixed(int64_t n, const double* __restrict__ v, double* __restrict__ out) {
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Lumped mass from positions (unknown order): M_uu = sum of incident areas / 3.
__global__ void mass_from_faces(int64_t nv, const int32_t* __restrict__ ptr, const int32_t* __restrict__ code,
                                const int32_t* __restrict__ vert_unk, const double* __restrict__ fg,
                                double* __restrict__ m) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int uu = vert_unk[v];
    if (uu < 0) return;
    double s = 0.0;
    for (int k = ptr[v]; k < ptr[v + 1]; k++) s += fg[4 * (int64_t)(code[k] / 3) + 3] / 3.0;
    m[uu] = s;
}

}  // namespace kern
}  // namespace smg
