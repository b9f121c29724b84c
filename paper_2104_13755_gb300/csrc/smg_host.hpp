// Host-side setup of the surface multigrid hierarchy (geometry only).
//
// Everything here runs once per mesh, before any system matrix exists
// (Alg. 1: the prolongations P_1..P_H are precomputed from V and F alone).
// The per-solve and per-frame work lives in the CUDA sources.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace smg {

struct MeshData {
    std::vector<double> V;   // 3 n, vertex positions
    std::vector<int32_t> F;  // 3 m, consistently oriented triangles
    int64_t n() const { return (int64_t)V.size() / 3; }
    int64_t m() const { return (int64_t)F.size() / 3; }
};

// Prolongation P_{l+1} in natural vertex orders: n_fine x n_coarse with up to
// three barycentric weights per row (Sec. 4.5); unused slots have idx = -1.
struct ProlongationRaw {
    int64_t n_fine = 0, n_coarse = 0;
    std::vector<int32_t> idx;  // 3 n_fine
    std::vector<double> w;     // 3 n_fine
};

struct DecimationStats {
    int64_t collapses = 0;
    int64_t rejected_link = 0;      // link condition / manifoldness
    int64_t rejected_boundary = 0;  // boundary topology (pinch, ear, short loop)
    int64_t rejected_flip = 0;      // a UV or 3D triangle would invert
    int64_t rejected_angle = 0;     // winding of a patch vertex is not one turn
    int64_t rejected_quality = 0;   // new 3D triangle below the minimum angle
    int64_t rejected_solve = 0;     // singular flattening system
    int64_t clamped = 0;            // barycentrics clamped beyond 1e-10
    double worst_negative = 0.0;    // most negative barycentric seen before clamping
};

// One level of uniform mid-point decimation with successive self-parameterization:
// collapse shortest edges (midpoint placement) until `target` vertices remain,
// flatten each edge 1-ring before and vertex 1-ring after the collapse jointly
// (Eq. jointEnergy, LSCM), and carry every vertex of `fine` through the
// collapses as a barycentric point.  Returns 0 on success.
int decimate_level(const MeshData& fine, int64_t target, MeshData& coarse,
                   ProlongationRaw& P, DecimationStats& st, std::string& err);

// Greedy colouring of Alg. 3 on the off-diagonal graph of a CSR pattern.
// Reading: degree = off-diagonal count, visit by degree descending with ties by
// ascending index, first listed palette colour that fits is taken and moved to
// the back, new colours are numbered in creation order.  Returns the colour count.
int32_t greedy_colouring(int64_t n, const std::vector<int64_t>& rowptr,
                         const std::vector<int32_t>& col, std::vector<int32_t>& colour);

}  // namespace smg
