// Internal: the geometry-only plan and its device-ready layouts.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/smg.h"
#include "smg_host.hpp"

namespace smg {

constexpr int kSlice = 32;  // rows per SELL slice (one warp)

// Per-slice header of the SELL-32 off-diagonal storage: 32 consecutive rows of
// one colour class; entry k of the row at local position r sits at slot
// off + 32 k + r, so a warp-wide load of one entry of 32 rows is one contiguous
// 128/256-byte segment.  Kernels may split a slice over R warps (R lanes per
// row, 32 / R rows per warp): each load step then reads R segments.
struct SliceMeta {
    int32_t row0;   // first (permuted) row of the slice
    int32_t nrows;  // rows in the slice (<= 32; the last slice of a colour may be short)
    int32_t width;  // padded off-diagonal entries per row
    int32_t off;    // first slot of the slice
};

inline int64_t slot_at(const SliceMeta& s, int r, int k) { return (int64_t)s.off + (int64_t)k * kSlice + r; }

// Slice header of the fused residual-restriction operator of a level (rows =
// coarse rows): 32 consecutive positions [pos0, pos0 + nrows); entry k of the
// position at local row r sits at slot off + 32 k + r: k < wb is the
// restriction segment (applied to the fine right-hand side), wb <= k < wb + wq
// the segment of Q = P^T A (applied to the fine iterate).
struct RQSlice {
    int32_t pos0;
    int32_t nrows;
    int32_t wb;
    int32_t wq;
    int32_t off;
    int32_t pad;
};

struct LevelPlan {
    int64_t n = 0;
    bool coarsest = false;
    // natural-order symbolic pattern (sorted, diagonal included)
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    // Alg. 3 colouring (natural numbering), permutation new -> natural and inverse
    int32_t ncolours = 0;
    std::vector<int32_t> colour, perm, iperm;
    // permuted layout: colour classes and SELL-32 off-diagonal slots
    std::vector<int32_t> colour_row;    // ncolours + 1
    std::vector<int32_t> colour_slice;  // ncolours + 1
    std::vector<SliceMeta> slices;
    std::vector<int32_t> sell_col;      // permuted column of every slot (padding: the row itself)
    int64_t nslots = 0;
    // flat value array of A_l: [diag (n, padded to sbase) | slots (nslots)], or dense
    // n x n at the coarsest; slot s lives at flat index sbase + s
    int64_t sbase = 0;
    int64_t nflat = 0;
    // natural-order reduced prolongation to the next level (3 per row, -1 unused)
    std::vector<int32_t> pn_idx;
    std::vector<double> pn_w;
    // permuted prolongation (slot-major [3][n]) and restriction CSR (rows = next level)
    std::vector<int32_t> p_idx;
    std::vector<double> p_w;
    std::vector<int32_t> pt_ptr, pt_row;
    std::vector<double> pt_w;
    // Residual fused with restriction (Alg. 2 "restrict residual" as one product):
    //   b_{l+1}[I] = sum_i P[i,I] b_l[i] - sum_j Q[I,j] x_l[j],  Q = P^T A_l,
    // in the RQSlice layout: rq_row[position] = coarse row, rq_col per slot (fine
    // row), rq_w per slot: -P[i,I] in the restriction segment, 0 in the Q
    // segment (Q is numeric, written by the Galerkin stage 1) and in padding.
    std::vector<RQSlice> rq_slices;
    std::vector<int32_t> rq_row, rq_col;
    std::vector<double> rq_w;
    int32_t rq_maxw = 0;
    // Galerkin product (Eq. gca) in two stages.  Stage 1, Q = P^T A_l: Q entry e
    // (slot q_dst[e] of the layout above) = sum over k in [q_ptr[e], q_ptr[e+1])
    // of flat_l[q_src[k]] * p_w[q_pw[k]].  Stage 2, A_{l+1} = Q P: next-level
    // flat entry d = sum over k in [g_ptr[d], g_ptr[d+1]) of rq[g_src[k]] * p_w[g_pw[k]].
    std::vector<int32_t> q_dst, q_ptr, q_src, q_pw;
    std::vector<int32_t> g_ptr, g_src, g_pw;
    // flat index -> position in the natural CSR pattern (for read-back)
    std::vector<int64_t> flat_to_csr;
    // 3|V| systems (block size 3): the operator in 3 x 3 blocks for the block
    // sweep.  Vertex p (permuted) owns rows 3p .. 3p + 2.  Slices of 32 vertices
    // of one launch class (SliceMeta: row0 = first vertex, nrows = vertices,
    // width = off-diagonal blocks, off = first block slot); neighbour block k of
    // local vertex r at slot off + 32 k + r (b_col: neighbour vertex, padding the
    // vertex itself); its value (a, e) at 9 off + 32 (9 k + 3 a + e) + r, taken
    // from flat entry b_src[...] (-1: structural zero).  Diagonal blocks:
    // value (a, e) of vertex p at (3 a + e) nv + p, from d_src.
    std::vector<SliceMeta> b_slices;
    std::vector<int32_t> b_colour_slice;
    std::vector<int32_t> b_col, b_src, d_src;
    int64_t b_nslots = 0;
};

struct AssemblyPlan {
    int64_t nv = 0, nf = 0;            // all mesh vertices, faces
    std::vector<int32_t> F;            // 3 nf
    std::vector<int32_t> row_vertex;   // permuted level-0 row -> mesh vertex
    std::vector<int32_t> inc_ptr;      // incident face corners per permuted row
    std::vector<int32_t> inc_code;     // face * 3 + corner of the row's vertex
    std::vector<int32_t> opp0, opp1;   // per slot: face * 3 + corner opposite the edge (-1 none)
    std::vector<int64_t> flat_to_user; // flat index -> user CSR position (-1 padding)
    // every mesh vertex: incident face corners, and its unknown index (-1 if known)
    std::vector<int32_t> vinc_ptr, vinc_code, vert_unk;
};

struct Plan {
    smg_options opts{};
    std::vector<MeshData> meshes;          // geometry levels 0..H
    std::vector<ProlongationRaw> praw;     // praw[l] = P_{l+1}
    std::vector<DecimationStats> stats;
    std::vector<uint8_t> known;            // n0
    std::vector<int32_t> unknowns;         // level-0 natural index -> vertex
    std::vector<int32_t> kept1;            // level-1 natural index -> mesh-1 vertex
    std::vector<LevelPlan> L;              // algebraic levels 0..H
    AssemblyPlan asmb;
};

// Build the algebraic part (patterns ... assembly plan) from meshes/praw/known.
int finalize_plan(Plan& p, std::string& err);
// Build everything from a mesh.
int build_plan(const double* V, int64_t n, const int32_t* F, int64_t m, const uint8_t* mask,
               const smg_options& o, Plan& p, std::string& err);

void set_error(const std::string& msg);

}  // namespace smg

struct smg_plan {
    smg::Plan p;
};
