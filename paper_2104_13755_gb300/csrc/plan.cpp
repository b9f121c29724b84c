// Geometry-only setup: level loop, Dirichlet reduction, symbolic Galerkin
// patterns, Alg. 3 colourings and the device-ready layouts.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "plan.hpp"

namespace smg {

// Run body(begin, end) over [0, n) in contiguous chunks on up to 16 host threads.
template <class Body>
static void parallel_rows(int64_t n, Body body) {
    int nt = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (n < 4096) nt = 1;
    std::vector<std::thread> th;
    for (int t = 0; t < nt; t++) {
        int64_t a = n * t / nt, b = n * (t + 1) / nt;
        if (t + 1 == nt) body(a, b);
        else th.emplace_back(body, a, b);
    }
    for (auto& x : th) x.join();
}

// Setup trace: with SMG_TRACE_SETUP set, every stage prints its wall time to stderr.
struct StageTimer {
    bool on = std::getenv("SMG_TRACE_SETUP") != nullptr;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void mark(const char* what) {
        if (!on) return;
        auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[smg setup] %-28s %8.3f s\n", what, std::chrono::duration<double>(now - t).count());
        t = now;
    }
};

static int validate_mesh(const double* V, int64_t n, const int32_t* F, int64_t m, std::string& err) {
    if (!V || !F || n < 3 || m < 1 || n > (int64_t)INT32_MAX / 4 || m > (int64_t)INT32_MAX / 4) {
        err = "invalid mesh sizes or null arrays";
        return SMG_ERR_INVALID_ARG;
    }
    for (int64_t k = 0; k < 3 * n; k++)
        if (!std::isfinite(V[k])) {
            err = "non-finite vertex position";
            return SMG_ERR_INVALID_ARG;
        }
    std::vector<int64_t> he;  // directed edges a*n+b
    he.reserve(3 * m);
    for (int64_t f = 0; f < m; f++) {
        int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
        if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) {
            err = "face index out of range";
            return SMG_ERR_INVALID_ARG;
        }
        if (a == b || b == c || c == a) {
            err = "degenerate face (repeated vertex)";
            return SMG_ERR_NONMANIFOLD;
        }
        he.push_back((int64_t)a * n + b);
        he.push_back((int64_t)b * n + c);
        he.push_back((int64_t)c * n + a);
    }
    std::sort(he.begin(), he.end());
    for (size_t k = 1; k < he.size(); k++)
        if (he[k] == he[k - 1]) {
            err = "directed edge used twice: non-manifold or inconsistently oriented mesh";
            return SMG_ERR_NONMANIFOLD;
        }
    return SMG_OK;
}

int build_plan(const double* V, int64_t n, const int32_t* F, int64_t m, const uint8_t* mask,
               const smg_options& o, Plan& p, std::string& err) {
    int st = validate_mesh(V, n, F, m, err);
    if (st) return st;
    if (!(o.ratio > 0.0 && o.ratio < 1.0) || o.mu_pre < 0 || o.mu_post < 0 ||
        (o.pattern_rings != 1 && o.pattern_rings != 2) || (o.block_size != 1 && o.block_size != 3)) {
        err = "invalid options";
        return SMG_ERR_INVALID_ARG;
    }
    p.opts = o;
    p.meshes.clear();
    p.praw.clear();
    p.stats.clear();
    MeshData m0;
    m0.V.assign(V, V + 3 * n);
    m0.F.assign(F, F + 3 * m);
    p.meshes.push_back(std::move(m0));
    p.known.assign(n, 0);
    if (mask)
        for (int64_t v = 0; v < n; v++) p.known[v] = mask[v] ? 1 : 0;
    // level loop (Sec. 5: ratio 0.25 per level, coarsest no smaller than 500)
    for (;;) {
        const MeshData& cur = p.meshes.back();
        int64_t nc = cur.n();
        if (o.max_levels > 0 && (int64_t)p.meshes.size() >= o.max_levels) break;
        int64_t target = (int64_t)std::nearbyint(o.ratio * (double)nc);
        if (o.max_coarse > 0) {
            if (nc <= o.max_coarse) break;
        } else if (target < o.min_coarse) {
            break;
        }
        if (target < 4 || target >= nc) break;
        MeshData next;
        ProlongationRaw P;
        DecimationStats ds;
        StageTimer dt;
        if (decimate_level(cur, target, next, P, ds, err) != 0) return SMG_ERR_DECIMATION;
        dt.mark("decimation level");
        if (next.n() >= nc) break;
        p.meshes.push_back(std::move(next));
        p.praw.push_back(std::move(P));
        p.stats.push_back(ds);
    }
    return finalize_plan(p, err);
}

// --------------------------------------------------------------------------
// symbolic P^T S P
static void galerkin_pattern(int64_t nf, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                             const std::vector<int32_t>& pidx, int64_t nc, std::vector<int64_t>& crp,
                             std::vector<int32_t>& cci) {
    std::vector<int64_t> tp(nc + 1, 0);
    for (int64_t i = 0; i < nf; i++)
        for (int a = 0; a < 3; a++)
            if (pidx[3 * i + a] >= 0) tp[pidx[3 * i + a] + 1]++;
    for (int64_t I = 0; I < nc; I++) tp[I + 1] += tp[I];
    std::vector<int32_t> trow(tp[nc]);
    std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
    for (int64_t i = 0; i < nf; i++)
        for (int a = 0; a < 3; a++)
            if (pidx[3 * i + a] >= 0) trow[fill[pidx[3 * i + a]]++] = (int32_t)i;
    std::vector<int64_t> mark(nc, -1);
    std::vector<int32_t> row;
    crp.assign(nc + 1, 0);
    cci.clear();
    for (int64_t I = 0; I < nc; I++) {
        row.clear();
        for (int64_t t = tp[I]; t < tp[I + 1]; t++) {
            int32_t i = trow[t];
            for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
                int32_t j = ci[q];
                for (int b = 0; b < 3; b++) {
                    int32_t J = pidx[3 * j + b];
                    if (J >= 0 && mark[J] != I) {
                        mark[J] = I;
                        row.push_back(J);
                    }
                }
            }
        }
        std::sort(row.begin(), row.end());
        cci.insert(cci.end(), row.begin(), row.end());
        crp[I + 1] = (int64_t)cci.size();
    }
}

static int64_t csr_find(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, int64_t r, int32_t c) {
    auto b = ci.begin() + rp[r], e = ci.begin() + rp[r + 1];
    auto it = std::lower_bound(b, e, c);
    if (it == e || *it != c) return -1;
    return (int64_t)(it - ci.begin());
}

int finalize_plan(Plan& p, std::string& err) {
    StageTimer tm;
    const int H = (int)p.meshes.size() - 1;
    const MeshData& m0 = p.meshes[0];
    const int64_t n0 = m0.n();
    p.L.assign(H + 1, LevelPlan());

    // ---- Dirichlet reduction (App. "Dirichlet Boundary Conditions")
    std::vector<int32_t> unk_of(n0, -1);
    p.unknowns.clear();
    for (int64_t v = 0; v < n0; v++)
        if (!p.known[v]) {
            unk_of[v] = (int32_t)p.unknowns.size();
            p.unknowns.push_back((int32_t)v);
        }
    if (p.unknowns.empty()) {
        err = "every vertex is Dirichlet-known";
        return SMG_ERR_INVALID_ARG;
    }
    std::vector<int32_t> kept_of;
    p.kept1.clear();
    if (H >= 1) {
        const ProlongationRaw& P1 = p.praw[0];
        std::vector<char> used(P1.n_coarse, 0);
        for (int32_t v : p.unknowns)
            for (int a = 0; a < 3; a++)
                if (P1.idx[3 * v + a] >= 0 && P1.w[3 * v + a] > 0) used[P1.idx[3 * v + a]] = 1;
        kept_of.assign(P1.n_coarse, -1);
        for (int64_t c = 0; c < P1.n_coarse; c++)
            if (used[c]) {
                kept_of[c] = (int32_t)p.kept1.size();
                p.kept1.push_back((int32_t)c);
            }
    }
    // level sizes and natural reduced prolongations
    for (int l = 0; l <= H; l++) {
        LevelPlan& lv = p.L[l];
        lv.coarsest = (l == H);
        lv.n = l == 0 ? (int64_t)p.unknowns.size() : (l == 1 ? (int64_t)p.kept1.size() : p.meshes[l].n());
    }
    for (int l = 0; l < H; l++) {
        LevelPlan& lv = p.L[l];
        const ProlongationRaw& P = p.praw[l];
        lv.pn_idx.assign(3 * lv.n, -1);
        lv.pn_w.assign(3 * lv.n, 0.0);
        for (int64_t r = 0; r < lv.n; r++) {
            int64_t src = l == 0 ? p.unknowns[r] : (l == 1 ? p.kept1[r] : r);
            int k = 0;
            for (int a = 0; a < 3; a++) {
                int32_t c = P.idx[3 * src + a];
                double w = P.w[3 * src + a];
                if (c < 0 || !(w > 0)) continue;
                int32_t cc = l == 0 ? kept_of[c] : c;
                if (cc < 0) {
                    err = "internal: kept column lookup failed";
                    return SMG_ERR_DECIMATION;
                }
                lv.pn_idx[3 * r + k] = cc;
                lv.pn_w[3 * r + k] = w;
                k++;
            }
            if (k == 0) {
                err = "prolongation row without weights";
                return SMG_ERR_DECIMATION;
            }
        }
        std::vector<char> hit(p.L[l + 1].n, 0);
        for (int64_t r = 0; r < lv.n; r++)
            for (int a = 0; a < 3; a++)
                if (lv.pn_idx[3 * r + a] >= 0) hit[lv.pn_idx[3 * r + a]] = 1;
        for (int64_t c = 0; c < p.L[l + 1].n; c++)
            if (!hit[c]) {
                err = "coarse vertex without support at level " + std::to_string(l + 1) +
                      " (too many Dirichlet-known vertices)";
                return SMG_ERR_DECIMATION;
            }
    }

    tm.mark("dirichlet + reduced P");
    // ---- unknowns per vertex: every vertex quantity becomes bs adjacent unknowns,
    // the prolongation P (x) I_bs (the weights act on each component alone)
    const int bs = p.opts.block_size;
    const int64_t nvu = p.L[0].n;  // vertex unknowns at level 0
    if (bs > 1) {
        for (int l = 0; l <= H; l++) {
            LevelPlan& lv = p.L[l];
            if (l < H) {
                std::vector<int32_t> idx(3 * bs * lv.n, -1);
                std::vector<double> w(3 * bs * lv.n, 0.0);
                for (int64_t r = 0; r < lv.n; r++)
                    for (int d = 0; d < bs; d++)
                        for (int a = 0; a < 3; a++) {
                            const int32_t c = lv.pn_idx[3 * r + a];
                            idx[3 * (bs * r + d) + a] = c < 0 ? -1 : bs * c + d;
                            w[3 * (bs * r + d) + a] = lv.pn_w[3 * r + a];
                        }
                lv.pn_idx.swap(idx);
                lv.pn_w.swap(w);
            }
            lv.n *= bs;
        }
    }
    // ---- symbolic patterns
    {
        LevelPlan& lv = p.L[0];
        std::vector<std::vector<int32_t>> adj(nvu);
        if (p.opts.pattern_rings == 2) {
            // 2-ring (Sec. 6: Bilaplacian, squared Hessian): unknowns joined by a path of
            // at most two mesh edges, through any vertex (known ones included, as in
            // L M^{-1} L)
            std::vector<std::vector<int32_t>> nb(n0);
            for (int64_t f = 0; f < m0.m(); f++)
                for (int c = 0; c < 3; c++) {
                    const int32_t a = m0.F[3 * f + c], b = m0.F[3 * f + (c + 1) % 3];
                    nb[a].push_back(b);
                    nb[b].push_back(a);
                }
            for (auto& v : nb) {
                std::sort(v.begin(), v.end());
                v.erase(std::unique(v.begin(), v.end()), v.end());
            }
            for (int64_t r = 0; r < nvu; r++) {
                const int32_t v = p.unknowns[r];
                for (int32_t w : nb[v]) {
                    if (unk_of[w] >= 0) adj[r].push_back(unk_of[w]);
                    for (int32_t z : nb[w])
                        if (unk_of[z] >= 0) adj[r].push_back(unk_of[z]);
                }
            }
        } else {
            for (int64_t f = 0; f < m0.m(); f++)
                for (int c = 0; c < 3; c++) {
                    int32_t a = unk_of[m0.F[3 * f + c]], b = unk_of[m0.F[3 * f + (c + 1) % 3]];
                    if (a >= 0 && b >= 0) {
                        adj[a].push_back(b);
                        adj[b].push_back(a);
                    }
                }
        }
        lv.rowptr.assign(lv.n + 1, 0);
        lv.col.clear();
        for (int64_t r = 0; r < nvu; r++) {
            auto& a = adj[r];
            a.push_back((int32_t)r);
            std::sort(a.begin(), a.end());
            a.erase(std::unique(a.begin(), a.end()), a.end());
        }
        for (int64_t row = 0; row < lv.n; row++) {  // unknown row = bs * vertex + component
            for (int32_t j : adj[row / bs])
                for (int e = 0; e < bs; e++) lv.col.push_back(bs * j + e);
            lv.rowptr[row + 1] = (int64_t)lv.col.size();
        }
    }
    for (int l = 0; l < H; l++)
        galerkin_pattern(p.L[l].n, p.L[l].rowptr, p.L[l].col, p.L[l].pn_idx, p.L[l + 1].n, p.L[l + 1].rowptr,
                         p.L[l + 1].col);
    if (p.L[H].n > 16384) {
        err = "coarsest level too large for the dense factor (" + std::to_string(p.L[H].n) + " > 16384)";
        return SMG_ERR_DECIMATION;
    }

    tm.mark("symbolic Galerkin patterns");
    // ---- colouring, permutation and SELL-32 layout per level
    for (int l = 0; l <= H; l++) {
        LevelPlan& lv = p.L[l];
        const int64_t n = lv.n;
        lv.perm.resize(n);
        lv.iperm.resize(n);
        if (lv.coarsest) {
            std::iota(lv.perm.begin(), lv.perm.end(), 0);
            std::iota(lv.iperm.begin(), lv.iperm.end(), 0);
            lv.ncolours = 0;
            lv.colour.clear();
            lv.nflat = n * n;
            continue;
        }
        std::vector<int32_t> len(n);
        for (int64_t r = 0; r < n; r++) len[r] = (int32_t)(lv.rowptr[r + 1] - lv.rowptr[r] - 1);
        std::iota(lv.perm.begin(), lv.perm.end(), 0);
        std::vector<int32_t> cls(n);  // launch class of every row
        if (bs == 1) {
            lv.ncolours = greedy_colouring(n, lv.rowptr, lv.col, lv.colour);
            cls = lv.colour;
            // colour classes one after another; longer rows first inside a class so a
            // warp's 32 rows have similar lengths (order inside a class does not change
            // the sweep: no two rows of a class are coupled)
            std::stable_sort(lv.perm.begin(), lv.perm.end(), [&](int32_t a, int32_t b) {
                if (lv.colour[a] != lv.colour[b]) return lv.colour[a] < lv.colour[b];
                return len[a] > len[b];
            });
        } else {
            // 3|V| systems: Alg. 3 on the vertex pattern; unknown (v, c) has colour
            // 3 C(v) + c and a vertex class is swept component by component in one
            // launch, so the launch classes are the vertex classes, with the three
            // unknowns of a vertex adjacent (longer rows first inside a class)
            const int64_t nv = n / bs;
            std::vector<int64_t> vrp(nv + 1, 0);
            std::vector<int32_t> vcol;
            for (int64_t v = 0; v < nv; v++) {
                for (int64_t q = lv.rowptr[bs * v]; q < lv.rowptr[bs * v + 1]; q++) {
                    const int32_t w = lv.col[q] / bs;
                    if (vcol.empty() || (int64_t)vcol.size() == vrp[v] || vcol.back() != w) vcol.push_back(w);
                }
                vrp[v + 1] = (int64_t)vcol.size();
            }
            std::vector<int32_t> vc;
            lv.ncolours = greedy_colouring(nv, vrp, vcol, vc);
            lv.colour.resize(n);
            for (int64_t r = 0; r < n; r++) {
                lv.colour[r] = bs * vc[r / bs] + (int32_t)(r % bs);
                cls[r] = vc[r / bs];
            }
            std::vector<int32_t> vperm(nv);
            std::iota(vperm.begin(), vperm.end(), 0);
            std::stable_sort(vperm.begin(), vperm.end(), [&](int32_t a, int32_t b) {
                if (vc[a] != vc[b]) return vc[a] < vc[b];
                return len[bs * a] > len[bs * b];
            });
            for (int64_t q = 0; q < nv; q++)
                for (int c = 0; c < bs; c++) lv.perm[bs * q + c] = bs * vperm[q] + c;
        }
        for (int64_t q = 0; q < n; q++) lv.iperm[lv.perm[q]] = (int32_t)q;
        const int rows_per_slice = kSlice;
        lv.colour_row.assign(lv.ncolours + 1, 0);
        for (int64_t r = 0; r < n; r++) lv.colour_row[cls[r] + 1]++;
        for (int c = 0; c < lv.ncolours; c++) lv.colour_row[c + 1] += lv.colour_row[c];
        lv.slices.clear();
        lv.colour_slice.assign(lv.ncolours + 1, 0);
        int64_t off = 0;
        for (int c = 0; c < lv.ncolours; c++) {
            for (int32_t r0 = lv.colour_row[c]; r0 < lv.colour_row[c + 1]; r0 += rows_per_slice) {
                SliceMeta s;
                s.row0 = r0;
                s.nrows = std::min(rows_per_slice, lv.colour_row[c + 1] - r0);
                s.width = 0;
                for (int k = 0; k < s.nrows; k++) s.width = std::max(s.width, len[lv.perm[r0 + k]]);
                if (off > (int64_t)INT32_MAX - (int64_t)s.width * kSlice) {
                    err = "level too large for 32-bit slot offsets";
                    return SMG_ERR_INVALID_ARG;
                }
                s.off = (int32_t)off;
                off += (int64_t)s.width * kSlice;
                lv.slices.push_back(s);
            }
            lv.colour_slice[c + 1] = (int32_t)lv.slices.size();
        }
        lv.nslots = off;
        lv.sbase = (n + kSlice - 1) / kSlice * kSlice;
        lv.nflat = lv.sbase + off;
        lv.sell_col.assign(off, 0);
        std::vector<int32_t> cols;
        for (const SliceMeta& s : lv.slices)
            for (int rl = 0; rl < rows_per_slice; rl++) {
                int32_t prow = s.row0 + (rl < s.nrows ? rl : 0);
                cols.clear();
                if (rl < s.nrows) {
                    int32_t r = lv.perm[prow];
                    for (int64_t q = lv.rowptr[r]; q < lv.rowptr[r + 1]; q++)
                        if (lv.col[q] != r) cols.push_back(lv.iperm[lv.col[q]]);
                    std::sort(cols.begin(), cols.end());
                }
                for (int k = 0; k < s.width; k++) lv.sell_col[slot_at(s, rl, k)] = k < (int)cols.size() ? cols[k] : prow;
            }
    }

    tm.mark("colouring + SELL layout");
    // ---- flat index -> natural CSR position
    for (int l = 0; l <= H; l++) {
        LevelPlan& lv = p.L[l];
        lv.flat_to_csr.assign(lv.nflat, -1);
        if (lv.coarsest) {
            for (int64_t I = 0; I < lv.n; I++)
                for (int64_t q = lv.rowptr[I]; q < lv.rowptr[I + 1]; q++) lv.flat_to_csr[I * lv.n + lv.col[q]] = q;
            continue;
        }
        for (int64_t pr = 0; pr < lv.n; pr++) lv.flat_to_csr[pr] = csr_find(lv.rowptr, lv.col, lv.perm[pr], lv.perm[pr]);
        for (const SliceMeta& s : lv.slices)
            for (int rl = 0; rl < s.nrows; rl++) {
                int32_t pr = s.row0 + rl;
                for (int k = 0; k < s.width; k++) {
                    int64_t slot = slot_at(s, rl, k);
                    int32_t pc = lv.sell_col[slot];
                    if (pc == pr) continue;
                    lv.flat_to_csr[lv.sbase + slot] = csr_find(lv.rowptr, lv.col, lv.perm[pr], lv.perm[pc]);
                }
            }
    }

    // ---- 3|V| systems: 3 x 3 block layout of every sparse level
    if (bs == 3)
        for (int l = 0; l < H; l++) {
            LevelPlan& lv = p.L[l];
            const int64_t nv = lv.n / 3;
            std::vector<int32_t> slice_of(lv.n, 0);
            for (size_t si = 0; si < lv.slices.size(); si++)
                for (int k = 0; k < lv.slices[si].nrows; k++) slice_of[lv.slices[si].row0 + k] = (int32_t)si;
            // neighbour vertices of every permuted vertex (ascending) and the flat
            // index of each scalar entry, keyed by (row component, column)
            std::vector<std::vector<int32_t>> nbr(nv);
            lv.d_src.assign(9 * nv, -1);
            for (int64_t pv = 0; pv < nv; pv++) {
                for (int a = 0; a < 3; a++) {
                    const int32_t pr = (int32_t)(3 * pv + a);
                    lv.d_src[(3 * a + a) * nv + pv] = pr;  // the diagonal entry
                    const SliceMeta& fs = lv.slices[slice_of[pr]];
                    const int rl = pr - fs.row0;
                    for (int k = 0; k < fs.width; k++) {
                        const int64_t slot = slot_at(fs, rl, k);
                        const int32_t pc = lv.sell_col[slot];
                        if (pc == pr) continue;
                        if (pc / 3 == pv) lv.d_src[(3 * a + pc % 3) * nv + pv] = (int32_t)(lv.sbase + slot);
                        else nbr[pv].push_back(pc / 3);
                    }
                }
                std::sort(nbr[pv].begin(), nbr[pv].end());
                nbr[pv].erase(std::unique(nbr[pv].begin(), nbr[pv].end()), nbr[pv].end());
            }
            lv.b_slices.clear();
            lv.b_colour_slice.assign(lv.ncolours + 1, 0);
            int64_t off = 0;
            for (int c = 0; c < lv.ncolours; c++) {
                const int32_t v0 = lv.colour_row[c] / 3, v1 = lv.colour_row[c + 1] / 3;
                for (int32_t q0 = v0; q0 < v1; q0 += kSlice) {
                    SliceMeta sm{};
                    sm.row0 = q0;
                    sm.nrows = std::min<int32_t>(kSlice, v1 - q0);
                    for (int r = 0; r < sm.nrows; r++) sm.width = std::max(sm.width, (int32_t)nbr[q0 + r].size());
                    if (9 * (off + (int64_t)sm.width * kSlice) > (int64_t)INT32_MAX) {
                        err = "level too large for 32-bit block slots";
                        return SMG_ERR_INVALID_ARG;
                    }
                    sm.off = (int32_t)off;
                    off += (int64_t)sm.width * kSlice;
                    lv.b_slices.push_back(sm);
                }
                lv.b_colour_slice[c + 1] = (int32_t)lv.b_slices.size();
            }
            lv.b_nslots = off;
            lv.b_col.assign(off, 0);
            lv.b_src.assign(9 * off, -1);
            for (const SliceMeta& sm : lv.b_slices)
                for (int r = 0; r < kSlice; r++) {
                    const int32_t pv = sm.row0 + (r < sm.nrows ? r : 0);
                    const int nk = r < sm.nrows ? (int)nbr[pv].size() : 0;
                    for (int k = 0; k < sm.width; k++) lv.b_col[(int64_t)sm.off + (int64_t)k * kSlice + r] = k < nk ? nbr[pv][k] : pv;
                    if (r >= sm.nrows) continue;
                    for (int a = 0; a < 3; a++) {
                        const int32_t pr = 3 * pv + a;
                        const SliceMeta& fs = lv.slices[slice_of[pr]];
                        const int rl = pr - fs.row0;
                        for (int k = 0; k < fs.width; k++) {
                            const int64_t slot = slot_at(fs, rl, k);
                            const int32_t pc = lv.sell_col[slot];
                            if (pc == pr || pc / 3 == pv) continue;
                            const int kb = (int)(std::lower_bound(nbr[pv].begin(), nbr[pv].end(), pc / 3) - nbr[pv].begin());
                            const int64_t at = 9 * (int64_t)sm.off + (int64_t)(9 * kb + 3 * a + pc % 3) * kSlice + r;
                            lv.b_src[at] = (int32_t)(lv.sbase + slot);
                        }
                    }
                }
        }

    tm.mark("flat -> CSR maps");
    // ---- permuted prolongation, restriction and Galerkin plans
    for (int l = 0; l < H; l++) {
        LevelPlan& lv = p.L[l];
        LevelPlan& nx = p.L[l + 1];
        const int64_t n = lv.n, nc = nx.n;
        lv.p_idx.assign(3 * n, 0);
        lv.p_w.assign(3 * n, 0.0);
        for (int64_t pr = 0; pr < n; pr++) {
            int32_t r = lv.perm[pr];
            int32_t first = nx.iperm[lv.pn_idx[3 * r]];
            for (int a = 0; a < 3; a++) {
                int32_t c = lv.pn_idx[3 * r + a];
                lv.p_idx[a * n + pr] = c >= 0 ? nx.iperm[c] : first;
                lv.p_w[a * n + pr] = c >= 0 ? lv.pn_w[3 * r + a] : 0.0;
            }
        }
        lv.pt_ptr.assign(nc + 1, 0);
        for (int64_t pr = 0; pr < n; pr++)
            for (int a = 0; a < 3; a++)
                if (lv.p_w[a * n + pr] != 0.0) lv.pt_ptr[lv.p_idx[a * n + pr] + 1]++;
        for (int64_t I = 0; I < nc; I++) lv.pt_ptr[I + 1] += lv.pt_ptr[I];
        lv.pt_row.assign(lv.pt_ptr[nc], 0);
        lv.pt_w.assign(lv.pt_ptr[nc], 0.0);
        {
            std::vector<int32_t> fill(lv.pt_ptr.begin(), lv.pt_ptr.end() - 1);
            for (int64_t pr = 0; pr < n; pr++)
                for (int a = 0; a < 3; a++)
                    if (lv.p_w[a * n + pr] != 0.0) {
                        int32_t I = lv.p_idx[a * n + pr];
                        lv.pt_row[fill[I]] = (int32_t)pr;
                        lv.pt_w[fill[I]] = lv.p_w[a * n + pr];
                        fill[I]++;
                    }
        }
        std::vector<int32_t> fine_slice(n, 0);
        for (size_t si = 0; si < lv.slices.size(); si++)
            for (int k = 0; k < lv.slices[si].nrows; k++) fine_slice[lv.slices[si].row0 + k] = (int32_t)si;
        // Entries of fine row pr as (column, flat index): the diagonal first, then
        // the off-diagonal slots in ascending column order.
        auto fine_row = [&](int32_t pr, std::vector<std::pair<int32_t, int32_t>>& out) {
            out.clear();
            out.emplace_back(pr, pr);
            const SliceMeta& fs = lv.slices[fine_slice[pr]];
            const int rl = pr - fs.row0;
            for (int k = 0; k < fs.width; k++) {
                const int64_t slot = slot_at(fs, rl, k);
                const int32_t pc = lv.sell_col[slot];
                if (pc != pr) out.emplace_back(pc, (int32_t)(lv.sbase + slot));
            }
        };
        // Slot a of P row pr that holds coarse row I.
        auto p_slot = [&](int32_t pr, int32_t I) -> int32_t {
            for (int a = 0; a < 3; a++)
                if (lv.p_w[a * n + pr] != 0.0 && lv.p_idx[a * n + pr] == I) return a;
            return -1;
        };
        if (lv.sbase + lv.nslots > (int64_t)INT32_MAX || 3 * n > (int64_t)INT32_MAX) {
            err = "level too large for 32-bit Galerkin indices";
            return SMG_ERR_INVALID_ARG;
        }
        // ---- Q = P^T A_l: columns of coarse row I = the fine rows of P^T row I
        // with their neighbours, ascending
        std::vector<int32_t> qlen(nc, 0);
        std::vector<std::vector<int32_t>> qcols_chunk;
        std::vector<int64_t> qrp(nc + 1, 0);
        std::vector<int32_t> qcols;
        {
            const int nt = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
            const int64_t chunks = nc < 4096 ? 1 : nt;
            qcols_chunk.assign(chunks, {});
            std::vector<std::thread> th;
            auto body = [&](int64_t c) {
                const int64_t I0 = nc * c / chunks, I1 = nc * (c + 1) / chunks;
                std::vector<int32_t> stamp(n, -1);
                std::vector<std::pair<int32_t, int32_t>> row;
                std::vector<int32_t> cols;
                for (int64_t I = I0; I < I1; I++) {
                    cols.clear();
                    for (int32_t t = lv.pt_ptr[I]; t < lv.pt_ptr[I + 1]; t++) {
                        fine_row(lv.pt_row[t], row);
                        for (auto& e : row)
                            if (stamp[e.first] != (int32_t)I) {
                                stamp[e.first] = (int32_t)I;
                                cols.push_back(e.first);
                            }
                    }
                    std::sort(cols.begin(), cols.end());
                    qlen[I] = (int32_t)cols.size();
                    qcols_chunk[c].insert(qcols_chunk[c].end(), cols.begin(), cols.end());
                }
            };
            for (int64_t c = 0; c + 1 < chunks; c++) th.emplace_back(body, c);
            body(chunks - 1);
            for (auto& x : th) x.join();
            for (int64_t I = 0; I < nc; I++) qrp[I + 1] = qrp[I] + qlen[I];
            qcols.reserve(qrp[nc]);
            for (auto& v : qcols_chunk) {
                qcols.insert(qcols.end(), v.begin(), v.end());
                std::vector<int32_t>().swap(v);
            }
        }
        // ---- layout: coarse rows by decreasing total width (ties: ascending row)
        lv.rq_row.resize(nc);
        std::iota(lv.rq_row.begin(), lv.rq_row.end(), 0);
        auto ptlen = [&](int32_t I) { return lv.pt_ptr[I + 1] - lv.pt_ptr[I]; };
        std::stable_sort(lv.rq_row.begin(), lv.rq_row.end(), [&](int32_t x, int32_t y) {
            return ptlen(x) + qlen[x] > ptlen(y) + qlen[y];
        });
        lv.rq_slices.clear();
        lv.rq_maxw = 0;
        {
            int64_t off = 0;
            for (int64_t p0 = 0; p0 < nc; p0 += kSlice) {
                RQSlice sl{};
                sl.pos0 = (int32_t)p0;
                sl.nrows = (int32_t)std::min<int64_t>(kSlice, nc - p0);
                for (int r = 0; r < sl.nrows; r++) {
                    const int32_t I = lv.rq_row[p0 + r];
                    sl.wb = std::max(sl.wb, ptlen(I));
                    sl.wq = std::max(sl.wq, qlen[I]);
                }
                if (off > (int64_t)INT32_MAX - (int64_t)(sl.wb + sl.wq) * kSlice) {
                    err = "level too large for 32-bit restriction slots";
                    return SMG_ERR_INVALID_ARG;
                }
                sl.off = (int32_t)off;
                off += (int64_t)(sl.wb + sl.wq) * kSlice;
                lv.rq_maxw = std::max(lv.rq_maxw, sl.wb + sl.wq);
                lv.rq_slices.push_back(sl);
            }
            lv.rq_col.assign(off, 0);
            lv.rq_w.assign(off, 0.0);
        }
        // position of every coarse row, and the stage-1 numbering of Q entries
        // (coarse rows in layout order, columns ascending)
        std::vector<int32_t> pos_of(nc);
        for (int64_t p0 = 0; p0 < nc; p0++) pos_of[lv.rq_row[p0]] = (int32_t)p0;
        std::vector<int64_t> qe0(nc + 1, 0);  // first Q entry of position p
        for (int64_t p0 = 0; p0 < nc; p0++) qe0[p0 + 1] = qe0[p0] + qlen[lv.rq_row[p0]];
        if (qe0[nc] > (int64_t)INT32_MAX) {
            err = "Galerkin plan too large";
            return SMG_ERR_INVALID_ARG;
        }
        lv.q_dst.assign(qe0[nc], 0);
        for (const RQSlice& sl : lv.rq_slices)
            for (int r = 0; r < kSlice; r++) {
                const bool ok = r < sl.nrows;
                const int32_t I = ok ? lv.rq_row[sl.pos0 + r] : 0;
                const int32_t nb = ok ? ptlen(I) : 0, nq = ok ? qlen[I] : 0;
                for (int k = 0; k < sl.wb; k++) {
                    const int64_t slot = (int64_t)sl.off + (int64_t)k * kSlice + r;
                    if (k < nb) {
                        lv.rq_col[slot] = lv.pt_row[lv.pt_ptr[I] + k];
                        lv.rq_w[slot] = -lv.pt_w[lv.pt_ptr[I] + k];
                    } else {
                        lv.rq_col[slot] = nb > 0 ? lv.pt_row[lv.pt_ptr[I]] : 0;
                    }
                }
                for (int k = 0; k < sl.wq; k++) {
                    const int64_t slot = (int64_t)sl.off + (int64_t)(sl.wb + k) * kSlice + r;
                    lv.rq_col[slot] = k < nq ? qcols[qrp[I] + k] : (nq > 0 ? qcols[qrp[I]] : 0);
                    if (k < nq) lv.q_dst[qe0[sl.pos0 + r] + k] = (int32_t)slot;
                }
            }
        // ---- stage 1 contributions: Q[I, j] = sum over the fine rows pr of P^T
        // row I (ascending) of P[pr, I] A_l[pr, j]
        lv.q_ptr.assign(qe0[nc] + 1, 0);
        std::atomic<bool> bad{false};
        for (int pass = 0; pass < 2 && !bad; pass++) {
            if (pass == 1) {
                int64_t tot = 0;
                for (int64_t e = 0; e < qe0[nc]; e++) {
                    tot += lv.q_ptr[e + 1];
                    if (tot > INT32_MAX - 1) {
                        err = "Galerkin plan too large";
                        return SMG_ERR_INVALID_ARG;
                    }
                    lv.q_ptr[e + 1] = (int32_t)tot;
                }
                lv.q_src.assign(tot, 0);
                lv.q_pw.assign(tot, 0);
            }
            parallel_rows(nc, [&](int64_t I0, int64_t I1) {
                std::vector<int32_t> loc(n, -1);
                std::vector<std::pair<int32_t, int32_t>> row;
                for (int64_t I = I0; I < I1 && !bad; I++) {
                    const int64_t e0 = qe0[pos_of[I]];
                    for (int64_t k = qrp[I]; k < qrp[I + 1]; k++) loc[qcols[k]] = (int32_t)(k - qrp[I]);
                    for (int32_t t = lv.pt_ptr[I]; t < lv.pt_ptr[I + 1]; t++) {
                        const int32_t pr = lv.pt_row[t];
                        const int32_t a = p_slot(pr, (int32_t)I);
                        if (a < 0) {
                            bad = true;
                            return;
                        }
                        fine_row(pr, row);
                        for (auto& en : row) {
                            const int64_t e = e0 + loc[en.first];
                            if (pass == 0) {
                                lv.q_ptr[e + 1]++;
                            } else {
                                const int32_t k = lv.q_ptr[e]++;
                                lv.q_src[k] = en.second;
                                lv.q_pw[k] = (int32_t)(a * n + pr);
                            }
                        }
                    }
                }
            });
            if (pass == 1) {  // the fill advanced every q_ptr[e] to the start of e + 1
                for (int64_t e = qe0[nc]; e > 0; e--) lv.q_ptr[e] = lv.q_ptr[e - 1];
                lv.q_ptr[0] = 0;
            }
        }
        // ---- stage 2 contributions: A_{l+1}[I, J] = sum over Q row I (ascending
        // fine column j) and the slots b of P row j with P[j, b] = J of Q[I, j] P[j, J]
        std::vector<int32_t> nx_slice_of_row;
        if (!nx.coarsest) {
            nx_slice_of_row.assign(nc, 0);
            for (size_t si = 0; si < nx.slices.size(); si++)
                for (int k = 0; k < nx.slices[si].nrows; k++) nx_slice_of_row[nx.slices[si].row0 + k] = (int32_t)si;
        }
        if (nx.nflat > (int64_t)INT32_MAX) {
            err = "level too large for 32-bit Galerkin indices";
            return SMG_ERR_INVALID_ARG;
        }
        lv.g_ptr.assign(nx.nflat + 1, 0);
        for (int pass = 0; pass < 2 && !bad; pass++) {
            if (pass == 1) {
                int64_t tot = 0;
                for (int64_t d = 0; d < nx.nflat; d++) {
                    tot += lv.g_ptr[d + 1];
                    if (tot > INT32_MAX - 1) {
                        err = "Galerkin plan too large";
                        return SMG_ERR_INVALID_ARG;
                    }
                    lv.g_ptr[d + 1] = (int32_t)tot;
                }
                lv.g_src.assign(tot, 0);
                lv.g_pw.assign(tot, 0);
            }
            parallel_rows(nc, [&](int64_t I0, int64_t I1) {
                std::vector<int32_t> stamp(nc, -1);
                std::vector<int64_t> slot_of(nc, -1);
                for (int64_t I = I0; I < I1 && !bad; I++) {
                    if (!nx.coarsest) {  // column -> flat slot of coarse row I
                        const SliceMeta& cs = nx.slices[nx_slice_of_row[I]];
                        const int rl = (int)(I - cs.row0);
                        for (int k = 0; k < cs.width; k++) {
                            int64_t slot = slot_at(cs, rl, k);
                            int32_t c = nx.sell_col[slot];
                            if (c == I) continue;
                            stamp[c] = (int32_t)I;
                            slot_of[c] = nx.sbase + slot;
                        }
                    }
                    auto dst_of = [&](int32_t J) -> int64_t {
                        if (nx.coarsest) return I * nc + J;
                        if (J == I) return I;
                        return stamp[J] == I ? slot_of[J] : -1;
                    };
                    const int64_t e0 = qe0[pos_of[I]];
                    for (int64_t k = qrp[I]; k < qrp[I + 1]; k++) {
                        const int32_t j = qcols[k];
                        const int32_t src = lv.q_dst[e0 + (k - qrp[I])];
                        for (int bb = 0; bb < 3; bb++) {
                            if (lv.p_w[bb * n + j] == 0.0) continue;
                            const int64_t d = dst_of(lv.p_idx[bb * n + j]);
                            if (d < 0) {
                                bad = true;
                                return;
                            }
                            if (pass == 0) {
                                lv.g_ptr[d + 1]++;
                            } else {
                                const int32_t q = lv.g_ptr[d]++;
                                lv.g_src[q] = src;
                                lv.g_pw[q] = (int32_t)(bb * n + j);
                            }
                        }
                    }
                }
            });
            if (pass == 1) {
                for (int64_t d = nx.nflat; d > 0; d--) lv.g_ptr[d] = lv.g_ptr[d - 1];
                lv.g_ptr[0] = 0;
            }
        }
        if (bad) {
            err = "internal: Galerkin destination missing from the symbolic pattern";
            return SMG_ERR_DECIMATION;
        }
    }

    tm.mark("transfer + Galerkin plans");
    // ---- level-0 assembly plan
    AssemblyPlan& A = p.asmb;
    const LevelPlan& l0 = p.L[0];
    A.nv = n0;
    A.nf = m0.m();
    A.F = m0.F;
    A.row_vertex.resize(l0.n);
    std::vector<int8_t> row_comp(l0.n);  // component of the row's unknown (0 when bs = 1)
    for (int64_t pr = 0; pr < l0.n; pr++) {
        A.row_vertex[pr] = p.unknowns[l0.perm[pr] / bs];
        row_comp[pr] = (int8_t)(l0.perm[pr] % bs);
    }
    {
        std::vector<int32_t> cnt(n0 + 1, 0);
        for (int64_t f = 0; f < A.nf; f++)
            for (int c = 0; c < 3; c++) cnt[A.F[3 * f + c] + 1]++;
        for (int64_t v = 0; v < n0; v++) cnt[v + 1] += cnt[v];
        std::vector<int32_t> vc(cnt[n0]);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t f = 0; f < A.nf; f++)
            for (int c = 0; c < 3; c++) vc[fill[A.F[3 * f + c]]++] = (int32_t)(3 * f + c);
        A.vinc_ptr.assign(cnt.begin(), cnt.end());
        A.vinc_code = vc;
        A.vert_unk = unk_of;
        A.inc_ptr.assign(l0.n + 1, 0);
        A.inc_code.clear();
        for (int64_t pr = 0; pr < l0.n; pr++) {
            int32_t v = A.row_vertex[pr];
            for (int32_t q = cnt[v]; q < cnt[v + 1]; q++) A.inc_code.push_back(vc[q]);
            A.inc_ptr[pr + 1] = (int32_t)A.inc_code.size();
        }
    }
    {
        // corners opposite edge (a, b): the two smallest corner codes 3f + c over
        // the faces f around a that also hold b, c the corner that is neither
        auto opp_of = [&](int64_t a, int64_t b, int32_t& o0, int32_t& o1) {
            o0 = o1 = -1;
            for (int32_t q = A.vinc_ptr[a]; q < A.vinc_ptr[a + 1]; q++) {
                const int32_t code = A.vinc_code[q];
                const int64_t f = code / 3;
                const int ca = code % 3;
                for (int c = 0; c < 3; c++) {
                    if (c == ca || A.F[3 * f + c] != b) continue;
                    const int32_t o = (int32_t)(3 * f + (3 - ca - c));
                    if (o0 < 0 || o < o0) { o1 = o0; o0 = o; }
                    else if (o1 < 0 || o < o1) { o1 = o; }
                }
            }
        };
        A.opp0.assign(l0.nflat, -1);
        A.opp1.assign(l0.nflat, -1);
        if (l0.coarsest) {
            for (int64_t I = 0; I < l0.n; I++)
                for (int64_t J = 0; J < l0.n; J++)
                    if (I != J && row_comp[I] == row_comp[J] && A.row_vertex[I] != A.row_vertex[J])
                        opp_of(A.row_vertex[I], A.row_vertex[J], A.opp0[I * l0.n + J], A.opp1[I * l0.n + J]);
        } else {
            for (const SliceMeta& s : l0.slices)
                for (int rl = 0; rl < s.nrows; rl++)
                    for (int k = 0; k < s.width; k++) {
                        int64_t slot = slot_at(s, rl, k);
                        int32_t pc = l0.sell_col[slot];
                        if (pc == s.row0 + rl || row_comp[pc] != row_comp[s.row0 + rl] ||
                            A.row_vertex[pc] == A.row_vertex[s.row0 + rl])
                            continue;  // other components of a vertex, or of a neighbour: (x) I_bs
                        opp_of(A.row_vertex[s.row0 + rl], A.row_vertex[pc], A.opp0[l0.sbase + slot],
                               A.opp1[l0.sbase + slot]);
                    }
        }
        A.flat_to_user = l0.flat_to_csr;
    }
    tm.mark("assembly plan");
    return SMG_OK;
}

}  // namespace smg
