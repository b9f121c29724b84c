// Uniform mid-point edge collapse with successive self-parameterization.
//
// Sec. 4.1 (successive self-parameterization, Eq. composition): each collapse
// gets its own bijective map between the edge 1-ring before and the vertex
// 1-ring after; the level-to-level map is their composition.
// Sec. 4.2 (joint flattening, Eq. jointEnergy1 / jointEnergy): both patches are
// flattened at once by minimising E(before) + E(after) over a joint UV variable
// whose patch-boundary entries are shared.  E is LSCM (Sec. 4.4: uniform
// decimation with LSCM gave the best convergence).
// Sec. 4.3 (boundary edges): an edge with one boundary vertex shares that
// vertex's UV with the new vertex; a boundary edge tries k = i, k = j and k on
// the line ij, each with its colinearity constraints v = 0, and keeps the
// lowest energy among the valid ones.
// Sec. 4.5 / App. "SSP": a fine vertex is carried through the collapses as a
// barycentric point; its final coordinates in a coarse triangle give a row of P.
//
// Readings where the paper is silent: priority = current edge length (shortest
// first); the new vertex sits at the 3D midpoint; the LSCM gauge pins the two
// patch-boundary vertices farthest apart; a collapse is rejected if it breaks
// the link condition, pinches the boundary, inverts a UV or 3D triangle, gives
// a patch vertex a winding other than one turn, or makes a 3D angle below 1
// degree (the validity rules the paper defers to another paper).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "smg_host.hpp"

namespace smg {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTanMinAngle = 0.017455064928217585;  // tan(1 degree)

struct V3 {
    double x, y, z;
};
inline V3 v3sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 v3cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double v3dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline double v3norm(V3 a) { return std::sqrt(v3dot(a, a)); }

struct HeapItem {
    double len2;
    int32_t a, b;
};
inline bool heap_less(const HeapItem& x, const HeapItem& y) {
    if (x.len2 != y.len2) return x.len2 < y.len2;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
}

// 4-ary min-heap: shallower than a binary heap, so fewer cache misses per pop.
class EdgeHeap {
   public:
    void assign(std::vector<HeapItem>&& v) {
        h_ = std::move(v);
        for (int64_t i = ((int64_t)h_.size() - 2) / 4; i >= 0; i--) down(i);
    }
    bool empty() const { return h_.empty(); }
    const HeapItem& top() const { return h_[0]; }
    void push(const HeapItem& x) {
        h_.push_back(x);
        int64_t i = (int64_t)h_.size() - 1;
        while (i > 0) {
            int64_t p = (i - 1) / 4;
            if (!heap_less(h_[i], h_[p])) break;
            std::swap(h_[i], h_[p]);
            i = p;
        }
    }
    void pop() {
        h_[0] = h_.back();
        h_.pop_back();
        if (!h_.empty()) down(0);
    }

   private:
    std::vector<HeapItem> h_;
    void down(int64_t i) {
        const int64_t n = (int64_t)h_.size();
        HeapItem x = h_[i];
        for (;;) {
            int64_t c = 4 * i + 1;
            if (c >= n) break;
            int64_t best = c;
            int64_t e = std::min(c + 4, n);
            for (int64_t k = c + 1; k < e; k++)
                if (heap_less(h_[k], h_[best])) best = k;
            if (!heap_less(h_[best], x)) break;
            h_[i] = h_[best];
            i = best;
        }
        h_[i] = x;
    }
};

// A small dense least-squares system: rows of the LSCM energy over 2*nv reals.
struct Flattening {
    int nv = 0;
    std::vector<double> N;    // (2nv)^2 normal matrix
    double energy_scale = 0;  // sum of areas
    mutable std::vector<char> isfix;
    mutable std::vector<int> freeidx;
    void reset(int nvars) {
        nv = nvars;
        N.assign((size_t)4 * nv * nv, 0.0);
        energy_scale = 0;
    }
    // LSCM term of one 3D triangle whose corners use variables t0, t1, t2:
    // E_T = |sum_c W_c w_c|^2 / (16 A), W_c = z_{c+1} - z_{c+2}, z the triangle in
    // a local orthonormal frame and w = u + i v its UV image.
    bool add_triangle(V3 p0, V3 p1, V3 p2, int t0, int t1, int t2) {
        V3 e1 = v3sub(p1, p0), e2 = v3sub(p2, p0);
        double l1 = v3norm(e1);
        V3 nrm = v3cross(e1, e2);
        double dbl = v3norm(nrm);
        if (!(l1 > 0) || !(dbl > 0)) return false;
        V3 ex = {e1.x / l1, e1.y / l1, e1.z / l1};
        V3 ey = v3cross({nrm.x / dbl, nrm.y / dbl, nrm.z / dbl}, ex);
        double zx[3] = {0.0, l1, v3dot(e2, ex)};
        double zy[3] = {0.0, 0.0, v3dot(e2, ey)};
        double area = 0.5 * dbl;
        double s = 1.0 / std::sqrt(16.0 * area);
        int t[3] = {t0, t1, t2};
        double a[3], b[3];
        for (int c = 0; c < 3; c++) {
            a[c] = s * (zx[(c + 1) % 3] - zx[(c + 2) % 3]);
            b[c] = s * (zy[(c + 1) % 3] - zy[(c + 2) % 3]);
        }
        // Real row: sum a u - b v ; imaginary row: sum b u + a v
        int idx[6];
        double re[6], im[6];
        for (int c = 0; c < 3; c++) {
            idx[2 * c] = 2 * t[c];
            idx[2 * c + 1] = 2 * t[c] + 1;
            re[2 * c] = a[c];
            re[2 * c + 1] = -b[c];
            im[2 * c] = b[c];
            im[2 * c + 1] = a[c];
        }
        int d = 2 * nv;
        for (int r = 0; r < 6; r++)
            for (int q = 0; q < 6; q++) N[(size_t)idx[r] * d + idx[q]] += re[r] * re[q] + im[r] * im[q];
        energy_scale += area;
        return true;
    }
    // Minimise with the coordinates in `fixed` (index into 2nv) held at `fixval`.
    // Returns false if the reduced normal matrix is not positive definite.
    bool solve(const std::vector<int>& fixed, const std::vector<double>& fixval, std::vector<double>& u,
               std::vector<double>& work) const {
        int d = 2 * nv;
        isfix.assign(d, 0);
        u.assign(d, 0.0);
        for (size_t k = 0; k < fixed.size(); k++) {
            isfix[fixed[k]] = 1;
            u[fixed[k]] = fixval[k];
        }
        freeidx.clear();
        for (int q = 0; q < d; q++)
            if (!isfix[q]) freeidx.push_back(q);
        int f = (int)freeidx.size();
        work.assign((size_t)f * f + f, 0.0);
        double* K = work.data();
        double* r = work.data() + (size_t)f * f;
        for (int a = 0; a < f; a++) {
            int ia = freeidx[a];
            for (int b = 0; b < f; b++) K[(size_t)a * f + b] = N[(size_t)ia * d + freeidx[b]];
            double s = 0;
            for (size_t k = 0; k < fixed.size(); k++) s -= N[(size_t)ia * d + fixed[k]] * fixval[k];
            r[a] = s;
        }
        // Cholesky in place (lower), then two triangular solves
        for (int j = 0; j < f; j++) {
            double dj = K[(size_t)j * f + j];
            for (int k = 0; k < j; k++) dj -= K[(size_t)j * f + k] * K[(size_t)j * f + k];
            if (!(dj > 1e-300)) return false;
            double ljj = std::sqrt(dj);
            K[(size_t)j * f + j] = ljj;
            const double* Kj = K + (size_t)j * f;
            int i = j + 1;
            // four rows' sums side by side: each keeps its own order of
            // operations, so the factor is bitwise the one-row-at-a-time one
            for (; i + 3 < f; i += 4) {
                double* K0 = K + (size_t)i * f;
                double* K1 = K0 + f;
                double* K2 = K1 + f;
                double* K3 = K2 + f;
                double s0 = K0[j], s1 = K1[j], s2 = K2[j], s3 = K3[j];
                for (int k = 0; k < j; k++) {
                    const double jk = Kj[k];
                    s0 -= K0[k] * jk;
                    s1 -= K1[k] * jk;
                    s2 -= K2[k] * jk;
                    s3 -= K3[k] * jk;
                }
                K0[j] = s0 / ljj;
                K1[j] = s1 / ljj;
                K2[j] = s2 / ljj;
                K3[j] = s3 / ljj;
            }
            for (; i < f; i++) {
                double s = K[(size_t)i * f + j];
                for (int k = 0; k < j; k++) s -= K[(size_t)i * f + k] * K[(size_t)j * f + k];
                K[(size_t)i * f + j] = s / ljj;
            }
        }
        for (int i = 0; i < f; i++) {
            double s = r[i];
            for (int k = 0; k < i; k++) s -= K[(size_t)i * f + k] * r[k];
            r[i] = s / K[(size_t)i * f + i];
        }
        for (int i = f - 1; i >= 0; i--) {
            double s = r[i];
            for (int k = i + 1; k < f; k++) s -= K[(size_t)k * f + i] * r[k];
            r[i] = s / K[(size_t)i * f + i];
        }
        for (int a = 0; a < f; a++) u[freeidx[a]] = r[a];
        return true;
    }
    double energy(const std::vector<double>& u) const {
        int d = 2 * nv;
        double e = 0;
        for (int a = 0; a < d; a++)
            for (int b = 0; b < d; b++) e += u[a] * N[(size_t)a * d + b] * u[b];
        return e;
    }
};

inline double cross2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

class Decimator {
   public:
    explicit Decimator(const MeshData& fine);
    int run(int64_t target, MeshData& coarse, ProlongationRaw& P, DecimationStats& st, std::string& err);

   private:
    // ---- mesh state
    int64_t n_ = 0, m_ = 0, alive_count_ = 0;
    std::vector<double> pos_;
    std::vector<int32_t> fv_;
    std::vector<char> valive_, falive_, vbnd_;
    std::vector<std::vector<int32_t>> vf_;
    // ---- tracked points (one per fine vertex)
    std::vector<int32_t> pface_;  // -1: still exactly at its own vertex
    std::vector<double> pbary_;
    std::vector<std::vector<int32_t>> fpts_;
    EdgeHeap heap_;
    DecimationStats* st_ = nullptr;

    // ---- per-collapse scratch
    std::vector<int32_t> Fb_, S_, Fa_, ring_;
    std::vector<int> var_of_;  // vertex -> variable (before roles), -1 if not in patch
    Flattening flat_;
    std::vector<double> u_, best_u_, work_;
    std::vector<int32_t> nb_, occ_, opp_, ni_, nj_, common_, moving_;
    std::vector<int> fixed_;
    std::vector<double> fixval_, angsum_, before_sum_, muv_, fuv_;
    std::vector<std::pair<int32_t, int>> bv_;
    // rejected edges, listed at both endpoints; re-queued when a neighbourhood changes
    std::vector<std::vector<int32_t>> rej_;

    V3 P(int32_t v) const { return {pos_[3 * v], pos_[3 * v + 1], pos_[3 * v + 2]}; }
    void push_edge(int32_t a, int32_t b);
    void push_vertex_edges(int32_t v);
    void neighbours(int32_t v, std::vector<int32_t>& out) const;
    bool boundary_neighbours(int32_t v, int32_t nb[2]) const;
    bool try_collapse(int32_t i, int32_t j);
};

Decimator::Decimator(const MeshData& fine) {
    n_ = fine.n();
    m_ = fine.m();
    pos_ = fine.V;
    fv_ = fine.F;
    valive_.assign(n_, 1);
    falive_.assign(m_, 1);
    vbnd_.assign(n_, 0);
    vf_.assign(n_, {});
    for (int64_t f = 0; f < m_; f++)
        for (int c = 0; c < 3; c++) vf_[fv_[3 * f + c]].push_back((int32_t)f);
    // boundary: an edge (v, w) seen in exactly one face around v
    std::vector<int32_t> nb;
    for (int64_t v = 0; v < n_; v++) {
        nb.clear();
        for (int32_t f : vf_[v])
            for (int c = 0; c < 3; c++) {
                int32_t w = fv_[3 * f + c];
                if (w != v) nb.push_back(w);
            }
        std::sort(nb.begin(), nb.end());
        for (size_t a = 0; a < nb.size();) {
            size_t b = a;
            while (b < nb.size() && nb[b] == nb[a]) b++;
            if (b - a == 1) vbnd_[v] = 1;
            a = b;
        }
    }
    pface_.assign(n_, -1);
    pbary_.assign(3 * n_, 0.0);
    fpts_.assign(m_, {});
    alive_count_ = n_;
    var_of_.assign(n_, -1);
    rej_.assign(n_, {});
}

void Decimator::push_edge(int32_t a, int32_t b) {
    if (a > b) std::swap(a, b);
    V3 d = v3sub(P(a), P(b));
    heap_.push({v3dot(d, d), a, b});
}

void Decimator::neighbours(int32_t v, std::vector<int32_t>& out) const {
    out.clear();
    for (int32_t f : vf_[v])
        for (int c = 0; c < 3; c++) {
            int32_t w = fv_[3 * f + c];
            if (w != v) out.push_back(w);
        }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
}

void Decimator::push_vertex_edges(int32_t v) {
    neighbours(v, nb_);
    for (int32_t w : nb_) push_edge(v, w);
}

bool Decimator::boundary_neighbours(int32_t v, int32_t nb[2]) const {
    std::vector<int32_t>& occ = const_cast<Decimator*>(this)->occ_;
    occ.clear();
    for (int32_t f : vf_[v])
        for (int c = 0; c < 3; c++) {
            int32_t w = fv_[3 * f + c];
            if (w != v) occ.push_back(w);
        }
    std::sort(occ.begin(), occ.end());
    int cnt = 0;
    for (size_t a = 0; a < occ.size();) {
        size_t b = a;
        while (b < occ.size() && occ[b] == occ[a]) b++;
        if (b - a == 1) {
            if (cnt < 2) nb[cnt] = occ[a];
            cnt++;
        }
        a = b;
    }
    return cnt == 2;
}

bool Decimator::try_collapse(int32_t i, int32_t j) {
    DecimationStats& st = *st_;
    // ---------------- topology
    Fb_.clear();
    S_.clear();
    for (int32_t f : vf_[i]) Fb_.push_back(f);
    for (int32_t f : vf_[j]) {
        bool has_i = fv_[3 * f] == i || fv_[3 * f + 1] == i || fv_[3 * f + 2] == i;
        if (has_i) S_.push_back(f);
        else Fb_.push_back(f);
    }
    if (S_.empty() || S_.size() > 2) {
        st.rejected_link++;
        return false;
    }
    const bool edge_bnd = S_.size() == 1;
    std::vector<int32_t>& opp = opp_;
    opp.clear();
    for (int32_t f : S_)
        for (int c = 0; c < 3; c++) {
            int32_t w = fv_[3 * f + c];
            if (w != i && w != j) opp.push_back(w);
        }
    std::sort(opp.begin(), opp.end());
    {   // link condition: common neighbours of i and j are exactly the opposite vertices
        std::vector<int32_t>&ni = ni_, &nj = nj_, &common = common_;
        common.clear();
        neighbours(i, ni);
        neighbours(j, nj);
        std::set_intersection(ni.begin(), ni.end(), nj.begin(), nj.end(), std::back_inserter(common));
        if (common != opp) {
            st.rejected_link++;
            return false;
        }
        if (edge_bnd && (ni.size() < 2 || nj.size() < 2)) {
            st.rejected_boundary++;
            return false;
        }
    }
    const bool bi = vbnd_[i], bj = vbnd_[j];
    if (bi && bj && !edge_bnd) {  // would pinch the boundary
        st.rejected_boundary++;
        return false;
    }
    if (!edge_bnd && alive_count_ <= 4) {
        st.rejected_boundary++;
        return false;
    }
    int32_t bp = -1, bq = -1;  // previous / next boundary vertex of a boundary edge
    if (edge_bnd) {
        int32_t nbi[2], nbj[2];
        if (!boundary_neighbours(i, nbi) || !boundary_neighbours(j, nbj)) {
            st.rejected_boundary++;
            return false;
        }
        bp = nbi[0] == j ? nbi[1] : nbi[0];
        bq = nbj[0] == i ? nbj[1] : nbj[0];
        if (bp == bq || bp == j || bq == i) {
            st.rejected_boundary++;  // boundary loop too short
            return false;
        }
    }

    // ---------------- ring and variables
    ring_.clear();
    for (int32_t f : Fb_)
        for (int c = 0; c < 3; c++) {
            int32_t w = fv_[3 * f + c];
            if (w != i && w != j) ring_.push_back(w);
        }
    std::sort(ring_.begin(), ring_.end());
    ring_.erase(std::unique(ring_.begin(), ring_.end()), ring_.end());
    for (size_t a = 0; a < ring_.size(); a++) var_of_[ring_[a]] = (int)a;
    const int nr = (int)ring_.size();
    const V3 pi = P(i), pj = P(j);
    const V3 pk = {0.5 * (pi.x + pj.x), 0.5 * (pi.y + pj.y), 0.5 * (pi.z + pj.z)};

    Fa_.clear();
    for (int32_t f : Fb_)
        if (std::find(S_.begin(), S_.end(), f) == S_.end()) Fa_.push_back(f);

    // cases: 0 interior; 1 boundary vertex i; 2 boundary vertex j; 3,4,5 boundary edge (k=i, k=j, k on ij)
    int cases[3], ncases = 1;
    if (edge_bnd) { cases[0] = 3; cases[1] = 4; cases[2] = 5; ncases = 3; }
    else cases[0] = bi ? 1 : (bj ? 2 : 0);

    // 3D quality of the new triangles (independent of the flattening)
    for (int32_t f : Fa_) {
        V3 q[3];
        for (int c = 0; c < 3; c++) {
            int32_t w = fv_[3 * f + c];
            q[c] = (w == i || w == j) ? pk : P(w);
        }
        V3 nb = v3cross(v3sub(P(fv_[3 * f + 1]), P(fv_[3 * f])), v3sub(P(fv_[3 * f + 2]), P(fv_[3 * f])));
        V3 na = v3cross(v3sub(q[1], q[0]), v3sub(q[2], q[0]));
        if (!(v3dot(na, nb) > 0)) {
            for (int32_t r : ring_) var_of_[r] = -1;
            st.rejected_flip++;
            return false;
        }
        for (int c = 0; c < 3; c++) {
            // angle < 1 degree  <=>  cos > 0 and |sin| < tan(1 deg) cos
            V3 e1 = v3sub(q[(c + 1) % 3], q[c]), e2 = v3sub(q[(c + 2) % 3], q[c]);
            double dt = v3dot(e1, e2);
            if (dt > 0 && !(v3norm(v3cross(e1, e2)) >= kTanMinAngle * dt)) {
                for (int32_t r : ring_) var_of_[r] = -1;
                st.rejected_quality++;
                return false;
            }
        }
    }

    double best_e = 0;
    int best_case = -1;
    int best_vi = -1, best_vj = -1, best_vk = -1, best_nv = 0;
    int last_reason = 0;  // 1 solve, 2 flip, 3 angle
    for (int ci_ = 0; ci_ < ncases; ci_++) {
        const int cs = cases[ci_];
        // variable ids: ring 0..nr-1, then i, j, k as the case shares them
        int vi = nr, vj = nr + 1, vk = nr + 2, nv = nr + 3;
        if (cs == 1 || cs == 3) { vk = vi; vj = nr + 1; nv = nr + 2; }
        if (cs == 2 || cs == 4) { vk = vj; nv = nr + 2; }
        auto var_before = [&](int32_t w) { return w == i ? vi : (w == j ? vj : var_of_[w]); };
        auto var_after = [&](int32_t w) { return (w == i || w == j) ? vk : var_of_[w]; };
        flat_.reset(nv);
        bool ok = true;
        for (int32_t f : Fb_) {
            int32_t a = fv_[3 * f], b = fv_[3 * f + 1], c = fv_[3 * f + 2];
            ok &= flat_.add_triangle(P(a), P(b), P(c), var_before(a), var_before(b), var_before(c));
        }
        for (int32_t f : Fa_) {
            int32_t a = fv_[3 * f], b = fv_[3 * f + 1], c = fv_[3 * f + 2];
            V3 qa = (a == i || a == j) ? pk : P(a), qb = (b == i || b == j) ? pk : P(b),
               qc = (c == i || c == j) ? pk : P(c);
            ok &= flat_.add_triangle(qa, qb, qc, var_after(a), var_after(b), var_after(c));
        }
        if (!ok) { last_reason = 1; continue; }
        std::vector<int>& fixed = fixed_;
        std::vector<double>& fixval = fixval_;
        fixed.clear();
        fixval.clear();
        if (cs <= 2) {
            // gauge: the two patch-boundary vertices farthest apart, at (0,0) and (d,0)
            std::vector<std::pair<int32_t, int>>& bv = bv_;
            bv.clear();
            for (int32_t r : ring_) bv.push_back({r, var_of_[r]});
            if (cs == 1) bv.push_back({i, vi});
            if (cs == 2) bv.push_back({j, vj});
            double dmax = -1;
            int pa = -1, pb = -1;
            for (size_t a = 0; a < bv.size(); a++)
                for (size_t b = a + 1; b < bv.size(); b++) {
                    double d = v3norm(v3sub(P(bv[a].first), P(bv[b].first)));
                    if (d > dmax) { dmax = d; pa = bv[a].second; pb = bv[b].second; }
                }
            fixed = {2 * pa, 2 * pa + 1, 2 * pb, 2 * pb + 1};
            fixval = {0.0, 0.0, dmax, 0.0};
        } else {
            // colinear vertices on v = 0; x of the two ends fixed by 3D path length
            double lpi = v3norm(v3sub(P(bp), pi)), lij = v3norm(v3sub(pi, pj)), ljq = v3norm(v3sub(pj, P(bq)));
            int vp = var_of_[bp], vq = var_of_[bq];
            // the patch must lie left of the line (positive orientation): run the
            // line from p to q along +u when the surviving face holds i -> j
            int32_t fs = S_[0];
            int ci = fv_[3 * fs] == i ? 0 : (fv_[3 * fs + 1] == i ? 1 : 2);
            double sg = fv_[3 * fs + (ci + 1) % 3] == j ? 1.0 : -1.0;
            int line[5], nline = 0;
            if (cs == 3) {
                line[0] = vi; line[1] = vj; line[2] = vq; nline = 3;
                fixed = {2 * vi, 2 * vq};
                fixval = {0.0, sg * (lij + ljq)};
            }
            if (cs == 4) {
                line[0] = vp; line[1] = vi; line[2] = vj; nline = 3;
                fixed = {2 * vp, 2 * vj};
                fixval = {0.0, sg * (lpi + lij)};
            }
            if (cs == 5) {
                line[0] = vp; line[1] = vi; line[2] = vk; line[3] = vj; line[4] = vq; nline = 5;
                fixed = {2 * vp, 2 * vq};
                fixval = {0.0, sg * (lpi + lij + ljq)};
            }
            for (int q = 0; q < nline; q++) { fixed.push_back(2 * line[q] + 1); fixval.push_back(0.0); }
        }
        if (!flat_.solve(fixed, fixval, u_, work_)) { last_reason = 1; continue; }
        // ---- validity: positive UV triangles, one turn around interior patch vertices
        double scale = 0;
        for (size_t q = 0; q < fixval.size(); q++) scale = std::max(scale, std::fabs(fixval[q]));
        double amin = 1e-12 * scale * scale;
        std::vector<double>& angsum = angsum_;
        angsum.assign(nv, 0.0);
        double uv_area = 0;
        auto tri_ok = [&](int t0, int t1, int t2) {
            double x0 = u_[2 * t0], y0 = u_[2 * t0 + 1], x1 = u_[2 * t1], y1 = u_[2 * t1 + 1];
            double x2 = u_[2 * t2], y2 = u_[2 * t2 + 1];
            double ar = 0.5 * cross2(x1 - x0, y1 - y0, x2 - x0, y2 - y0);
            if (!(ar > amin)) return false;
            uv_area += ar;
            int tt[3] = {t0, t1, t2};
            double xs[3] = {x0, x1, x2}, ys[3] = {y0, y1, y2};
            for (int c = 0; c < 3; c++) {
                if (tt[c] < nr) continue;  // winding is checked at i, j, k only
                double ax = xs[(c + 1) % 3] - xs[c], ay = ys[(c + 1) % 3] - ys[c];
                double bx = xs[(c + 2) % 3] - xs[c], by = ys[(c + 2) % 3] - ys[c];
                angsum[tt[c]] += std::atan2(cross2(ax, ay, bx, by), ax * bx + ay * by);
            }
            return true;
        };
        bool valid = true;
        for (int32_t f : Fb_) {
            int32_t a = fv_[3 * f], b = fv_[3 * f + 1], c = fv_[3 * f + 2];
            valid &= tri_ok(var_before(a), var_before(b), var_before(c));
        }
        std::vector<double>& before_sum = before_sum_;
        before_sum = angsum;
        std::fill(angsum.begin(), angsum.end(), 0.0);
        for (int32_t f : Fa_) {
            int32_t a = fv_[3 * f], b = fv_[3 * f + 1], c = fv_[3 * f + 2];
            valid &= tri_ok(var_after(a), var_after(b), var_after(c));
        }
        if (!valid) { last_reason = 2; continue; }
        const double tol = 1e-6;
        bool wind = true;
        if (cs == 0) {
            wind &= std::fabs(before_sum[vi] - 2 * kPi) < tol && std::fabs(before_sum[vj] - 2 * kPi) < tol;
            wind &= std::fabs(angsum[vk] - 2 * kPi) < tol;
        } else if (cs == 1 || cs == 2) {
            int vin = cs == 1 ? vj : vi;  // the interior one of i, j
            wind &= std::fabs(before_sum[vin] - 2 * kPi) < tol;
            wind &= angsum[vk] < 2 * kPi - tol;
        } else {
            wind &= angsum[vk] < 2 * kPi - tol;
        }
        if (!wind) { last_reason = 3; continue; }
        // LSCM energy scales with the square of the UV size: compare cases per UV area
        double e = flat_.energy(u_) / uv_area;
        if (best_case < 0 || e < best_e) {
            best_e = e;
            best_case = cs;
            best_u_ = u_;
            best_vi = vi; best_vj = vj; best_vk = vk; best_nv = nv;
        }
    }
    if (best_case < 0) {
        for (int32_t r : ring_) var_of_[r] = -1;
        if (last_reason == 1) st.rejected_solve++;
        else if (last_reason == 3) st.rejected_angle++;
        else st.rejected_flip++;
        return false;
    }
    (void)best_nv;

    // ---------------- relocate tracked points through the joint UV domain
    const std::vector<double>& U = best_u_;
    auto var_before = [&](int32_t w) { return w == i ? best_vi : (w == j ? best_vj : var_of_[w]); };
    auto var_after = [&](int32_t w) { return (w == i || w == j) ? best_vk : var_of_[w]; };
    std::vector<int32_t>& moving = moving_;
    std::vector<double>& muv = muv_;
    moving.clear();
    muv.clear();
    for (int32_t f : Fb_) {
        for (int32_t p : fpts_[f]) {
            double x = 0, y = 0;
            for (int c = 0; c < 3; c++) {
                int t = var_before(fv_[3 * f + c]);
                x += pbary_[3 * p + c] * U[2 * t];
                y += pbary_[3 * p + c] * U[2 * t + 1];
            }
            moving.push_back(p);
            muv.push_back(x);
            muv.push_back(y);
        }
        fpts_[f].clear();
    }
    for (int32_t v : {i, j})
        if (pface_[v] < 0) {  // the fine vertex still sitting exactly on v
            int t = var_before(v);
            moving.push_back(v);
            muv.push_back(U[2 * t]);
            muv.push_back(U[2 * t + 1]);
        }

    // ---------------- topology update: k takes i's slot, j dies
    for (int32_t f : S_) falive_[f] = 0;
    for (int32_t f : Fa_)
        for (int c = 0; c < 3; c++)
            if (fv_[3 * f + c] == j) fv_[3 * f + c] = i;
    for (int32_t r : ring_) {
        auto& L = vf_[r];
        L.erase(std::remove_if(L.begin(), L.end(), [&](int32_t f) { return !falive_[f]; }), L.end());
    }
    vf_[i] = Fa_;
    std::sort(vf_[i].begin(), vf_[i].end());
    vf_[j].clear();
    valive_[j] = 0;
    vbnd_[i] = (char)(vbnd_[i] | vbnd_[j]);
    pos_[3 * i] = pk.x;
    pos_[3 * i + 1] = pk.y;
    pos_[3 * i + 2] = pk.z;
    alive_count_--;

    // UV corners and doubled area of every new face, once per collapse
    std::vector<double>& fuv = fuv_;
    fuv.resize(7 * Fa_.size());
    for (size_t a = 0; a < Fa_.size(); a++) {
        const int32_t f = Fa_[a];
        int t0 = var_after(fv_[3 * f]), t1 = var_after(fv_[3 * f + 1]), t2 = var_after(fv_[3 * f + 2]);
        double* g = &fuv[7 * a];
        g[0] = U[2 * t0]; g[1] = U[2 * t0 + 1]; g[2] = U[2 * t1]; g[3] = U[2 * t1 + 1];
        g[4] = U[2 * t2]; g[5] = U[2 * t2 + 1];
        g[6] = cross2(g[2] - g[0], g[3] - g[1], g[4] - g[0], g[5] - g[1]);
    }
    for (size_t q = 0; q < moving.size(); q++) {
        double x = muv[2 * q], y = muv[2 * q + 1];
        int32_t best_f = -1;
        double best_min = -1e300, bb[3] = {0, 0, 0};
        for (size_t a = 0; a < Fa_.size(); a++) {
            const int32_t f = Fa_[a];
            const double* g = &fuv[7 * a];
            double x0 = g[0], y0 = g[1], x1 = g[2], y1 = g[3], x2 = g[4], y2 = g[5];
            double dbl = g[6];
            double b0 = cross2(x1 - x, y1 - y, x2 - x, y2 - y) / dbl;
            double b1 = cross2(x2 - x, y2 - y, x0 - x, y0 - y) / dbl;
            double b2 = cross2(x0 - x, y0 - y, x1 - x, y1 - y) / dbl;
            double mn = std::min(b0, std::min(b1, b2));
            if (mn > best_min) {
                best_min = mn;
                best_f = f;
                bb[0] = b0; bb[1] = b1; bb[2] = b2;
            }
        }
        if (best_min < 0) {
            if (best_min < -1e-10) st.clamped++;
            st.worst_negative = std::min(st.worst_negative, best_min);
        }
        // a point within 1e-12 of an edge is taken to lie on it: negative or tiny
        // barycentrics become zero and the rest are renormalised
        double s = 0;
        for (int c = 0; c < 3; c++) {
            if (bb[c] < 1e-12) bb[c] = 0;
            s += bb[c];
        }
        int32_t p = moving[q];
        for (int c = 0; c < 3; c++) pbary_[3 * p + c] = bb[c] / s;
        pface_[p] = best_f;
        fpts_[best_f].push_back(p);
    }
    for (int32_t r : ring_) var_of_[r] = -1;

    // ---------------- new heap entries: only k moved, so only its edges change
    // length; rejected edges around the patch get another chance
    rej_[i].clear();
    rej_[j].clear();
    push_vertex_edges(i);
    for (int32_t r : ring_) {
        for (int32_t w : rej_[r])
            if (valive_[w] && w != i) push_edge(r, w);
        rej_[r].clear();
    }
    st.collapses++;
    return true;
}

int Decimator::run(int64_t target, MeshData& coarse, ProlongationRaw& Pout, DecimationStats& st,
                   std::string& err) {
    st_ = &st;
    {
        std::vector<HeapItem> init;
        init.reserve(3 * m_ / 2 + 16);
        for (int64_t f = 0; f < m_; f++)
            for (int c = 0; c < 3; c++) {
                int32_t a = fv_[3 * f + c], b = fv_[3 * f + (c + 1) % 3];
                if (a < b || vbnd_[a] || vbnd_[b]) {
                    int32_t lo = std::min(a, b), hi = std::max(a, b);
                    V3 d = v3sub(P(lo), P(hi));
                    init.push_back({v3dot(d, d), lo, hi});
                }
            }
        heap_.assign(std::move(init));
    }
    while (alive_count_ > target && !heap_.empty()) {
        HeapItem e = heap_.top();
        heap_.pop();
        if (!valive_[e.a] || !valive_[e.b]) continue;
        // only a collapse's new vertex moves, so an entry whose length no longer
        // matches is stale (its current length has its own entry)
        V3 d = v3sub(P(e.a), P(e.b));
        if (v3dot(d, d) != e.len2) continue;
        if (!try_collapse(e.a, e.b)) {
            rej_[e.a].push_back(e.b);
            rej_[e.b].push_back(e.a);
        }
    }
    // ---------------- coarse mesh and P_{l+1}
    std::vector<int32_t> newid(n_, -1);
    int64_t nc = 0;
    for (int64_t v = 0; v < n_; v++)
        if (valive_[v]) newid[v] = (int32_t)nc++;
    coarse.V.assign(3 * nc, 0.0);
    for (int64_t v = 0; v < n_; v++)
        if (valive_[v])
            for (int c = 0; c < 3; c++) coarse.V[3 * newid[v] + c] = pos_[3 * v + c];
    coarse.F.clear();
    for (int64_t f = 0; f < m_; f++)
        if (falive_[f])
            for (int c = 0; c < 3; c++) coarse.F.push_back(newid[fv_[3 * f + c]]);
    Pout.n_fine = n_;
    Pout.n_coarse = nc;
    Pout.idx.assign(3 * n_, -1);
    Pout.w.assign(3 * n_, 0.0);
    for (int64_t p = 0; p < n_; p++) {
        if (pface_[p] < 0) {
            if (!valive_[p]) {
                err = "internal: a collapsed vertex was not relocated";
                return 1;
            }
            Pout.idx[3 * p] = newid[p];
            Pout.w[3 * p] = 1.0;
            continue;
        }
        int32_t f = pface_[p];
        if (!falive_[f]) {
            err = "internal: a point sits in a removed face";
            return 1;
        }
        int k = 0;
        for (int c = 0; c < 3; c++) {
            double w = pbary_[3 * p + c];
            if (w > 0) {
                Pout.idx[3 * p + k] = newid[fv_[3 * f + c]];
                Pout.w[3 * p + k] = w;
                k++;
            }
        }
    }
    (void)err;
    return 0;
}

}  // namespace

int decimate_level(const MeshData& fine, int64_t target, MeshData& coarse, ProlongationRaw& P,
                   DecimationStats& st, std::string& err) {
    if (fine.n() < 4 || fine.m() < 1) {
        err = "mesh too small to decimate";
        return 1;
    }
    Decimator d(fine);
    return d.run(target, coarse, P, st, err);
}

int32_t greedy_colouring(int64_t n, const std::vector<int64_t>& rowptr, const std::vector<int32_t>& col,
                         std::vector<int32_t>& colour) {
    std::vector<int64_t> deg(n);
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; v++) {
        int64_t d = 0;
        for (int64_t p = rowptr[v]; p < rowptr[v + 1]; p++) d += (col[p] != v);
        deg[v] = d;
        maxdeg = std::max(maxdeg, d);
    }
    // descending degree, ascending index within a degree (bucketed, stable)
    std::vector<int64_t> start(maxdeg + 2, 0), order(n);
    for (int64_t v = 0; v < n; v++) start[maxdeg - deg[v] + 1]++;
    for (int64_t d = 1; d <= maxdeg + 1; d++) start[d] += start[d - 1];
    for (int64_t v = 0; v < n; v++) order[start[maxdeg - deg[v]]++] = v;

    colour.assign(n, -1);
    std::vector<int32_t> palette;
    std::vector<int64_t> stamp;
    for (int64_t v : order) {
        for (int64_t p = rowptr[v]; p < rowptr[v + 1]; p++) {
            int32_t u = col[p];
            if (u != v && colour[u] >= 0) stamp[colour[u]] = v;
        }
        int64_t pos = -1;
        for (size_t q = 0; q < palette.size(); q++)
            if (stamp[palette[q]] != v) {
                pos = (int64_t)q;
                break;
            }
        int32_t c;
        if (pos < 0) {
            c = (int32_t)palette.size();
            palette.push_back(c);
            stamp.push_back(-1);
        } else {
            c = palette[pos];
            palette.erase(palette.begin() + pos);
            palette.push_back(c);
        }
        colour[v] = c;
    }
    return (int32_t)palette.size();
}

}  // namespace smg
