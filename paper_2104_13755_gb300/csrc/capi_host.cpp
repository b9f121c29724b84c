// Host half of the C ABI: options, status strings, plan build / queries / save / load.
#include <cstdio>
#include <cstring>
#include <new>

#include "plan.hpp"

namespace smg {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace smg

using namespace smg;

namespace {
// ---------------------------------------------------------------- save / load
const char kMagic[8] = {'S', 'M', 'G', 'P', 'L', 'A', 'N', '1'};
const int32_t kVersion = 6;  // 3: smg_options gained `solver`; 4: `smoother`, `jacobi_omega`; 5: `pattern_rings`; 6: `block_size`

template <class T>
bool wvec(FILE* f, const std::vector<T>& v) {
    int64_t k = (int64_t)v.size();
    return fwrite(&k, sizeof k, 1, f) == 1 && (k == 0 || fwrite(v.data(), sizeof(T), (size_t)k, f) == (size_t)k);
}
template <class T>
bool rvec(FILE* f, std::vector<T>& v) {
    int64_t k = 0;
    if (fread(&k, sizeof k, 1, f) != 1 || k < 0 || k > ((int64_t)1 << 36)) return false;
    v.resize((size_t)k);
    return k == 0 || fread(v.data(), sizeof(T), (size_t)k, f) == (size_t)k;
}

}  // namespace

extern "C" {

void smg_default_options(smg_options* o) {
    if (!o) return;
    o->mu_pre = 2;
    o->mu_post = 2;
    o->ratio = 0.25;
    o->min_coarse = 500;
    o->max_coarse = 0;
    o->max_levels = 0;
    o->max_cycles = 100;
    o->rtol = 1e-10;
    o->precision = SMG_FP64;
    o->post_reverse = 1;
    o->autotune = 1;
    o->solver = SMG_SOLVER_VCYCLE;
    o->smoother = SMG_SMOOTHER_GS;
    o->jacobi_omega = 2.0 / 3.0;
    o->pattern_rings = 1;
    o->block_size = 1;
}

const char* smg_status_string(int s) {
    switch (s) {
        case SMG_OK: return "ok";
        case SMG_ERR_INVALID_ARG: return "invalid argument";
        case SMG_ERR_NONMANIFOLD: return "mesh is not an oriented manifold";
        case SMG_ERR_DECIMATION: return "hierarchy construction failed";
        case SMG_ERR_NOT_SPD: return "coarsest operator not positive definite";
        case SMG_ERR_NOT_CONVERGED: return "not converged within max_cycles";
        case SMG_ERR_DIVERGED: return "residual became non-finite";
        case SMG_ERR_TIMEOUT: return "device wait timed out";
        case SMG_ERR_CUDA: return "CUDA error";
        case SMG_ERR_NO_MEMORY: return "out of memory";
        case SMG_ERR_STATE: return "call out of order";
        case SMG_ERR_IO: return "plan file error";
        default: return "unknown status";
    }
}

const char* smg_last_error(void) { return g_last_error.c_str(); }

int smg_plan_build(const double* V, int64_t n, const int32_t* F, int64_t m, const uint8_t* mask,
                   const smg_options* opts, smg_plan** out) {
    if (!out) {
        set_error("out is null");
        return SMG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    smg_options o;
    if (opts) o = *opts;
    else smg_default_options(&o);
    smg_plan* p = new (std::nothrow) smg_plan();
    if (!p) return SMG_ERR_NO_MEMORY;
    std::string err;
    int st;
    try {
        st = build_plan(V, n, F, m, mask, o, p->p, err);
    } catch (const std::bad_alloc&) {
        st = SMG_ERR_NO_MEMORY;
        err = "host allocation failed during setup";
    } catch (...) {
        st = SMG_ERR_DECIMATION;
        err = "unexpected exception during setup";
    }
    if (st != SMG_OK) {
        set_error(err);
        delete p;
        return st;
    }
    *out = p;
    return SMG_OK;
}

void smg_plan_destroy(smg_plan* p) { delete p; }

int smg_plan_num_levels(const smg_plan* p) { return p ? (int)p->p.L.size() : 0; }

static bool bad_level(const smg_plan* p, int level) {
    if (!p || level < 0 || level >= (int)p->p.L.size()) {
        set_error("invalid plan or level");
        return true;
    }
    return false;
}

int smg_plan_level_info(const smg_plan* p, int level, int64_t* n, int64_t* nnz, int32_t* ncol) {
    if (bad_level(p, level)) return SMG_ERR_INVALID_ARG;
    const LevelPlan& lv = p->p.L[level];
    if (n) *n = lv.n;
    if (nnz) *nnz = (int64_t)lv.col.size();
    if (ncol) *ncol = lv.ncolours;
    return SMG_OK;
}

int smg_plan_mesh(const smg_plan* p, int level, int64_t* n, int64_t* m, const double** V, const int32_t** F) {
    if (bad_level(p, level)) return SMG_ERR_INVALID_ARG;
    const MeshData& md = p->p.meshes[level];
    if (n) *n = md.n();
    if (m) *m = md.m();
    if (V) *V = md.V.data();
    if (F) *F = md.F.data();
    return SMG_OK;
}

int smg_plan_prolongation(const smg_plan* p, int level, int64_t* nf, int64_t* nc, const int32_t** idx,
                          const double** w) {
    if (bad_level(p, level) || level < 1) {
        set_error("prolongation level must be 1..H");
        return SMG_ERR_INVALID_ARG;
    }
    const ProlongationRaw& P = p->p.praw[level - 1];
    if (nf) *nf = P.n_fine;
    if (nc) *nc = P.n_coarse;
    if (idx) *idx = P.idx.data();
    if (w) *w = P.w.data();
    return SMG_OK;
}

int smg_plan_pattern(const smg_plan* p, int level, const int64_t** rowptr, const int32_t** col) {
    if (bad_level(p, level)) return SMG_ERR_INVALID_ARG;
    if (rowptr) *rowptr = p->p.L[level].rowptr.data();
    if (col) *col = p->p.L[level].col.data();
    return SMG_OK;
}

int smg_plan_colouring(const smg_plan* p, int level, const int32_t** colour) {
    if (bad_level(p, level)) return SMG_ERR_INVALID_ARG;
    if (p->p.L[level].coarsest) {
        set_error("the coarsest level is not coloured");
        return SMG_ERR_INVALID_ARG;
    }
    if (colour) *colour = p->p.L[level].colour.data();
    return SMG_OK;
}

int smg_plan_unknowns(const smg_plan* p, int64_t* nu, const int32_t** v) {
    if (!p) return SMG_ERR_INVALID_ARG;
    if (nu) *nu = (int64_t)p->p.unknowns.size();
    if (v) *v = p->p.unknowns.data();
    return SMG_OK;
}

int smg_plan_kept_coarse(const smg_plan* p, int64_t* nk, const int32_t** kept) {
    if (!p) return SMG_ERR_INVALID_ARG;
    if (nk) *nk = (int64_t)p->p.kept1.size();
    if (kept) *kept = p->p.kept1.data();
    return SMG_OK;
}

int smg_plan_stats(const smg_plan* p, int level, int64_t out[9]) {
    if (!p || level < 0 || level >= (int)p->p.stats.size() || !out) {
        set_error("stats level must be 0..H-1");
        return SMG_ERR_INVALID_ARG;
    }
    const DecimationStats& s = p->p.stats[level];
    out[0] = s.collapses;
    out[1] = s.rejected_link;
    out[2] = s.rejected_boundary;
    out[3] = s.rejected_flip;
    out[4] = s.rejected_angle;
    out[5] = s.rejected_quality;
    out[6] = s.rejected_solve;
    out[7] = s.clamped;
    out[8] = (int64_t)(s.worst_negative * 1e15);
    return SMG_OK;
}

int smg_plan_save(const smg_plan* p, const char* path) {
    if (!p || !path) return SMG_ERR_INVALID_ARG;
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error(std::string("cannot open ") + path);
        return SMG_ERR_IO;
    }
    const Plan& P = p->p;
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&kVersion, sizeof kVersion, 1, f) == 1 &&
              fwrite(&P.opts, sizeof P.opts, 1, f) == 1 && wvec(f, P.known);
    int32_t nl = (int32_t)P.meshes.size();
    ok = ok && fwrite(&nl, sizeof nl, 1, f) == 1;
    for (int32_t l = 0; ok && l < nl; l++) ok = wvec(f, P.meshes[l].V) && wvec(f, P.meshes[l].F);
    for (int32_t l = 0; ok && l + 1 < nl; l++) {
        const ProlongationRaw& R = P.praw[l];
        ok = fwrite(&R.n_fine, sizeof R.n_fine, 1, f) == 1 && fwrite(&R.n_coarse, sizeof R.n_coarse, 1, f) == 1 &&
             wvec(f, R.idx) && wvec(f, R.w) && fwrite(&P.stats[l], sizeof(DecimationStats), 1, f) == 1;
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error(std::string("write failed: ") + path);
        return SMG_ERR_IO;
    }
    return SMG_OK;
}

int smg_plan_load(const char* path, smg_plan** out) {
    if (!path || !out) return SMG_ERR_INVALID_ARG;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error(std::string("cannot open ") + path);
        return SMG_ERR_IO;
    }
    smg_plan* p = new (std::nothrow) smg_plan();
    if (!p) {
        fclose(f);
        return SMG_ERR_NO_MEMORY;
    }
    Plan& P = p->p;
    char magic[8];
    int32_t ver = 0, nl = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(&ver, sizeof ver, 1, f) == 1 &&
              ver == kVersion && fread(&P.opts, sizeof P.opts, 1, f) == 1 && rvec(f, P.known) &&
              fread(&nl, sizeof nl, 1, f) == 1 && nl >= 1 && nl < 64;
    if (ok) P.meshes.resize(nl);
    for (int32_t l = 0; ok && l < nl; l++) ok = rvec(f, P.meshes[l].V) && rvec(f, P.meshes[l].F);
    if (ok) {
        P.praw.resize(nl - 1);
        P.stats.resize(nl - 1);
    }
    for (int32_t l = 0; ok && l + 1 < nl; l++) {
        ProlongationRaw& R = P.praw[l];
        ok = fread(&R.n_fine, sizeof R.n_fine, 1, f) == 1 && fread(&R.n_coarse, sizeof R.n_coarse, 1, f) == 1 &&
             rvec(f, R.idx) && rvec(f, R.w) && fread(&P.stats[l], sizeof(DecimationStats), 1, f) == 1;
    }
    fclose(f);
    std::string err;
    if (ok && (int64_t)P.known.size() != P.meshes[0].n()) ok = false;
    if (!ok) {
        set_error(std::string("corrupt or incompatible plan file: ") + path);
        delete p;
        return SMG_ERR_IO;
    }
    int st;
    try {
        st = finalize_plan(P, err);
    } catch (...) {
        st = SMG_ERR_NO_MEMORY;
        err = "allocation failed while loading";
    }
    if (st != SMG_OK) {
        set_error(err);
        delete p;
        return st;
    }
    *out = p;
    return SMG_OK;
}

}  // extern "C"
