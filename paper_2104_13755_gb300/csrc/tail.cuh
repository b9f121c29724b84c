// Cluster tail of the V-cycle: the levels below a tuned size run inside one
// thread-block cluster (16 CTAs, one per SM; 8 where 16 cannot be scheduled),
// one launch for the whole down-sweep (pre-relaxation, residual, restriction of
// every tail level) and one for the up-sweep (prolongation with correction,
// post-relaxation).  The arithmetic per row is that of the full-GPU kernels
// (Alg. 2 with the multicolour Gauss-Seidel of App. "Multi-Color Gauss Seidel").
//
// Every CTA keeps a full replica of each tail level's iterate x in its shared
// memory, so the gathers of a colour step are local shared-memory loads; a
// row's new value is written into all replicas with st.async (spread over the
// row's lanes) and counted on the receivers' step mbarriers.  Remote
// shared-memory loads have a small fraction of the throughput of local ones,
// which is why x is replicated rather than distributed.  The right-hand side b
// and the residual r are distributed: row i belongs to CTA (i / 32) mod CS at
// local slot (i / (32 CS)) * 32 + i mod 32.  The work of a colour step is split
// into warp-sized units (a slice's rows in groups of 32 / R, R lanes per row)
// dealt round-robin over all CTAs, because binary64 issue, not memory, bounds a
// step here.  Each warp loads the matrix entries, diagonal and right-hand side
// of its next step before waiting for the current one; where they fit, a CTA's
// units are staged in shared memory at kernel entry.  Global copies of x and b
// are read at entry and written at exit (the coarsest solve and the full-GPU
// levels run between the two launches).
#pragma once

#include "kernels.cuh"

namespace smg {

// Device view of one level for the tail kernels (one precision).
//
// The host deals each colour's work units (slice, row group g) round-robin over
// the CTAs and writes, per CTA, a table of its units, which the kernels copy to
// shared memory at entry:
//   [n_my, E] [cfirst: ncolours + 1] [rows: ncolours] [n_my x {off, W, row0, nrows, soff, g}]
// (cfirst[c] = index of the CTA's first unit of colour c, rows[c] = values a
// step of colour c delivers to every replica: the colour's rows plus one token
// from each CTA without a unit in it, off = the slice's SELL offset, row0 / nrows = the
// unit's rows, E = sum W * 32 / R, soff = the unit's first entry in the staged
// copy).  When the level is staged, the CTA also copies its units' column
// indices, values, reciprocal diagonal and diagonal to shared memory, so a
// colour step touches global memory not at all.
template <typename T>
struct TailLevel {
    const SliceMeta* slices;
    const int32_t* col;
    const T* sval;
    const T* dinv;
    const T* diag;
    const int32_t* colour_row;    // ncolours + 1 row offsets
    const int32_t* table;         // per-CTA slice tables, concatenated
    const int32_t* table_off;     // CS + 1 offsets into table
    T* x;                         // global copies (entry and exit)
    T* b;
    int nslices, ncolours, n;
    int rlg;                      // log2 of the lanes per row R (kTailPre entries per lane cover the longest row)
    int nloc;                     // distributed slots per CTA (multiple of 32)
    int npad;                     // replica slots of x (n rounded up to 32)
    int nwork;                    // slots of the local copy of b for this CTA's rows (32 per unit, max over CTAs)
    int sbase;                    // first slot of this level's arrays: x replica at sbase, b at +npad, r at
                                  // +npad+nloc, local b at +npad+2 nloc
    int staged;                   // matrix entries copied to shared memory
    int rbase;                    // byte offset of this level's table (and staged entries) in shared memory
    int tbytes;                   // bytes reserved for the table (maximum over CTAs, multiple of 16)
    // restriction into level + 1
    const int32_t* pt_ptr;
    const int32_t* pt_row;
    const T* pt_w;
    int n_next;
    T* b_next;                    // global arrays of level + 1 (used when it is outside the tail)
    T* x_next;
    int* err;                     // set when a step barrier wait times out
    // prolongation from level + 1
    const int32_t* p_idx;
    const T* p_w;
};

// Byte layout of a staged copy of E entries over n_rows unit rows (value type T).
template <typename T>
struct StageLayout {
    int col, val, dinv, diag, bytes;
    __host__ __device__ StageLayout(int E, int n_rows) {  // n_rows = units x rows per unit
        col = 0;
        val = ((E * 4 + 15) / 16) * 16;
        dinv = val + ((E * (int)sizeof(T) + 15) / 16) * 16;
        diag = dinv + ((n_rows * (int)sizeof(T) + 15) / 16) * 16;
        bytes = diag + ((n_rows * (int)sizeof(T) + 15) / 16) * 16;
    }
};

namespace kern {

// Threads per CTA: binary64 steps are bound by FP64 issue, and eight warps
// cover a colour's units at the tail sizes; binary32 steps are latency-bound
// and use more, narrower units.
template <typename T>
struct TailThreads {
    static constexpr int value = sizeof(T) == 8 ? 256 : 512;
    static constexpr int warps = value / 32;
};
constexpr int kTailPre = 8;  // entries per lane held in registers

// Cluster barrier with release / acquire ordering at cluster scope (the
// non-.aligned form: a warp may reach it after divergent loops).  Separates
// the phases other than the colour steps (copies, residual, restriction,
// prolongation), which use the step mbarriers below.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cta address -> shared::cluster address of the same offset in CTA `rank`
__device__ __forceinline__ uint32_t dsm(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ double ldc(uint32_t a, double*) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float ldc(uint32_t a, float*) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void stc(uint32_t a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void stc(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
template <typename T>
__device__ __forceinline__ T ldc(uint32_t a) {
    return ldc(a, (T*)nullptr);
}

__device__ __forceinline__ unsigned char* tail_smem() {
    extern __shared__ __align__(16) unsigned char tail_dyn_smem[];
    return tail_dyn_smem;
}

__device__ __forceinline__ double lds(uint32_t a, double*) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds(uint32_t a, float*) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
template <typename T>
__device__ __forceinline__ T lds(uint32_t a) {
    return lds(a, (T*)nullptr);
}
__device__ __forceinline__ void sts(uint32_t a, double v) {
    asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void sts(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

__device__ __forceinline__ int lds_i(uint32_t a) {
    int v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_i(uint32_t a, int v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Asynchronous global -> shared copies (4, 8 or 16 bytes, both addresses
// aligned to the size), all in flight together until cp_async_wait_all().
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, int bytes) {
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Rows over the CS = 1 << lg CTAs of the cluster (distributed arrays) and the
// local replicas.
struct Dist {
    uint32_t base;  // shared::cta address of the per-level arrays
    int lg;
    uint32_t rank;
    __device__ __forceinline__ uint32_t owner(int i) const { return (uint32_t)(i >> 5) & ((1u << lg) - 1u); }
    __device__ __forceinline__ int local(int i) const { return ((i >> (5 + lg)) << 5) | (i & 31); }
    __device__ __forceinline__ int global(int li) const {
        return ((li >> 5) << (5 + lg)) | (int)(rank << 5) | (li & 31);
    }
    // cluster address of value 0 of distributed row i in the array at slot offset arr
    template <typename T, int K>
    __device__ __forceinline__ uint32_t at(int arr, int i) const {
        return dsm(base + (uint32_t)(((arr + local(i)) * K) * (int)sizeof(T)), owner(i));
    }
    // this CTA's own slot li of distributed array arr (cluster address)
    template <typename T, int K>
    __device__ __forceinline__ uint32_t own(int arr, int li) const {
        return dsm(base + (uint32_t)(((arr + li) * K) * (int)sizeof(T)), rank);
    }
    // shared::cta address of value 0 of row i in the local replica at slot offset arr
    template <typename T, int K>
    __device__ __forceinline__ uint32_t rep(int arr, int i) const {
        return base + (uint32_t)(((arr + i) * K) * (int)sizeof(T));
    }
};

// This CTA's view of one tail level: its slice table (and staged entries) in
// shared memory, by shared::cta address.
template <typename T>
struct LevelCtx {
    const TailLevel<T>* L;
    // the level's global arrays, read once at staging so that no per-step load
    // goes through the level record in global memory first
    const int32_t* gcol;
    const T *gval, *gdinv, *gdiag;
    uint32_t tab;  // [n_my, E, cfirst[nc + 1], rows[nc], 6 * n_my]
    int n_my, nc, rlg, staged;
    uint32_t scol, sval, sdinv, sdiag;
    uint32_t bw;  // local copy of b (32 / R rows per unit)
    uint32_t xr;  // this CTA's replica of x (shared::cta address of row 0)
    __device__ __forceinline__ int cfirst(int c) const { return lds_i(tab + 4u * (2 + c)); }
    __device__ __forceinline__ int rows(int c) const { return lds_i(tab + 4u * (3 + nc + c)); }
    // field f of work unit i: 0 SELL offset of its slice, 1 W, 2 first row, 3 rows, 4 staged offset,
    // 5 row group g within the slice (rows g * 32 / R ...)
    __device__ __forceinline__ int unit(int i, int f) const { return lds_i(tab + 4u * (3 + 2 * nc + 6 * i + f)); }
};

// mbarrier helpers (shared::cta addresses; mbar_init is in kernels.cuh).
// A value into shared::cluster address a, counted on the mbarrier at cluster
// address bar (in the CTA that owns a) as sizeof(value) completed bytes.
__device__ __forceinline__ void st_async(uint32_t a, double v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(a), "d"(v), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async(uint32_t a, float v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(a), "f"(v), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_local(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cluster.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// Wait for phase `parity` with acquire at cluster scope, at most 2^22 polls; a
// thread whose wait ran out sets *err and does not wait again (gave_up).
__device__ __forceinline__ void mbar_wait_cluster(uint32_t bar, uint32_t parity, int* err, bool& gave_up) {
    if (gave_up) return;
    for (int it = 0; it < (1 << 22); it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return;
    }
    gave_up = true;
    atomicExch(err, 1);
}

// Step barriers of the relaxation: two mbarriers (even and odd steps) per CTA,
// each with one arrival (the CTA's own, announcing the step's byte count) and
// completing when the step's values have landed in this CTA: every row of the
// colour (into the replica of x) and one token from each CTA without a unit
// in the colour.  Every CTA thus sends something in every step, and only after
// its wait for the step before, so no CTA can reach step k + 2 (whose values
// count on the same barrier as step k) before every CTA has passed step k:
// two barriers suffice.
struct StepBars {
    uint32_t bar0;  // shared::cta address of the even-step mbarrier (the odd one follows)
    uint32_t step;  // steps taken so far in this launch
    bool gave_up;   // a wait of this thread ran out
    __device__ __forceinline__ uint32_t bar() const { return bar0 + 8u * (step & 1u); }
    __device__ __forceinline__ uint32_t parity() const { return (step >> 1) & 1u; }
};

// Copy this CTA's slice table into shared memory, and its slices' matrix
// entries too when the level is staged (4-16 byte asynchronous copies, all in
// flight together); gather b of its slices' rows into the local copy.
// CTA-local, ends with __syncthreads.
template <typename T, int K>
__device__ __forceinline__ LevelCtx<T> stage_level(const TailLevel<T>* Lp, const Dist& D) {
    const TailLevel<T>& L = *Lp;
    const uint32_t sm = (uint32_t)__cvta_generic_to_shared(tail_smem()) + (uint32_t)L.rbase;
    const int t0 = L.table_off[D.rank], t1 = L.table_off[D.rank + 1];
    for (int e = threadIdx.x; e < t1 - t0; e += TailThreads<T>::value) cp_async(sm + 4u * e, L.table + t0 + e, 4);
    cp_async_wait_all();
    __syncthreads();
    LevelCtx<T> C;
    C.L = Lp;
    C.gcol = L.col;
    C.gval = L.sval;
    C.gdinv = L.dinv;
    C.gdiag = L.diag;
    C.tab = sm;
    C.n_my = lds_i(sm);
    const int E = lds_i(sm + 4u);
    C.nc = L.ncolours;
    C.rlg = L.rlg;
    C.staged = L.staged;
    const StageLayout<T> lay(E, C.n_my << (5 - C.rlg));
    const uint32_t st = sm + (uint32_t)L.tbytes;
    C.scol = st + lay.col;
    C.sval = st + lay.val;
    C.sdinv = st + lay.dinv;
    C.sdiag = st + lay.diag;
    C.bw = D.template rep<T, K>(L.sbase + L.npad + 2 * L.nloc, 0);
    C.xr = D.template rep<T, K>(L.sbase, 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rl_lg = 5 - C.rlg, RL = 1 << rl_lg;  // rows per unit
    if (C.staged) {
        // entries (k, rl) of a unit's rows, unit-major: staged index soff + k * RL + rl.  Per k the
        // unit's RL column indices and values are contiguous in the SELL arrays (and RL-aligned), so
        // they move as a few 4-16 byte asynchronous copies, all of the CTA's in flight together.
        const bool a16 = ((reinterpret_cast<uintptr_t>(L.col) | reinterpret_cast<uintptr_t>(L.sval)) & 15u) == 0;
        const int cb = RL * 4, cps = !a16 ? 4 : (cb < 16 ? cb : 16), cpn = cb / cps;
        const int vb = RL * (int)sizeof(T), vps = !a16 ? (int)sizeof(T) : (vb < 16 ? vb : 16), vpn = vb / vps;
        for (int i = warp; i < C.n_my; i += TailThreads<T>::warps) {
            const int off = C.unit(i, 0), W = C.unit(i, 1), soff = C.unit(i, 4), g = C.unit(i, 5);
            for (int k = lane; k < W; k += 32) {  // one k of the unit per lane: its RL indices and values
                const int src = off + k * 32 + g * RL, dst = soff + k * RL;
                const char* sc = (const char*)(L.col + src);
                const char* sv = (const char*)(L.sval + src);
                const uint32_t dc = C.scol + 4u * dst, dv = C.sval + (uint32_t)sizeof(T) * dst;
                for (int p = 0; p < cpn; p++) cp_async(dc + (uint32_t)(p * cps), sc + p * cps, cps);
                for (int p = 0; p < vpn; p++) cp_async(dv + (uint32_t)(p * vps), sv + p * vps, vps);
            }
        }
    }
    // per unit row: reciprocal diagonal and diagonal (staged), b from the distributed array;
    // one thread per row so the remote loads are all in flight together
    for (int t = threadIdx.x; t < (C.n_my << rl_lg); t += TailThreads<T>::value) {
        const int i = t >> rl_lg, r = t & (RL - 1);
        if (r >= C.unit(i, 3)) continue;
        const int row = C.unit(i, 2) + r;
        if (C.staged) {
            cp_async(C.sdinv + (uint32_t)sizeof(T) * t, L.dinv + row, (int)sizeof(T));
            cp_async(C.sdiag + (uint32_t)sizeof(T) * t, L.diag + row, (int)sizeof(T));
        }
        const uint32_t src = D.template at<T, K>(L.sbase + L.npad, row);
        T bv[K];
#pragma unroll
        for (int q = 0; q < K; q++) bv[q] = ldc<T>(src + q * (int)sizeof(T));
#pragma unroll
        for (int q = 0; q < K; q++) sts(C.bw + (uint32_t)((t * K + q) * (int)sizeof(T)), bv[q]);
    }
    cp_async_wait_all();
    __syncthreads();
    return C;
}

// One warp's share of a SELL-32 slice (R = 2^rlg lanes per row, 32 / R rows per
// warp), loaded ahead of the barrier that precedes its use.
template <typename T, int K>
struct TailRows {
    static constexpr int PRE = kTailPre;
    int cx[PRE];       // column of each entry (its x replica address is formed where x is read, so the
                       // column loads of an unstaged level stay in flight across the step barrier)
    T v[PRE];
    T bb[K];
    T d;
    uint32_t xrow;     // local replica address of this row's x (GS: offset for the broadcast)
    uint32_t rself;    // cluster address of this row's r (residual)
    int base;     // entry (k, r) of the unit is at base + k * rstride + r: staged (shared) or SELL (global)
    int rstride;  // rows per unit when staged, 32 in the SELL arrays
    int W, r, sub, rlg;
    bool live, valid, staged;

    __device__ __forceinline__ int col_at(const LevelCtx<T>& C, int k) const {
        const int e = base + k * rstride + r;
        return staged ? lds_i(C.scol + 4u * e) : __ldg(C.gcol + e);
    }
    __device__ __forceinline__ T val_at(const LevelCtx<T>& C, int k) const {
        const int e = base + k * rstride + r;
        return staged ? lds<T>(C.sval + (uint32_t)sizeof(T) * e) : __ldg(C.gval + e);
    }

    // work unit i (or none when i < 0); RESIDUAL: diagonal, else its reciprocal.
    // Lane = sub * RL + r: entries k = sub, sub + R, ... of the unit's row r.
    template <bool RESIDUAL>
    __device__ __forceinline__ void load(const LevelCtx<T>& C, const Dist& D, int i, int lane) {
        live = i >= 0;
        if (!live) return;
        const TailLevel<T>& L = *C.L;
        staged = C.staged != 0;
        rlg = C.rlg;
        const int rl_lg = 5 - rlg;  // log2 rows per unit
        W = C.unit(i, 1);
        const int row0 = C.unit(i, 2), nrows = C.unit(i, 3);
        sub = lane >> rl_lg;
        r = lane & ((1 << rl_lg) - 1);
        base = staged ? C.unit(i, 4) : C.unit(i, 0) + (C.unit(i, 5) << rl_lg);
        rstride = staged ? (1 << rl_lg) : 32;
        valid = r < nrows;
        const int row = row0 + (valid ? r : 0);
#pragma unroll
        for (int u = 0; u < PRE; u++) {
            const int k = sub + (u << rlg);
            if (k < W) {
                cx[u] = col_at(C, k);
                v[u] = val_at(C, k);
            }
        }
        if (staged) d = lds<T>((RESIDUAL ? C.sdiag : C.sdinv) + (uint32_t)sizeof(T) * ((i << rl_lg) + r));
        else d = RESIDUAL ? C.gdiag[row] : C.gdinv[row];
        const uint32_t ba = C.bw + (uint32_t)((((i << rl_lg) + r) * K) * (int)sizeof(T));
#pragma unroll
        for (int q = 0; q < K; q++) bb[q] = lds<T>(ba + q * (int)sizeof(T));
        xrow = C.xr + (uint32_t)(row * K * (int)sizeof(T));
        if (RESIDUAL) rself = D.template at<T, K>(L.sbase + L.npad + L.nloc, row);
    }

    // GS: x_row <- (b_row - sum a x) / a_rr into every replica; residual:
    // r_row <- b_row - a_rr x_row - sum a x at the owner
    template <bool RESIDUAL>
    __device__ __forceinline__ void run(const LevelCtx<T>& C, const Dist& D, uint32_t sbar = 0) const {
        if (!live) return;  // uniform over the warp
        T xv[PRE][K];
#pragma unroll
        for (int u = 0; u < PRE; u++)
            if (sub + (u << rlg) < W)
#pragma unroll
                for (int q = 0; q < K; q++) xv[u][q] = lds<T>(C.xr + (uint32_t)((cx[u] * K + q) * (int)sizeof(T)));
        // one chain per lane: every binary64 instruction holds the warp for the
        // same time whether or not it depends on the previous one, so fewer
        // instructions, not shorter chains, shorten a step; the row's first lane
        // starts from b (Gauss-Seidel) or b - a_rr x_r (residual)
        T a0[K];
#pragma unroll
        for (int q = 0; q < K; q++) {
            a0[q] = T(0);
            if (sub == 0) a0[q] = RESIDUAL ? bb[q] - d * lds<T>(xrow + q * (int)sizeof(T)) : bb[q];
        }
#pragma unroll
        for (int u = 0; u < PRE; u++)
            if (sub + (u << rlg) < W)
#pragma unroll
                for (int q = 0; q < K; q++) a0[q] -= v[u] * xv[u][q];
        for (int k = sub + (PRE << rlg); k < W; k += 1 << rlg) {  // rows longer than PRE * R
            const int c = col_at(C, k);
            const T vv = val_at(C, k);
            const uint32_t a = C.xr + (uint32_t)(c * K * (int)sizeof(T));
#pragma unroll
            for (int q = 0; q < K; q++) a0[q] -= vv * lds<T>(a + q * (int)sizeof(T));
        }
        T acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = a0[q];
        for (int o = 16; o >= (32 >> rlg); o >>= 1)  // every lane of the row ends with the sum
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        if (!valid) return;
        if (RESIDUAL) {
            if (sub == 0)
#pragma unroll
                for (int q = 0; q < K; q++)
                    stc(rself + q * (int)sizeof(T), acc[q]);
        } else {
            T out[K];
#pragma unroll
            for (int q = 0; q < K; q++) out[q] = acc[q] * d;  // (b - sum a x) / a_rr
            const int cs = 1 << D.lg;
            for (int j = sub; j < cs; j += 1 << rlg) {  // the row's lanes share the CS replica writes
                const uint32_t a = dsm(xrow, (uint32_t)j);
                const uint32_t bj = dsm(sbar, (uint32_t)j);
#pragma unroll
                for (int q = 0; q < K; q++) st_async(a + q * (int)sizeof(T), out[q], bj);
            }
        }
    }
};

// Landing slot of the tokens (same offset in every CTA; never read).
__shared__ __align__(8) double tail_token[4];

// Gauss-Seidel over the colour sequence of `steps` steps (colour of step k from
// col_of(k)).  New values go to every replica by st.async, counted on the
// receivers' step barriers (a CTA without a unit in the colour sends its
// token instead); each CTA then arrives on its own barrier with the step's
// byte count, loads its next step's entries and waits.  The loop ends with a
// cluster barrier, so no store of the relaxation is in flight afterwards.
template <typename T, int K, class ColourOf>
__device__ __forceinline__ void tail_relax(const LevelCtx<T>& C, const Dist& D, int steps, ColourOf col_of,
                                           int warp, int lane, StepBars& sb) {
    // Binary64 with one right-hand side: the warp's first two units of a step
    // are both loaded before the preceding barrier (a colour class of a level
    // above the staged sizes has up to ~2 units per warp at 8 warps per CTA);
    // further units are loaded in the step.
    constexpr bool TWO = sizeof(T) == 8 && K == 1;
    constexpr int NW = TailThreads<T>::warps;
    TailRows<T, K> cur, nxt;
    const uint32_t tok = (uint32_t)__cvta_generic_to_shared(tail_token);
    auto load = [&](TailRows<T, K>& t, int c, int u) {
        const int i = C.cfirst(c) + u;
        t.template load<false>(C, D, i < C.cfirst(c + 1) ? i : -1, lane);
    };
    auto load_step = [&](int c) {
        load(cur, c, warp);
        if (TWO) load(nxt, c, warp + NW);
    };
    if (steps > 0) load_step(col_of(0));
    for (int k = 0; k < steps; k++) {
        const int c = col_of(k);
        const int units = C.cfirst(c + 1) - C.cfirst(c);
        const uint32_t bar = sb.bar();
        cur.template run<false>(C, D, bar);
        if (TWO) nxt.template run<false>(C, D, bar);
        for (int u = warp + (TWO ? 2 : 1) * NW; u < units; u += NW) {
            load(cur, c, u);
            cur.template run<false>(C, D, bar);
        }
        if (warp == 0) {
            if (units == 0 && lane < (1 << D.lg))  // no unit in this colour: a token to every CTA
#pragma unroll
                for (int q = 0; q < K; q++)
                    st_async(dsm(tok + q * (uint32_t)sizeof(T), (uint32_t)lane), T(0), dsm(bar, (uint32_t)lane));
            if (lane == 0) mbar_arrive_expect_local(bar, (uint32_t)C.rows(c) * (uint32_t)(K * sizeof(T)));
        }
        if (k + 1 < steps) load_step(col_of(k + 1));
        mbar_wait_cluster(bar, sb.parity(), C.L->err, sb.gave_up);
        sb.step++;
    }
    cluster_sync();
}

// r = b - A x over all rows (this CTA's units of every colour).  With the
// entries staged, one thread per row: no colour order to respect here, and a
// lane that walks its row needs one binary64 instruction per entry instead of
// the entries over R lanes plus the log R reduction steps, so the step, which
// binary64 issue bounds, takes about half the instructions.
template <typename T, int K>
__device__ __forceinline__ void tail_residual(const LevelCtx<T>& C, const Dist& D, int warp, int lane) {
    if (C.staged) {
        const TailLevel<T>& L = *C.L;
        const int rl_lg = 5 - C.rlg, RL = 1 << rl_lg;
        for (int t = threadIdx.x; t < (C.n_my << rl_lg); t += TailThreads<T>::value) {
            const int i = t >> rl_lg, r = t & (RL - 1);
            if (r >= C.unit(i, 3)) continue;
            const int W = C.unit(i, 1), soff = C.unit(i, 4), row = C.unit(i, 2) + r;
            const T d = lds<T>(C.sdiag + (uint32_t)sizeof(T) * t);
            const uint32_t xrow = C.xr + (uint32_t)(row * K * (int)sizeof(T));
            T acc[K];
#pragma unroll
            for (int q = 0; q < K; q++)
                acc[q] = lds<T>(C.bw + (uint32_t)((t * K + q) * (int)sizeof(T))) - d * lds<T>(xrow + q * (int)sizeof(T));
#pragma unroll 4
            for (int k = 0; k < W; k++) {
                const int e = soff + k * RL + r;
                const uint32_t xa = C.xr + (uint32_t)(lds_i(C.scol + 4u * e) * K * (int)sizeof(T));
                const T v = lds<T>(C.sval + (uint32_t)sizeof(T) * e);
#pragma unroll
                for (int q = 0; q < K; q++) acc[q] -= v * lds<T>(xa + q * (int)sizeof(T));
            }
            const uint32_t rs = D.template at<T, K>(L.sbase + L.npad + L.nloc, row);
#pragma unroll
            for (int q = 0; q < K; q++) stc(rs + q * (int)sizeof(T), acc[q]);
        }
        return;
    }
    TailRows<T, K> cur;
    for (int u = warp; u < C.n_my; u += TailThreads<T>::warps) {
        cur.template load<true>(C, D, u, lane);
        cur.template run<true>(C, D);
    }
}

// b_{l+1} = P^T r_l for the coarse rows this CTA owns (four lanes per row);
// into distributed memory when level l+1 is in the tail (Ln != nullptr), with
// this CTA's replica of x_{l+1} set to the zero start, else into level l+1's
// global arrays (b and the zero x of the rows this CTA owns).
template <typename T, int K>
__device__ __forceinline__ void tail_restrict(const TailLevel<T>& L, const TailLevel<T>* Ln, const Dist& D) {
    constexpr int RR = 4;
    const int sub = threadIdx.x % RR;
    constexpr int per_pass = TailThreads<T>::value / RR;
    const int nloc_next = ((L.n_next + (32 << D.lg) - 1) >> (5 + D.lg)) << 5;
    const int passes = (nloc_next + per_pass - 1) / per_pass;
    const int sr = L.sbase + L.npad + L.nloc;
    for (int pass = 0; pass < passes; pass++) {
        const int li = pass * per_pass + (int)threadIdx.x / RR;
        const int I0 = D.global(li);
        const bool ok = li < nloc_next && I0 < L.n_next;
        const int I = ok ? I0 : 0;
        T acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = T(0);
        const int k1 = ok ? L.pt_ptr[I + 1] : 0;
        for (int k = (ok ? L.pt_ptr[I] : 0) + sub; k < k1; k += RR) {
            const int i = L.pt_row[k];
            const T wk = L.pt_w[k];
            const uint32_t a = D.template at<T, K>(sr, i);
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += wk * ldc<T>(a + q * (int)sizeof(T));
        }
#pragma unroll
        for (int o = RR / 2; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        if (ok && sub == 0) {
            if (Ln) {
                const uint32_t ba = D.template own<T, K>(Ln->sbase + Ln->npad, li);
#pragma unroll
                for (int q = 0; q < K; q++) stc(ba + q * (int)sizeof(T), acc[q]);
            } else {
#pragma unroll
                for (int q = 0; q < K; q++) {
                    L.b_next[(int64_t)I * K + q] = acc[q];
                    L.x_next[(int64_t)I * K + q] = T(0);
                }
            }
        }
    }
    if (Ln)
        for (int e = threadIdx.x; e < Ln->n * K; e += TailThreads<T>::value) sts(D.template rep<T, 1>(Ln->sbase * K, e), T(0));
}

// x_l += P x_{l+1} for the rows of level l this CTA owns, written to level l's
// global x (the replicas are refreshed from it after the next barrier);
// x_{l+1} from the local replica (Ln != nullptr) or from global memory.
template <typename T, int K>
__device__ __forceinline__ void tail_prolong(const TailLevel<T>& L, const TailLevel<T>* Ln, const Dist& D) {
    for (int li = threadIdx.x; li < L.nloc; li += TailThreads<T>::value) {
        const int p = D.global(li);
        if (p >= L.n) continue;
        T acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = T(0);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int c = L.p_idx[(int64_t)a * L.n + p];
            const T wa = L.p_w[(int64_t)a * L.n + p];
            if (Ln) {
                const uint32_t ca = D.template rep<T, K>(Ln->sbase, c);
#pragma unroll
                for (int q = 0; q < K; q++) acc[q] += wa * lds<T>(ca + q * (int)sizeof(T));
            } else {
#pragma unroll
                for (int q = 0; q < K; q++) acc[q] += wa * L.x_next[(int64_t)c * K + q];
            }
        }
        const uint32_t xa = D.template rep<T, K>(L.sbase, p);
#pragma unroll
        for (int q = 0; q < K; q++) L.x[(int64_t)p * K + q] = lds<T>(xa + q * (int)sizeof(T)) + acc[q];
    }
}

// Global x of a level into this CTA's replica (all rows): 16-byte asynchronous
// copies where both sides are aligned, single values otherwise.  Completes
// before return (CTA-local; the caller's barrier publishes it).
template <typename T, int K>
__device__ __forceinline__ void tail_load_x(const TailLevel<T>& L, const Dist& D) {
    const uint32_t dst = D.template rep<T, 1>(L.sbase * K, 0);
    const int bytes = L.n * K * (int)sizeof(T);
    const bool aligned = ((reinterpret_cast<uintptr_t>(L.x) | dst) & 15u) == 0;
    const int chunks = aligned ? bytes / 16 : 0;
    for (int c = threadIdx.x; c < chunks; c += TailThreads<T>::value)
        cp_async(dst + 16u * c, (const char*)L.x + 16 * c, 16);
    for (int e = chunks * 16 / (int)sizeof(T) + threadIdx.x; e < L.n * K; e += TailThreads<T>::value)
        cp_async(dst + (uint32_t)(e * (int)sizeof(T)), L.x + e, (int)sizeof(T));
    cp_async_wait_all();
}

// This CTA's rows of b between global memory and the distributed array, and
// (TO_SHARED = false) its rows of x from the replica to global memory.
template <typename T, int K, bool TO_SHARED>
__device__ __forceinline__ void tail_copy_own(const TailLevel<T>& L, const Dist& D, bool with_b) {
    for (int e = threadIdx.x; e < L.nloc * K; e += TailThreads<T>::value) {
        const int li = e / K, q = e - li * K;
        const int i = D.global(li);
        if (i >= L.n) continue;
        const uint32_t ba = D.template own<T, K>(L.sbase + L.npad, li) + q * (int)sizeof(T);
        if (TO_SHARED) {
            stc(ba, L.b[(int64_t)i * K + q]);
        } else {
            L.x[(int64_t)i * K + q] = lds<T>(D.template rep<T, K>(L.sbase, i) + q * (int)sizeof(T));
            if (with_b) L.b[(int64_t)i * K + q] = ldc<T>(ba);
        }
    }
}

__device__ __forceinline__ Dist make_dist(int lg, int dbase) {
    Dist D;
    D.base = (uint32_t)__cvta_generic_to_shared(tail_smem()) + (uint32_t)dbase;
    D.lg = lg;
    D.rank = cluster_rank();
    return D;
}

// Down-sweep of levels [l0, l1): pre-relaxation, residual, restriction.  The
// per-level arrays start at byte dbase of the dynamic shared memory, after the
// slice tables and staged entries of the tail levels.
template <typename T, int K>
__global__ void __launch_bounds__(TailThreads<T>::value, 1) tail_down(const TailLevel<T>* __restrict__ lv, int l0, int l1,
                                                             int mu_pre, int lg, int dbase) {
    const Dist D = make_dist(lg, dbase);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ __align__(8) unsigned long long mbar[2];  // step barriers: even, odd steps
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
    StepBars sb{bar, 0u, false};
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 8u, 1);
    }
    pdl_wait();
    pdl_trigger();
    tail_load_x<T, K>(lv[l0], D);
    tail_copy_own<T, K, true>(lv[l0], D, true);
    cluster_sync();
    for (int l = l0; l < l1; l++) {
        const LevelCtx<T> C = stage_level<T, K>(&lv[l], D);
        const int nc = C.nc;
        tail_relax<T, K>(C, D, mu_pre * nc, [nc](int k) { return k % nc; }, warp, lane, sb);
        tail_residual<T, K>(C, D, warp, lane);
        cluster_sync();
        tail_restrict<T, K>(lv[l], l + 1 < l1 ? &lv[l + 1] : nullptr, D);
        cluster_sync();
    }
    for (int l = l0; l < l1; l++) tail_copy_own<T, K, false>(lv[l], D, true);
}

// Up-sweep of levels [l0, l1) from level l1 - 1 upwards: prolongation with the
// correction add, then post-relaxation (colour classes reversed if asked).
template <typename T, int K>
__global__ void __launch_bounds__(TailThreads<T>::value, 1) tail_up(const TailLevel<T>* __restrict__ lv, int l0, int l1,
                                                           int mu_post, int reverse, int lg, int dbase) {
    const Dist D = make_dist(lg, dbase);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ __align__(8) unsigned long long mbar[2];  // step barriers: even, odd steps
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
    StepBars sb{bar, 0u, false};
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 8u, 1);
    }
    pdl_wait();
    pdl_trigger();
    for (int l = l0; l < l1; l++) {
        tail_load_x<T, K>(lv[l], D);
        tail_copy_own<T, K, true>(lv[l], D, true);
    }
    __syncthreads();
    for (int l = l1 - 1; l >= l0; l--) {
        tail_prolong<T, K>(lv[l], l + 1 < l1 ? &lv[l + 1] : nullptr, D);
        cluster_sync();  // level l's corrected x is in global memory
        tail_load_x<T, K>(lv[l], D);
        const LevelCtx<T> C = stage_level<T, K>(&lv[l], D);
        cluster_sync();  // every replica refreshed before any step writes into it
        const int nc = C.nc;
        tail_relax<T, K>(C, D, mu_post * nc, [nc, reverse](int k) { return reverse ? nc - 1 - k % nc : k % nc; },
                         warp, lane, sb);
    }
    tail_copy_own<T, K, false>(lv[l0], D, false);
}

}  // namespace kern
}  // namespace smg
