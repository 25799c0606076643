// The Chief (arXiv 1806.04211, Section 3, Algorithm "The Chief") as a host
// planner driving the job kernels, and the recursive single-block
// echelonisation ECH built on it (Section 2.3.2).
//
// Step 1: Tasks ClearDown, Extend, UpdateRow and UpdateRowTrafo (Section 4.2)
// Step 2: Task RowLengthen
// Step 3: Tasks Copy, PreClearUp and ClearUp
//
// Layout (internal codec, see gfe_internal.h):
//   * the matrix C being echelonised is held in place; block row i is the row
//     panel starting at row ro[i], its current (not yet pivotal) rows are
//     compacted at the top of the panel (REX keeps order, Section 2.3.4);
//   * B_j (pivot rows of block column j restricted to block columns k > j)
//     is one row panel per j, columns [co[j+1], beta);
//   * D_j.R is r_j x (b_j - r_j);
//   * K_ih (h <= i) live in one row panel per block row i, block row h's
//     stored columns at column offset ro[h]; M_jh likewise in one panel per j.
//   Only the columns the paper keeps are stored and multiplied (Section 3.1.1,
//   "transformation matrix abbreviation"); unstored zero columns are riffled
//   in (CRZ) and identity columns added (ADI) as Task UpdateRowTrafo says.
//
// Readings of points the paper leaves open (all validated against the oracle):
//   * u / delta from UNH mark NEW indices with 1; CRZ puts the stored columns
//     at the 0 positions and zero columns at the 1 positions; ADI puts the
//     identity 1 of the t-th new pivot row at the t-th 1 position of delta.
//   * RowLengthen keeps the stored columns at the positions of E_hj.rho inside
//     E_hb.rho (MKR's 1s) and riffles zeros elsewhere.
//   * ClearDown's second MAD is R' + A.E x R (the pseudo-code's form).
//   * "i = 1" means the first block row; every job accepts empty operands.
#include "gfe_internal.h"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <stdexcept>

namespace gfe {

struct OomError : std::runtime_error {
    OomError() : std::runtime_error("workspace too small") {}
};
struct CudaError : std::runtime_error {
    explicit CudaError(const std::string &s) : std::runtime_error(s) {}
};

// ---------------------------------------------------------------------------
// workspace arena (stack discipline) and host<->device staging
// ---------------------------------------------------------------------------
struct Arena {
    char *base = nullptr;
    size_t cap = 0, top = 0, peak = 0;
    bool dry = false;
    void *alloc(size_t bytes) {
        size_t a = (top + 255) & ~(size_t)255;
        top = a + ((bytes + 255) & ~(size_t)255);
        if (top > peak) peak = top;
        if (dry) return nullptr;
        if (top > cap) throw OomError();
        return base + a;
    }
    size_t mark() const { return top; }
    void release(size_t m) { top = m; }
};

constexpr size_t STAGE_BYTES = 8u << 20;

struct Stage {  // pinned host buffer + device ring for small index arrays
    char *host = nullptr;
    char *dev = nullptr;
    size_t top = 0;
};

// pinned host staging buffers (download area + upload ring), borrowed by
// each planner run and returned at its end
static std::mutex g_stage_mu;
static std::vector<char *> g_stage_free;

static char *stage_acquire() {
    {
        std::lock_guard<std::mutex> g(g_stage_mu);
        if (!g_stage_free.empty()) {
            char *p = g_stage_free.back();
            g_stage_free.pop_back();
            return p;
        }
    }
    char *p = nullptr;
    // mapped: the leaf ECH writes its pivot sets straight into the first 4 KB
    if (cudaHostAlloc((void **)&p, STAGE_BYTES + 4096, cudaHostAllocMapped) != cudaSuccess) return nullptr;
    return p;
}

static void stage_release(char *p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(g_stage_mu);
    g_stage_free.push_back(p);
}

struct StageGuard {
    char *p = nullptr;
    ~StageGuard() { stage_release(p); }
};

// side streams (non-blocking), borrowed per planner run and returned at its
// end; a stream belongs to the device that was current when it was made.
// Their priority is one below the critical path's and above the default, so
// that beside other work on the device (the batched form's one-launch
// kernels, whose CTAs hold an SM for long) the planner's CTAs are scheduled
// first as SMs come free.
static std::mutex g_stream_mu;
static std::vector<std::pair<int, cudaStream_t>> g_stream_free;

static cudaStream_t stream_acquire(int dev) {
    {
        std::lock_guard<std::mutex> g(g_stream_mu);
        for (size_t q = 0; q < g_stream_free.size(); ++q)
            if (g_stream_free[q].first == dev) {
                cudaStream_t s = g_stream_free[q].second;
                g_stream_free.erase(g_stream_free.begin() + q);
                return s;
            }
    }
    cudaStream_t s = nullptr;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return nullptr;
    const int prio = greatest < least ? greatest + 1 : least;
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio) != cudaSuccess) return nullptr;
    return s;
}

static void stream_release(int dev, cudaStream_t s) {
    if (!s) return;
    std::lock_guard<std::mutex> g(g_stream_mu);
    g_stream_free.push_back({dev, s});
}

// ordering events (no timing), borrowed per planner run: many small calls
// (the batched form) would otherwise create and destroy several per call
static std::vector<std::pair<int, cudaEvent_t>> g_event_free;

static cudaEvent_t event_acquire(int dev) {
    {
        std::lock_guard<std::mutex> g(g_stream_mu);
        for (size_t q = g_event_free.size(); q-- > 0;)
            if (g_event_free[q].first == dev) {
                cudaEvent_t e = g_event_free[q].second;
                g_event_free.erase(g_event_free.begin() + q);
                return e;
            }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

static void event_release(int dev, const std::vector<cudaEvent_t> &evs) {
    std::lock_guard<std::mutex> g(g_stream_mu);
    for (cudaEvent_t e : evs) g_event_free.push_back({dev, e});
}

// the critical path's stream: the device's highest priority, so its CTAs are
// scheduled before the side streams' when SMs come free
static std::vector<std::pair<int, cudaStream_t>> g_hp_free;

static cudaStream_t hp_acquire(int dev) {
    {
        std::lock_guard<std::mutex> g(g_stream_mu);
        for (size_t q = 0; q < g_hp_free.size(); ++q)
            if (g_hp_free[q].first == dev) {
                cudaStream_t s = g_hp_free[q].second;
                g_hp_free.erase(g_hp_free.begin() + q);
                return s;
            }
    }
    int least = 0, greatest = 0;
    cudaStream_t s = nullptr;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return nullptr;
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest) != cudaSuccess) return nullptr;
    return s;
}

static void hp_release(int dev, cudaStream_t s) {
    if (!s) return;
    std::lock_guard<std::mutex> g(g_stream_mu);
    g_hp_free.push_back({dev, s});
}

// What one level of the Chief runs beside its ClearDown chain: a side stream
// and the events that order the two (see chief()).
struct Level {
    cudaStream_t s1 = nullptr, s2 = nullptr;
    cudaEvent_t start = nullptr, aa = nullptr, cd = nullptr, b = nullptr, e4[4] = {nullptr, nullptr, nullptr, nullptr},
                join = nullptr, join2 = nullptr;
};

struct Ctx {
    Launch L;
    Arena ar;
    Stage sg;
    char *pinned = nullptr;  // download area (first 4 KB of the staging buffer)
    int32_t *info = nullptr;    // the same area as the device sees it: the leaf ECH's result
    cudaEvent_t ev = nullptr;   // marks the download of the leaf's result
    bool dry = false;
    int es = 1;
    int64_t syncs = 0;
    int dev = 0;
    int64_t thr = 2048, blk = 2048;  // block policy of this run
    int64_t leaf_rows = ECH_LEAF_ROWS;
    cudaStream_t main_st = nullptr;  // the critical path's stream (high priority)
    int depth = 0;                 // nesting depth of the Chief being planned
    std::vector<Level> levels;     // per depth, made on first use
    std::vector<cudaEvent_t> owned_events;

    ~Ctx() {
        for (auto &lv : levels) {
            stream_release(dev, lv.s1);
            stream_release(dev, lv.s2);
        }
        event_release(dev, owned_events);
    }
    cudaEvent_t make_event() {
        cudaEvent_t e = event_acquire(dev);
        if (!e) throw CudaError("cudaEventCreate failed");
        owned_events.push_back(e);
        return e;
    }
    Level &level(int d) {
        while ((int)levels.size() <= d) levels.emplace_back();
        Level &lv = levels[d];
        if (!dry && !lv.s1) {
            lv.s1 = stream_acquire(dev);
            lv.s2 = stream_acquire(dev);
            if (!lv.s1 || !lv.s2) throw CudaError("cudaStreamCreate failed");
            lv.start = make_event();
            lv.aa = make_event();
            lv.cd = make_event();
            lv.b = make_event();
            for (auto &e : lv.e4) e = make_event();
            lv.join = make_event();
            lv.join2 = make_event();
        }
        return lv;
    }
    // event ordering between the current stream and another
    void signal(cudaEvent_t e) {
        if (!dry) check(cudaEventRecord(e, L.st), "cudaEventRecord");
    }
    void await(cudaEvent_t e) {
        if (!dry) check(cudaStreamWaitEvent(L.st, e, 0), "cudaStreamWaitEvent");
    }

    void check(cudaError_t e, const char *what) {
        if (e != cudaSuccess) throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
    }
    static double now_ms() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
            .count();
    }
    void sync() {
        if (dry) return;
        const double t0 = now_ms();
        check(host_wait(main_st), "cudaStreamSynchronize");
        for (auto &lv : levels) {
            if (lv.s1) check(host_wait(lv.s1), "cudaStreamSynchronize");
            if (lv.s2) check(host_wait(lv.s2), "cudaStreamSynchronize");
        }
        check(cudaGetLastError(), "kernel launch");
        sg.top = 0;
        ++syncs;
        prof_count_sync(now_ms() - t0);
        prof_sync_point();
    }
    // wait for the work queued before the last record(); later work keeps
    // running and the upload ring is not recycled here
    void record() {
        if (!dry) check(cudaEventRecord(ev, L.st), "cudaEventRecord");
    }
    void wait_event() {
        if (dry) return;
        const double t0 = now_ms();
        check(cudaEventSynchronize(ev), "cudaEventSynchronize");
        check(cudaGetLastError(), "kernel launch");
        ++syncs;
        prof_count_sync(now_ms() - t0);
        prof_sync_point();
    }
    // upload an index array; returns its device address
    const int32_t *put(const std::vector<int32_t> &v) {
        if (dry || v.empty()) return nullptr;
        size_t bytes = (v.size() * 4 + 255) & ~(size_t)255;
        if (bytes > STAGE_BYTES) throw std::runtime_error("index array too large");
        if (sg.top + bytes > STAGE_BYTES) sync();
        std::memcpy(sg.host + sg.top, v.data(), v.size() * 4);
        check(cudaMemcpyAsync(sg.dev + sg.top, sg.host + sg.top, v.size() * 4, cudaMemcpyHostToDevice, L.st),
              "upload");
        const int32_t *d = (const int32_t *)(sg.dev + sg.top);
        sg.top += bytes;
        return d;
    }
    // leading dimensions are multiples of 64 elements (128 B): every view
    // that starts at a block boundary is then a legal TMA operand
    DMat mat(int64_t rows, int64_t cols) {
        DMat d;
        d.rows = rows;
        d.cols = cols;
        d.ld = cols > 0 ? (cols + 63) / 64 * 64 : 64;
        d.ptr = ar.alloc((size_t)(rows > 0 ? rows : 1) * (size_t)d.ld * es);
        return d;
    }
    void *at(const DMat &d, int64_t r, int64_t c) const {
        return dry ? nullptr : (char *)d.ptr + (r * d.ld + c) * es;
    }
};

static DMat sub(const Ctx &X, const DMat &d, int64_t r0, int64_t c0, int64_t rows, int64_t cols) {
    DMat s;
    s.ptr = X.at(d, r0, c0);
    s.rows = rows;
    s.cols = cols;
    s.ld = d.ld;
    return s;
}

// a view that the tensor-core multiply-add can take as its A or B operand
// (16-byte aligned start and pitch); always true in the dry run
static bool tma_ok(const Ctx &X, const DMat &d) {
    if (X.dry) return true;
    return ((uintptr_t)d.ptr & 15) == 0 && (d.ld * X.es) % 16 == 0;
}

// ---- job wrappers (no-ops in the dry run that sizes the workspace) ----
static void j_mad(Ctx &X, int64_t m, int64_t n, int64_t k, const DMat *W, const DMat &A, const DMat &B,
                  const DMat &C) {
    if (X.dry || m <= 0 || n <= 0) return;
    mad(X.L, m, n, k, W ? W->ptr : nullptr, W ? W->ld : 0, A.ptr, A.ld, B.ptr, B.ld, C.ptr, C.ld);
}
// an index array for a launch: short ones go by value with the launch,
// longer ones through the upload ring
static IdxMap idx(Ctx &X, const std::vector<int32_t> &v) {
    IdxMap m;
    m.n = (int64_t)v.size();
    if (m.n <= MAP_INLINE) m.host = v.data();
    else m.dev = X.put(v);
    return m;
}
static void j_rows(Ctx &X, int64_t nrows, int64_t ncols, const DMat &dst, const DMat &A, const DMat *B,
                   const std::vector<int32_t> &map) {
    if (X.dry || nrows <= 0 || ncols <= 0) return;
    gather_rows(X.L, nrows, ncols, dst.ptr, dst.ld, A.ptr, A.ld, B ? B->ptr : nullptr, B ? B->ld : 0, idx(X, map));
}
static void j_cols(Ctx &X, int64_t nrows, int64_t ncols, const DMat &dst, const DMat &src,
                   const std::vector<int32_t> &map) {
    if (X.dry || nrows <= 0 || ncols <= 0) return;
    gather_cols(X.L, nrows, ncols, dst.ptr, dst.ld, src.ptr, src.ld, idx(X, map));
}
static void j_copy(Ctx &X, int64_t rows, int64_t cols, const DMat &dst, const DMat &src) {
    if (X.dry || rows <= 0 || cols <= 0) return;
    copy2d(X.L, rows, cols, dst.ptr, dst.ld, src.ptr, src.ld);
}
static void j_zero(Ctx &X, int64_t rows, int64_t cols, const DMat &dst) {
    if (X.dry || rows <= 0 || cols <= 0) return;
    zero2d(X.L, rows, cols, dst.ptr, dst.ld);
}

// ---- subset bookkeeping (jobs UNH, UN0, MKR; Section 4.1) on the host ----
static std::vector<int32_t> complement(const std::vector<int32_t> &s, int64_t n) {
    std::vector<int32_t> out;
    out.reserve(n - (int64_t)s.size());
    size_t k = 0;
    for (int32_t x = 0; x < (int32_t)n; ++x) {
        if (k < s.size() && s[k] == x) ++k;
        else out.push_back(x);
    }
    return out;
}
// UNH: rho = rho1 U {x_i : i in rho2}, x = complement of rho1; u_l = 1 iff new
static void unh(const std::vector<int32_t> &rho1, const std::vector<int32_t> &rho2, int64_t alpha,
                std::vector<int32_t> &rho, std::vector<int32_t> &u) {
    std::vector<int32_t> x = complement(rho1, alpha);
    std::vector<int32_t> nw;
    for (int32_t i : rho2) nw.push_back(x[i]);
    rho.clear();
    u.clear();
    size_t a = 0, b = 0;
    while (a < rho1.size() || b < nw.size()) {
        if (b >= nw.size() || (a < rho1.size() && rho1[a] < nw[b])) {
            rho.push_back(rho1[a++]);
            u.push_back(0);
        } else {
            rho.push_back(nw[b++]);
            u.push_back(1);
        }
    }
}
// RRF map: row l <- (u_l == 0 ? B row #zeros-so-far : C row #ones-so-far)
static std::vector<int32_t> riffle_map(const std::vector<int32_t> &u) {
    std::vector<int32_t> m(u.size());
    int32_t z = 0, o = 0;
    for (size_t l = 0; l < u.size(); ++l) m[l] = u[l] ? -1 - (o++) : (z++);
    return m;
}
// CRZ map: new column t <- (newmask_t ? zero : old column #zeros-so-far)
static std::vector<int32_t> crz_map(const std::vector<int32_t> &newmask) {
    std::vector<int32_t> m(newmask.size());
    int32_t z = 0;
    for (size_t t = 0; t < newmask.size(); ++t) m[t] = newmask[t] ? -1 : (z++);
    return m;
}
static std::vector<int32_t> ones_positions(const std::vector<int32_t> &mask) {
    std::vector<int32_t> pos;
    for (size_t t = 0; t < mask.size(); ++t)
        if (mask[t]) pos.push_back((int32_t)t);
    return pos;
}

struct EchRes {
    int64_t r = 0;
    std::vector<int32_t> rho, gamma;
};

void chief(Ctx &X, const DMat &H, const std::vector<int64_t> &arows, const std::vector<int64_t> &bcols,
           bool trafo, bool wantR, const DMat &Mo, const DMat &Ko, const DMat &Ro, EchRes &out);

// ---------------------------------------------------------------------------
// ECH(H) -> (M, K, R, rho, gamma); H (alpha x beta) is destroyed.  Leaves go
// to the one-CTA kernel; larger blocks are split by the Chief itself, which
// is the paper's recursive scheme with a general rather than 2-way split.
// ---------------------------------------------------------------------------
// 0, 0: the block side comes from auto_block; otherwise it was fixed by
// gfe_set_block_policy
int64_t g_block_threshold = 0, g_block_big = 0;
// rows of a leaf block in the leaf grid; 0: auto_leaf_rows
int64_t g_leaf_rows = 0;
// tiles per CTA of the side streams' multiply-adds (0: one persistent CTA per SM)
int g_side_tiles = 4;

thread_local cudaEvent_t g_wait_event = nullptr;

cudaError_t host_wait(cudaStream_t s) {
    if (!g_wait_event) return cudaStreamSynchronize(s);
    cudaError_t e = cudaEventRecord(g_wait_event, s);
    return e != cudaSuccess ? e : cudaEventSynchronize(g_wait_event);
}

int64_t auto_leaf_rows(int p, int64_t m, int64_t n) {
    (void)m;
    (void)n;
    return ech_leaf_rows(p);
}

// Top-level block side (the a_i, b_j of Section 3.1) by field and size,
// from sweeps of the C2/C3 workloads on GB300: GF(2) is fastest with 3072
// from n ~ 12288 and 6144 from n ~ 65536, 3 <= p <= 13 with 2048 and
// p > 13 (256-row leaves) with 1024.  Sides are multiples of the 1024-row
// leaf; ragged ones (2560, 3584) were slower.
int64_t auto_block(int p, int64_t m, int64_t n) {
    const int64_t s = std::max(m, n);
    if (p == 2) return s >= 65536 ? 6144 : (s >= 12288 ? 3072 : 2048);
    if (p > 13) return 1024;  // the fp32 leaf takes 256 rows: smaller blocks keep its grid small
    return 2048;
}

static void block_policy(const Ctx &X, int64_t alpha, int64_t beta, std::vector<int64_t> &a,
                         std::vector<int64_t> &b) {
    int64_t ra, cb;
    if (std::max(alpha, beta) <= X.thr) {
        ra = X.leaf_rows;
        cb = ech_leaf_cols(X.L.p);
    } else {
        ra = cb = X.blk;
    }
    a.clear();
    b.clear();
    for (int64_t x = 0; x < alpha; x += ra) a.push_back(std::min(ra, alpha - x));
    for (int64_t x = 0; x < beta; x += cb) b.push_back(std::min(cb, beta - x));
}

// ech_start queues the ECH; for a leaf the pivot sets are still on their way
// to the host (ech_finish waits for them), so independent work can be queued
// in between.  A larger block runs the Chief, which returns complete.
static void ech_start(Ctx &X, const DMat &H, const DMat &Mo, const DMat &Ko, const DMat &Ro, EchRes &out,
                      bool &pending) {
    const int64_t alpha = H.rows, beta = H.cols;
    pending = false;
    out.r = 0;
    out.rho.clear();
    out.gamma.clear();
    if (alpha == 0 || beta == 0) return;
    const int lc = ech_leaf_cols(X.L.p);
    if (alpha <= ech_leaf_rows(X.L.p) && beta <= lc) {
        if (!X.dry) {
            // the kernel writes (r, rho, gamma) into mapped host memory; the
            // event after it makes them visible to the host
            ech_leaf(X.L, alpha, beta, H.ptr, H.ld, X.info, Mo.ptr, Mo.ld, Ko.ptr, Ko.ld, Ro.ptr, Ro.ld);
            X.record();
            pending = true;
        }
        return;
    }
    std::vector<int64_t> a, b;
    block_policy(X, alpha, beta, a, b);
    chief(X, H, a, b, true, true, Mo, Ko, Ro, out);
}

static void ech_finish(Ctx &X, EchRes &out, bool pending) {
    if (!pending) return;
    const int lc = ech_leaf_cols(X.L.p);
    X.wait_event();
    const int32_t *h = (const int32_t *)X.pinned;
    out.r = h[0];
    out.rho.assign(h + 1, h + 1 + out.r);
    out.gamma.assign(h + 1 + lc, h + 1 + lc + out.r);
}

void ech(Ctx &X, const DMat &H, const DMat &Mo, const DMat &Ko, const DMat &Ro, EchRes &out) {
    bool pending = false;
    ech_start(X, H, Mo, Ko, Ro, out, pending);
    ech_finish(X, out, pending);
}

// Is H, larger than a leaf, entirely zero?  One reduction and one wait: far
// cheaper than the Chief over its leaves discovering rank 0 leaf by leaf
// (a rank-deficient input leaves whole row blocks zero past its rank).
static bool block_is_zero(Ctx &X, const DMat &H) {
    if (X.dry || H.rows == 0 || H.cols == 0) return false;
    if (H.rows <= ech_leaf_rows(X.L.p) && H.cols <= ech_leaf_cols(X.L.p)) return false;  // a leaf: just run it
    volatile int32_t *flag = (volatile int32_t *)X.pinned;
    *flag = 0;
    any_nonzero(X.L, H.rows, H.cols, H.ptr, H.ld, X.info);
    X.record();
    X.wait_event();
    return *flag == 0;
}

// ---------------------------------------------------------------------------
// The Chief
// ---------------------------------------------------------------------------
void chief(Ctx &X, const DMat &H, const std::vector<int64_t> &arows, const std::vector<int64_t> &bcols,
           bool trafo, bool wantR, const DMat &Mo, const DMat &Ko, const DMat &Ro, EchRes &out) {
    const size_t mark0 = X.ar.mark();
    const int a = (int)arows.size(), b = (int)bcols.size();
    const int64_t alpha = H.rows, beta = H.cols;
    std::vector<int64_t> ro(a + 1, 0), co(b + 1, 0);
    for (int i = 0; i < a; ++i) ro[i + 1] = ro[i] + arows[i];
    for (int j = 0; j < b; ++j) co[j + 1] = co[j] + bcols[j];
    const int64_t maxa = *std::max_element(arows.begin(), arows.end());
    const int64_t maxb = *std::max_element(bcols.begin(), bcols.end());
    const int64_t minab = std::min(maxa, maxb);

    // ---- streams ----
    // The ClearDown chain is the critical path.  It runs on the planner's
    // high-priority stream s0 together with UpdateRow on the near columns (block column
    // j+1, which the next ClearDown reads).  Meanwhile UpdateRow on the far
    // columns (j+2 onwards) runs on side stream s1 and UpdateRowTrafo on
    // side stream s2 (they share no output).  Events order them:
    //   aa       s0 -> s1,s2  A.A of step t is ready (steps (1) may start)
    //   cd       s0 -> s1,s2  ClearDown of step t is done (A.M, A.K, A.E)
    //   b        s1 -> s0     step t's far columns are done; step t+1's near
    //                         columns are among them (and s1 is then done
    //                         with step t-1's copies of A.A, A.M, A.K, A.E)
    //   e4[t%4]  s2 -> s0     step t's UpdateRowTrafo is done; A.A, A.M, A.K
    //                         and A.E rotate through four copies, so
    //                         ClearDown of step t+4 may then overwrite them
    //   join     s1,s2 -> s0  end of Step 1
    // A nested Chief (the ECH of a large block) runs on s0 with side streams
    // of its own and joins them before it returns.
    const cudaStream_t s0 = X.L.st;
    const Level lv = X.level(X.depth);
    const cudaStream_t s1 = lv.s1, s2 = lv.s2;
    ++X.depth;
    // side-stream multiply-adds take at most g_side_tiles tiles per CTA, so
    // the ClearDown chain (on a higher-priority stream) gets SMs as tiles finish
    const int SIDE_TILES = g_side_tiles;
    auto on = [&](cudaStream_t s) {
        X.L.st = s;
        X.L.tiles_per_cta = s == s0 ? 0 : SIDE_TILES;
    };
    X.signal(lv.start);
    on(s1);
    X.await(lv.start);
    on(s2);
    X.await(lv.start);
    on(s0);

    // ---- buffers ----
    std::vector<int64_t> cur(arows.begin(), arows.end());  // current rows per block row
    std::vector<DMat> Bp(b);
    std::vector<int64_t> rB(b, 0);
    // B panels, D_j.R and M panels are swapped with a spare by the riffles,
    // so each family has one uniform capacity and leading dimension
    int64_t bcap = 0, bw = 0;
    for (int j = 0; j < b; ++j) {
        bcap = std::max(bcap, std::min(bcols[j], alpha));
        bw = std::max(bw, beta - co[j + 1]);
    }
    bw = std::max<int64_t>(bw, 1);
    for (int j = 0; j < b; ++j) Bp[j] = X.mat(bcap, bw);
    DMat Bsp = X.mat(bcap, bw);
    std::vector<DMat> DR(b);
    std::vector<std::vector<int32_t>> gam(b);
    for (int j = 0; j < b; ++j) DR[j] = X.mat(maxb, maxb);
    DMat DRsp = X.mat(maxb, maxb);
    // ClearDown outputs rotate through NRING copies: the side streams may
    // still read step t's while ClearDown runs steps t+1 .. t+NRING-1
    constexpr int NRING = 4;
    DMat AA[NRING], AM[NRING], AK[NRING], AE[NRING];
    for (int q = 0; q < NRING; ++q) {
        AA[q] = X.mat(maxa, maxb);
        AM[q] = X.mat(minab, minab);
        AK[q] = X.mat(maxa, minab);
        AE[q] = X.mat(maxb, maxb);
    }
    DMat Hb = X.mat(maxa, maxb), Rech = X.mat(minab, maxb), Rp = X.mat(maxb, maxb);
    // UpdateRow scratch, one set per stream: V stacked on W (one REX gather), X
    DMat VW0 = X.mat(maxa, maxb), X0 = X.mat(minab, maxb);
    DMat VW1 = X.mat(maxa, bw), X1 = X.mat(minab, bw);
    std::vector<DMat> Kp(a), Mp(b);
    DMat Msp, Zt, VWt, Xt, St;
    // stored widths of K_ih / M_jh; -1 = not stored yet (implicitly zero)
    std::vector<std::vector<int64_t>> wK(a, std::vector<int64_t>(a, 0)), wM(b, std::vector<int64_t>(a, -1));
    if (trafo) {
        for (int i = 0; i < a; ++i) {
            Kp[i] = X.mat(arows[i], ro[i + 1]);
        }
        for (int j = 0; j < b; ++j) Mp[j] = X.mat(bcap, alpha);
        Msp = X.mat(bcap, alpha);
        Zt = X.mat(maxa, maxa);
        VWt = X.mat(maxa, maxa);
        Xt = X.mat(minab, maxa);
        St = X.mat(std::min(maxb, alpha), maxa);
    }
    // E_ij.rho / E_ij.delta for every (i, j)
    std::vector<std::vector<std::vector<int32_t>>> Erho(a, std::vector<std::vector<int32_t>>(b)),
        Edel(a, std::vector<std::vector<int32_t>>(b));

    // ================= Step 1 =================
    // block rows whose ECH has found no pivot in some block: their later
    // blocks are tested for being zero before their ECH
    std::vector<char> zero_rows(a, 0);
    int64_t t = 0;  // step counter; t % NRING picks the copy of the ClearDown outputs
    for (int i = 0; i < a; ++i) {
        for (int j = 0; j < b; ++j, ++t) {
            const int q = (int)(t % NRING);
            const int64_t al = cur[i], bj = bcols[j];
            const int64_t r = (int64_t)gam[j].size();
            DMat Cij = sub(X, H, ro[i], co[j], al, bj);
            const int64_t wc = beta - co[j + 1];                   // UpdateRow panel width
            const int64_t wn = j + 1 < b ? bcols[j + 1] : 0;       // near columns (s0)
            const int64_t wf = wc - wn;                            // far columns (s1)
            DMat Z = sub(X, H, ro[i], co[j + 1], al, wc);
            bool near_ready = j == 0;  // step t-1's far columns are another row panel
            auto need_near = [&]() {
                if (!near_ready) X.await(lv.b);
                near_ready = true;
            };
            if (t >= NRING) X.await(lv.e4[q]);  // step t-NRING has let go of these buffers
            // ---------- Task ClearDown ----------
            EchRes e;
            std::vector<int32_t> lam;
            DMat AAv = AA[q];  // A.A (a gathered copy or a view of C_ij)
            bool ur1_done = false;                  // UpdateRow step (1) already queued
            std::vector<char> urt1_done(i + 1, 0);  // UpdateRowTrafo step (1) already queued
            if (i == 0) {
                DMat Rd = DR[j];
                if (!(zero_rows[i] && block_is_zero(X, Cij))) ech(X, Cij, AM[q], AK[q], Rd, e);
                if (e.r == 0 && al > 0 && bj > 0) zero_rows[i] = 1;
                gam[j] = e.gamma;
                lam.assign(e.r, 1);
            } else {
                const std::vector<int32_t> &g = gam[j];
                std::vector<int32_t> ng = complement(g, bj);
                // (CEX) A.A = C gamma^tr, A' = C gamma_bar^tr.  When gamma is the
                // leading columns 0..r-1 both are column ranges of C: use views
                // (C_ij is dead after ClearDown; ECH may overwrite A' in place).
                bool prefix = true;
                for (int64_t x = 0; x < r && prefix; ++x) prefix = g[x] == x;
                DMat Hh;
                if (prefix && tma_ok(X, Cij)) {
                    AAv = sub(X, Cij, 0, 0, al, r);
                    Hh = sub(X, Cij, 0, r, al, bj - r);
                } else {
                    j_cols(X, al, r, AA[q], Cij, g);
                    Hh = sub(X, Hb, 0, 0, al, bj - r);
                    j_cols(X, al, bj - r, Hh, Cij, ng);
                }
                X.signal(lv.aa);
                // (MAD) H := A' + A.A x D.R
                j_mad(X, al, bj - r, r, &Hh, AAv, DR[j], Hh);
                // (ECH), and meanwhile the steps (1) of UpdateRow and of
                // UpdateRowTrafo for h < i, which do not depend on its result
                bool pending = false;
                if (!(zero_rows[i] && block_is_zero(X, Hh))) ech_start(X, Hh, AM[q], AK[q], Rech, e, pending);
                if (wc > 0) {  // UpdateRow (1): Z := C + A.A x B
                    if (wn > 0) {
                        need_near();
                        DMat Zn = sub(X, Z, 0, 0, al, wn);
                        j_mad(X, al, wn, r, &Zn, AAv, Bp[j], Zn);
                    }
                    if (wf > 0) {
                        on(s1);
                        X.await(lv.aa);
                        DMat Zf = sub(X, Z, 0, wn, al, wf);
                        j_mad(X, al, wf, r, &Zf, AAv, sub(X, Bp[j], 0, wn, r, wf), Zf);
                        on(s0);
                    }
                    ur1_done = true;
                }
                if (trafo) {
                    on(s2);
                    X.await(lv.aa);
                    for (int h = 0; h < i; ++h) {
                        const std::vector<int32_t> &del = Edel[h][j];
                        const int64_t nc = (int64_t)del.size();
                        bool nonew = true;
                        for (int32_t dbit : del) nonew = nonew && dbit == 0;
                        if (j != 0 && !nonew) continue;             // needs CRZ: done after the ECH
                        DMat Kih = sub(X, Kp[i], 0, ro[h], al, nc);
                        DMat Mjh = sub(X, Mp[j], 0, ro[h], r, nc);
                        if (wM[j][h] != nc) {  // M_jh not stored yet: it is zero
                            j_zero(X, r, nc, Mjh);
                            wM[j][h] = nc;
                        }
                        j_mad(X, al, nc, r, j == 0 ? nullptr : &Kih, AAv, Mjh, Kih);   // UpdateRowTrafo (1)
                        urt1_done[h] = 1;
                    }
                    on(s0);
                }
                ech_finish(X, e, pending);
                if (e.r == 0 && al > 0 && bj - r > 0) zero_rows[i] = 1;
                const int64_t rp = e.r;
                if (rp > 0) {
                    // (CEX) A.E = D.R gamma'^tr, R' = D.R gamma'_bar^tr
                    std::vector<int32_t> ngp = complement(e.gamma, bj - r);
                    j_cols(X, r, rp, AE[q], DR[j], e.gamma);
                    j_cols(X, r, bj - r - rp, Rp, DR[j], ngp);
                    // (MAD) R' := R' + A.E x R
                    j_mad(X, r, bj - r - rp, rp, &Rp, AE[q], Rech, Rp);
                    // (UNH) and (RRF)
                    std::vector<int32_t> newg;
                    unh(g, e.gamma, bj, newg, lam);
                    j_rows(X, r + rp, bj - r - rp, DRsp, Rp, &Rech, riffle_map(lam));
                    std::swap(DR[j], DRsp);
                    gam[j] = newg;
                } else {
                    lam.assign(r, 0);
                }
            }
            const int64_t rp = e.r;
            X.signal(lv.cd);
            // ---------- Task Extend (UN0 / UNH) ----------
            unh(j == 0 ? std::vector<int32_t>() : Erho[i][j - 1], e.rho, arows[i], Erho[i][j], Edel[i][j]);
            std::vector<int32_t> nrho = complement(e.rho, al);
            std::vector<int32_t> rex(e.rho);  // REX into V (pivot rows) stacked on W (the others)
            rex.insert(rex.end(), nrho.begin(), nrho.end());
            const std::vector<int32_t> lmap = riffle_map(lam);
            // ---------- Task UpdateRow for all k > j at once (row panel) ----------
            // columns [c0, c0 + w) of the panel, scratch VW / Xs of the stream
            auto update_row = [&](int64_t c0, int64_t w, const DMat &VW, const DMat &Xs) {
                if (w <= 0) return;
                DMat Zc = sub(X, Z, 0, c0, al, w);
                DMat Bc = sub(X, Bp[j], 0, c0, r, w);
                if (i > 0 && !ur1_done) j_mad(X, al, w, r, &Zc, AAv, Bc, Zc);  // (1) Z := C + A.A x B
                if (rp == 0) return;
                DMat Vv = sub(X, VW, 0, 0, rp, w), Ww = sub(X, VW, rp, 0, al - rp, w);
                j_rows(X, al, w, VW, Zc, nullptr, rex);                 // (2) REX
                if (i > 0) {
                    j_mad(X, rp, w, rp, nullptr, AM[q], Vv, Xs);        // (3) X := A.M x V
                    j_mad(X, r, w, rp, &Bc, AE[q], Xs, Bc);             // (4) S := B + A.E x X
                    DMat Bs = sub(X, Bsp, 0, c0, r + rp, w);
                    j_rows(X, r + rp, w, Bs, Bc, &Xs, lmap);            // (5) RRF
                } else {
                    j_mad(X, rp, w, rp, nullptr, AM[q], Vv, Bc);        // (3)+(5) B := A.M x V
                }
                j_mad(X, al - rp, w, rp, &Ww, AK[q], Vv, Zc);           // (6) C := W + A.K x V
            };
            if (wc > 0) {
                need_near();
                update_row(0, wn, VW0, X0);
                on(s1);
                X.await(lv.cd);
                update_row(wn, wf, VW1, X1);
                X.signal(lv.b);
                on(s0);
                if (i > 0 && rp > 0) std::swap(Bp[j], Bsp);
            }
            cur[i] = al - rp;
            rB[j] = r + rp;
            // ---------- Task UpdateRowTrafo for h = 1..i (side stream s2) ----------
            on(s2);
            X.await(lv.cd);
            if (trafo && (rp > 0 || i > 0)) {
                for (int h = 0; h <= i; ++h) {
                    const std::vector<int32_t> &del = Edel[h][j];
                    const int64_t nc = (int64_t)del.size();
                    DMat Kih = sub(X, Kp[i], 0, ro[h], al, nc);
                    DMat Mjh = sub(X, Mp[j], 0, ro[h], r, nc);
                    const bool first_j = (j == 0);
                    if (h != i && wM[j][h] != nc) {  // M_jh not stored yet: it is zero
                        j_zero(X, r, nc, Mjh);
                        wM[j][h] = nc;
                    }
                    // Z is built in place in K_ih's slot when CRZ would not move
                    // a column (no new pivot rows of block row h here), or when
                    // K_ih is 0 so far (j = 1, h != i); otherwise in Zt.
                    bool nonew = true;
                    for (int32_t dbit : del) nonew = nonew && dbit == 0;
                    const bool inplace = first_j ? (h != i) : nonew;
                    DMat Zz = inplace ? Kih : Zt;
                    // (+) CRZ, (1)
                    if (!first_j && !inplace) {
                        DMat Kold = sub(X, Kp[i], 0, ro[h], al, wK[i][h]);
                        j_cols(X, al, nc, Zz, Kold, crz_map(del));
                    }
                    if (h != i && !urt1_done[h]) j_mad(X, al, nc, r, first_j ? nullptr : &Zz, AAv, Mjh, Zz);
                    if (rp == 0) {  // nothing pivotal: K := Z, M unchanged
                        if (!inplace) j_copy(X, al, nc, Kih, Zz);
                        wK[i][h] = nc;
                        continue;
                    }
                    DMat Xx = Xt;
                    if (first_j && h == i) {
                        j_copy(X, rp, nc, Xx, AM[q]);                      // (3) X := A.M   (V is 1)
                        j_copy(X, al - rp, nc, Kih, AK[q]);                // (6) K := A.K   (V is 1, W is 0)
                    } else {
                        DMat Vv = sub(X, VWt, 0, 0, rp, nc), Ww = sub(X, VWt, rp, 0, al - rp, nc);
                        j_rows(X, al, nc, VWt, Zz, nullptr, rex);          // (2) REX
                        if (h == i && !X.dry) {                            // (+) ADI
                            const std::vector<int32_t> pos = ones_positions(del);
                            set_ones(X.L, rp, Vv.ptr, Vv.ld, idx(X, pos));
                        }
                        j_mad(X, rp, nc, rp, nullptr, AM[q], Vv, Xx);      // (3) X := A.M x V
                        j_mad(X, al - rp, nc, rp, &Ww, AK[q], Vv, Kih);    // (6) K := W + A.K x V
                    }
                    wK[i][h] = nc;
                    // (4) S and (5) M := RRF(lambda, S, X)
                    DMat Mn = sub(X, Msp, 0, ro[h], r + rp, nc);
                    if (h != i) {
                        j_mad(X, r, nc, rp, &Mjh, AE[q], Xx, Mjh);
                        j_rows(X, r + rp, nc, Mn, Mjh, &Xx, lmap);
                    } else if (i != 0) {
                        DMat Ss = St;
                        j_mad(X, r, nc, rp, nullptr, AE[q], Xx, Ss);
                        j_rows(X, r + rp, nc, Mn, Ss, &Xx, lmap);
                    } else {
                        j_copy(X, rp, nc, Mn, Xx);
                    }
                    wM[j][h] = nc;
                }
                if (rp > 0) std::swap(Mp[j], Msp);
            }
            X.signal(lv.e4[q]);
            on(s0);
        }
    }
    on(s1);
    X.signal(lv.join);
    on(s2);
    X.signal(lv.join2);
    on(s0);
    X.await(lv.join);
    X.await(lv.join2);
    --X.depth;

    // ---- results: rank, Upsilon, varrho, offsets ----
    int64_t rank = 0;
    std::vector<int64_t> rowoff(b + 1, 0), nonoff(b + 1, 0), rhooff(a + 1, 0), kroff(a + 1, 0);
    for (int j = 0; j < b; ++j) {
        rowoff[j + 1] = rowoff[j] + (int64_t)gam[j].size();
        nonoff[j + 1] = nonoff[j] + bcols[j] - (int64_t)gam[j].size();
    }
    for (int i = 0; i < a; ++i) {
        rhooff[i + 1] = rhooff[i] + (int64_t)Erho[i][b - 1].size();
        kroff[i + 1] = kroff[i] + arows[i] - (int64_t)Erho[i][b - 1].size();
    }
    rank = rowoff[b];
    out.r = rank;
    out.gamma.clear();
    out.rho.clear();
    for (int j = 0; j < b; ++j)
        for (int32_t g : gam[j]) out.gamma.push_back((int32_t)(co[j] + g));
    for (int i = 0; i < a; ++i)
        for (int32_t x : Erho[i][b - 1]) out.rho.push_back((int32_t)(ro[i] + x));
    if (X.dry) {  // worst case: every block keeps all its columns
        rank = 0;
    }

    // ================= Step 2: RowLengthen (into the output M) =================
    // Block row j of the output M takes, for every h, M_jh widened to
    // E_hb.rho: MKR marks E_hj.rho inside E_hb.rho, CRZ puts the stored
    // columns at the marks and zeros elsewhere.  All h at once: one column
    // gather per j over the full width (-1 = a zero column).
    if (trafo && rank > 0) {
        std::vector<int32_t> map(rank);
        for (int j = 0; j < b; ++j) {
            const int64_t rj = (int64_t)gam[j].size();
            if (rj == 0) continue;
            for (int h = 0; h < a; ++h) {
                const std::vector<int32_t> &fin = Erho[h][b - 1];
                const std::vector<int32_t> &ej = Erho[h][j];
                const int64_t nf = (int64_t)fin.size();
                const bool stored = wM[j][h] == (int64_t)ej.size();  // else M_jh = 0
                size_t q = 0;
                int32_t z = 0;
                for (int64_t t = 0; t < nf; ++t) {
                    const bool keep = q < ej.size() && ej[q] == fin[t];
                    if (keep) ++q;
                    map[rhooff[h] + t] = (keep && stored) ? (int32_t)(ro[h] + z) : -1;
                    if (keep) ++z;
                }
            }
            j_cols(X, rj, rank, sub(X, Mo, rowoff[j], 0, rj, rank), Mp[j], map);
        }
        // K output: block row i takes slot h's stored columns for h <= i,
        // zeros for h > i; one column gather per i
        for (int i = 0; i < a; ++i) {
            const int64_t nk = kroff[i + 1] - kroff[i];
            if (nk == 0) continue;
            for (int h = 0; h < a; ++h)
                for (int64_t t = rhooff[h]; t < rhooff[h + 1]; ++t)
                    map[t] = h <= i ? (int32_t)(ro[h] + t - rhooff[h]) : -1;
            j_cols(X, nk, rank, sub(X, Ko, kroff[i], 0, nk, rank), Kp[i], map);
        }
    }

    // ================= Step 3: Copy, PreClearUp, ClearUp =================
    // R is assembled in a workspace whose block columns start at multiples
    // of 64 (padding columns stay zero), so every ClearUp operand is a legal
    // TMA tensor; the dense R is gathered from it at the end.
    if (wantR) {
        const int64_t nr = beta - rank;
        std::vector<int64_t> pad(b + 1, 0);
        for (int j = 0; j < b; ++j) pad[j + 1] = pad[j] + (bcols[j] - (int64_t)gam[j].size() + 63) / 64 * 64;
        DMat Rw = X.mat(std::min(alpha, beta), std::max<int64_t>(pad[b], 1));
        j_zero(X, rank, pad[b], Rw);
        for (int j = 0; j < b; ++j) {  // Copy: R_jj := D_j.R
            const int64_t rj = (int64_t)gam[j].size();
            j_copy(X, rj, bcols[j] - rj, sub(X, Rw, rowoff[j], pad[j], rj, bcols[j] - rj), DR[j]);
        }
        DMat Xcat = X.mat(std::min(alpha, beta), maxb);
        for (int k = b - 1; k >= 0; --k) {
            const int64_t rk = (int64_t)gam[k].size();
            std::vector<int32_t> ngk = complement(gam[k], bcols[k]);
            // PreClearUp for every j < k at once: (X_jk, R_jk) := CEX(B_jk, D_k.gamma);
            // the rows of B_1k .. B_(k-1)k are addressed through a row-pointer list
            if (rowoff[k] > 0 && !X.dry) {
                std::vector<int32_t> rp32(2 * rowoff[k]);
                for (int j = 0; j < k; ++j) {
                    const int64_t rj = (int64_t)gam[j].size();
                    for (int64_t l = 0; l < rj; ++l) {
                        const uint64_t a = (uint64_t)(uintptr_t)X.at(Bp[j], l, co[k] - co[j + 1]);
                        rp32[2 * (rowoff[j] + l)] = (int32_t)(uint32_t)(a & 0xFFFFFFFFu);
                        rp32[2 * (rowoff[j] + l) + 1] = (int32_t)(uint32_t)(a >> 32);
                    }
                }
                const uint64_t *rows = (const uint64_t *)X.put(rp32);
                if (rk > 0) gather_rowptr(X.L, rowoff[k], rk, Xcat.ptr, Xcat.ld, rows, X.put(gam[k]));
                if (bcols[k] - rk > 0) {
                    DMat Rjk = sub(X, Rw, 0, pad[k], rowoff[k], bcols[k] - rk);
                    gather_rowptr(X.L, rowoff[k], bcols[k] - rk, Rjk.ptr, Rjk.ld, rows, X.put(ngk));
                }
            }
            if (rk == 0 || rowoff[k] == 0) continue;
            // ClearUp for every j < k at once: R_jl += X_jk R_kl (l >= k), M_j += X_jk M_k
            DMat Rtop = sub(X, Rw, 0, pad[k], rowoff[k], pad[b] - pad[k]);
            DMat Rk = sub(X, Rw, rowoff[k], pad[k], rk, pad[b] - pad[k]);
            j_mad(X, rowoff[k], pad[b] - pad[k], rk, &Rtop, Xcat, Rk, Rtop);
            if (trafo) {
                DMat Mtop = sub(X, Mo, 0, 0, rowoff[k], rank);
                DMat Mk = sub(X, Mo, rowoff[k], 0, rk, rank);
                j_mad(X, rowoff[k], rank, rk, &Mtop, Xcat, Mk, Mtop);
            }
        }
        // dense R: non-pivot column t of block k sits at pad[k] + (t - nonoff[k])
        std::vector<int32_t> gmap(nr);
        for (int k = 0; k < b; ++k)
            for (int64_t t = nonoff[k]; t < nonoff[k + 1]; ++t) gmap[t] = (int32_t)(pad[k] + t - nonoff[k]);
        j_cols(X, rank, nr, Ro, Rw, gmap);
    }
    X.ar.release(mark0);
}

// ---------------------------------------------------------------------------
// entry used by the C ABI
// ---------------------------------------------------------------------------

// Runs the method on the (already imported) internal matrix H.
// Mo/Ko/Ro sized min(m,n) x min(m,n), m x min(m,n), min(m,n) x n.
void run_chief(const Launch &L, char *ws, size_t ws_bytes, bool dry, const DMat &H, bool trafo, bool wantR,
               const DMat &Mo, const DMat &Ko, const DMat &Ro, TopResult &res, size_t *peak, size_t base_used,
               int64_t *syncs) {
    Ctx X;
    X.L = L;
    X.dry = dry;
    X.es = codec_bytes(L.codec);
    X.ar.dry = dry;
    X.ar.base = ws;
    X.ar.cap = ws_bytes;
    X.ar.top = base_used;
    X.ar.peak = base_used;
    X.main_st = L.st;
    StageGuard guard;
    if (!dry) {
        X.check(cudaGetDevice(&X.dev), "cudaGetDevice");
        guard.p = stage_acquire();
        if (!guard.p) throw CudaError("cudaHostAlloc of the staging buffer failed");
        // layout: [0, 4096) download area, then the upload ring
        X.pinned = guard.p;
        X.sg.host = guard.p + 4096;
    }
    X.sg.dev = (char *)X.ar.alloc(STAGE_BYTES);
    if (!dry) {
        void *dinfo = nullptr;
        X.check(cudaHostGetDevicePointer(&dinfo, X.pinned, 0), "cudaHostGetDevicePointer");
        X.info = (int32_t *)dinfo;
    }
    struct EvGuard {
        cudaEvent_t e = nullptr;
        ~EvGuard() {
            if (e) cudaEventDestroy(e);
        }
    } evg;
    // the critical path runs on a high-priority stream of our own, after the
    // work already queued on the caller's stream
    struct HpGuard {
        int dev = 0;
        cudaStream_t s = nullptr;
        ~HpGuard() { hp_release(dev, s); }
    } hpg;
    if (!dry) {
        X.check(cudaEventCreateWithFlags(&evg.e, cudaEventDisableTiming | (g_wait_event ? cudaEventBlockingSync : 0)),
                "cudaEventCreate");
        X.ev = evg.e;
        hpg.dev = X.dev;
        hpg.s = hp_acquire(X.dev);
        if (!hpg.s) throw CudaError("cudaStreamCreateWithPriority failed");
        X.check(cudaEventRecord(X.ev, L.st), "cudaEventRecord");
        X.check(cudaStreamWaitEvent(hpg.s, X.ev, 0), "cudaStreamWaitEvent");
        X.L.st = X.main_st = hpg.s;
    }
    // one block side for the whole run (nested blocks of that side become leaves)
    if (g_block_threshold > 0) {
        X.thr = g_block_threshold;
        X.blk = g_block_big;
    } else {
        X.thr = X.blk = auto_block(L.p, H.rows, H.cols);
    }
    X.leaf_rows = std::min<int64_t>(g_leaf_rows > 0 ? g_leaf_rows : auto_leaf_rows(L.p, H.rows, H.cols),
                                    ech_leaf_rows(L.p));
    std::vector<int64_t> a, b;
    block_policy(X, H.rows, H.cols, a, b);
    EchRes e;
    const double t0 = Ctx::now_ms();
    if (H.rows > 0 && H.cols > 0) chief(X, H, a, b, trafo, wantR, Mo, Ko, Ro, e);
    if (!dry) {
        X.sync();
        if (g_prof_on) prof_host_ms(Ctx::now_ms() - t0);
    }
    res.r = e.r;
    res.rho = e.rho;
    res.gamma = e.gamma;
    if (peak) *peak = X.ar.peak;
    if (syncs) *syncs = X.syncs;
}

}  // namespace gfe
