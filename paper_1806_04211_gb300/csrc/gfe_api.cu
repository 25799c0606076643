// C ABI of libgfe (include/gfe.h): argument checks, workspace layout,
// conversion between the API storage and the internal codec, profiling.
#include "gfe.h"
#include "gfe_internal.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <tuple>
#include <mutex>
#include <thread>
#include <stdexcept>
#include <vector>

namespace gfe {

static int g_batch_workers = 0;  // 0 = default (8)

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string t_err;
void set_error(const std::string &s) { t_err = s; }
bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

// ---------------------------------------------------------------------------
// profiling: CUDA events around every launch while enabled
// ---------------------------------------------------------------------------
bool g_prof_on = false;
static int32_t g_prof_mask = -1;  // kinds whose launches are timed with events
static std::mutex g_prof_mu;
static gfe_profile g_prof;
struct Pending {
    int kind;
    cudaEvent_t a, b;
    int64_t m, n, k;
    cudaStream_t st;
};
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_evpool;
// launch trace: records of timed launches, start times relative to t0
static int64_t g_trace_cap = 0;
static std::vector<gfe_trace_record> g_trace;
static cudaEvent_t g_trace_t0 = nullptr;
// launches that time themselves on the device: a slot each in a device
// buffer ({start, end, CTAs in, CTAs out}, %globaltimer ns), read back when
// the profile or the trace is read
struct DevSlot {
    int kind;
    int64_t m, n, k;
    cudaStream_t st;
};
static uint64_t *g_dslots = nullptr;
static int64_t g_dcap = 0, g_dnext = 0, g_dresolved = 0;
static int g_ddev = -1;
static std::vector<DevSlot> g_dmeta;
static std::vector<std::pair<uint64_t, uint64_t>> g_dtimes;  // resolved {start, end}

static cudaEvent_t ev_get() {
    if (!g_evpool.empty()) {
        cudaEvent_t e = g_evpool.back();
        g_evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

uint64_t *prof_device_slot(const Launch &L, Kind k, int64_t m, int64_t n, int64_t kk) {
    if (!g_prof_on) return nullptr;
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!(g_prof_mask & (1 << k)) || !g_dslots || g_dnext >= g_dcap) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g_ddev) return nullptr;
    g_dmeta.push_back({(int)k, m, n, kk, L.st});
    return g_dslots + 4 * (g_dnext++);
}

void prof_count(Kind k) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.launches[k] += 1;
}

// device-timed launches issued since the last call: wait for the device,
// fetch their slots, add their times to the profile
static void resolve_device_locked() {
    if (!g_dslots || g_dresolved >= g_dnext) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != g_ddev) cudaSetDevice(g_ddev);
    cudaDeviceSynchronize();
    std::vector<uint64_t> v((size_t)(g_dnext - g_dresolved) * 4);
    cudaMemcpy(v.data(), g_dslots + 4 * g_dresolved, v.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    if (cur != g_ddev) cudaSetDevice(cur);
    for (int64_t q = g_dresolved; q < g_dnext; ++q) {
        const uint64_t t0 = v[(size_t)(q - g_dresolved) * 4], t1 = v[(size_t)(q - g_dresolved) * 4 + 1];
        const DevSlot &d = g_dmeta[(size_t)q];
        g_prof.ms[d.kind] += t1 > t0 ? (double)(t1 - t0) * 1e-6 : 0.0;
        g_prof.timed[d.kind] += 1;
        g_dtimes.push_back({t0, t1});
    }
    g_dresolved = g_dnext;
}

void prof_begin(const Launch &L, Kind k, cudaEvent_t *ev0) {
    *ev0 = nullptr;
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.launches[k] += 1;
    if (!(g_prof_mask & (1 << k))) return;
    if (g_trace_cap > 0 && !g_trace_t0) {  // the first traced launch starts the clock
        g_trace_t0 = ev_get();
        cudaEventRecord(g_trace_t0, L.st);
    }
    *ev0 = ev_get();
    cudaEventRecord(*ev0, L.st);
}

void prof_end(const Launch &L, Kind k, cudaEvent_t ev0, double madds, double bytes, int64_t m, int64_t n,
              int64_t kk) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.madds[k] += madds;
    g_prof.bytes[k] += bytes;
    if (!ev0) return;
    cudaEvent_t e1 = ev_get();
    cudaEventRecord(e1, L.st);
    g_pending.push_back({(int)k, ev0, e1, m, n, kk, L.st});
}

static void resolve_locked() {
    for (auto &p : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        g_prof.ms[p.kind] += ms;
        g_prof.timed[p.kind] += 1;
        if (g_trace_t0 && (int64_t)g_trace.size() < g_trace_cap) {
            float t = 0.f;
            cudaEventElapsedTime(&t, g_trace_t0, p.a);
            gfe_trace_record r{};
            r.kind = p.kind;
            r.m = p.m;
            r.n = p.n;
            r.k = p.k;
            r.stream = (uint64_t)(uintptr_t)p.st;
            r.start_ms = t;
            r.ms = ms;
            g_trace.push_back(r);
        }
        g_evpool.push_back(p.a);
        g_evpool.push_back(p.b);
    }
    g_pending.clear();
}

void prof_sync_point() {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (g_pending.size() > 4096) resolve_locked();
}

void prof_count_sync(double wait_ms) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.host_syncs += 1;
    g_prof.host_wait_ms += wait_ms;
}

void prof_host_ms(double ms) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.host_ms += ms;
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static bool is_prime(int p) {
    if (p < 2) return false;
    for (int d = 2; d * d <= p; ++d)
        if (p % d == 0) return false;
    return true;
}

bool field_ok(int p) { return is_prime(p) && p <= 251; }

static gfe_status check_matrix(const gfe_matrix *A) {
    if (!A) return (set_error("matrix argument is NULL"), GFE_EINVAL);
    if (!is_prime(A->p) || A->p > 251) return (set_error("p must be a prime <= 251"), GFE_EINVAL);
    if (A->m < 0 || A->n < 0) return (set_error("negative size"), GFE_EINVAL);
    if (A->m > (int64_t)1 << 30 || A->n > (int64_t)1 << 30) return (set_error("size too large"), GFE_EINVAL);
    if (A->fmt == GFE_BITS64) {
        if (A->p != 2) return (set_error("GFE_BITS64 needs p = 2"), GFE_EINVAL);
        if (A->ld % 8 || A->ld < 8 * ((A->n + 63) / 64)) return (set_error("ld too small for GFE_BITS64"), GFE_EINVAL);
    } else if (A->fmt == GFE_U8) {
        if (A->ld < A->n) return (set_error("ld < n"), GFE_EINVAL);
    } else {
        return (set_error("unknown storage format"), GFE_EINVAL);
    }
    if (A->m > 0 && A->n > 0 && !A->data) return (set_error("data is NULL"), GFE_EINVAL);
    return GFE_OK;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
static int64_t ld64(int64_t x) { return x > 0 ? (x + 63) / 64 * 64 : 64; }

struct Layout {
    size_t H, Mo, Ko, Ro, maps, err, arena, total;
};

static Layout layout(const gfe_matrix *A, bool trafo, bool wantR) {
    const int es = codec_bytes(codec_for(A->p));
    const int64_t m = A->m, n = A->n, mn = std::min(m, n);
    Layout Lo;
    size_t off = 0;
    Lo.H = off;
    off += al256((size_t)std::max<int64_t>(m, 1) * ld64(n) * es);
    Lo.Mo = off;
    off += trafo ? al256((size_t)std::max<int64_t>(mn, 1) * ld64(mn) * es) : 256;
    Lo.Ko = off;
    off += trafo ? al256((size_t)std::max<int64_t>(m, 1) * ld64(mn) * es) : 256;
    Lo.Ro = off;
    off += wantR ? al256((size_t)std::max<int64_t>(mn, 1) * ld64(n) * es) : 256;
    Lo.maps = off;
    off += al256((size_t)(m + n + 2) * 4);
    Lo.err = off;  // the call's error word
    off += 256;
    Lo.arena = off;
    Lo.total = off;
    return Lo;
}

static void launch_for(const gfe_matrix *A, uint32_t flags, void *stream, Launch &L) {
    L.st = (cudaStream_t)stream;
    L.p = A->p;
    L.codec = codec_for(A->p);
    L.impl = (flags & GFE_IMPL_PLAIN) ? 1 : 0;
}

// The workspace need depends only on the field (its codec and leaf width),
// the shape, the two flags and the block policy; the planner's dry run that
// finds it walks the whole block schedule, so its answers are memoised.
using QueryKey = std::tuple<int, int64_t, int64_t, bool, bool, int64_t, int64_t, int64_t>;
static std::mutex g_query_mu;
static std::map<QueryKey, size_t> g_query_memo;

static gfe_status query(const gfe_matrix *A, bool trafo, bool wantR, size_t *ws) {
    const QueryKey key{A->p, A->m, A->n, trafo, wantR, g_block_threshold, g_block_big, g_leaf_rows};
    {
        std::lock_guard<std::mutex> g(g_query_mu);
        auto it = g_query_memo.find(key);
        if (it != g_query_memo.end()) {
            *ws = it->second;
            return GFE_OK;
        }
    }
    Layout Lo = layout(A, trafo, wantR);
    Launch L;
    launch_for(A, 0, nullptr, L);
    DMat H;
    H.rows = A->m;
    H.cols = A->n;
    H.ld = ld64(A->n);
    DMat Mo, Ko, Ro;
    TopResult res;
    size_t peak = 0;
    try {
        run_chief(L, nullptr, 0, true, H, trafo, wantR, Mo, Ko, Ro, res, &peak, Lo.arena, nullptr);
    } catch (const std::exception &e) {
        set_error(e.what());
        return GFE_EINTERNAL;
    }
    *ws = al256(peak) + 4096;
    std::lock_guard<std::mutex> g(g_query_mu);
    if (g_query_memo.size() >= 4096) g_query_memo.clear();
    g_query_memo[key] = *ws;
    return GFE_OK;
}

static gfe_status run(const gfe_matrix *A, const gfe_result *out, int64_t *rank_dev, int64_t *pcols,
                      int64_t *prows, uint32_t flags, bool trafo, bool wantR, void *ws, size_t ws_bytes,
                      void *stream) {
    gfe_status st = check_matrix(A);
    if (st) return st;
    size_t need = 0;
    st = query(A, trafo, wantR, &need);
    if (st) return st;
    if (!ws || ws_bytes < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return GFE_EINVAL;
    }
    const bool wantE = out && (flags & GFE_WANT_DENSE_E) && out->E;
    const bool wantT = out && (flags & GFE_WANT_DENSE_T) && out->T;
    if (wantT && !trafo) return (set_error("dense T needs GFE_WANT_TRANSFORM"), GFE_EINVAL);
    Launch L;
    launch_for(A, flags, stream, L);
    Layout Lo = layout(A, trafo, wantR);
    char *base = (char *)ws;
    // this call's error word, in its own workspace: concurrent calls (the
    // batch's workers, the server's) never read one another's
    L.err = (int *)(base + Lo.err);
    if (!cuda_ok(cudaMemsetAsync(L.err, 0, sizeof(int), L.st), "error word")) return GFE_ECUDA;
    const int64_t m = A->m, n = A->n, mn = std::min(m, n);
    DMat H;
    H.ptr = base + Lo.H;
    H.rows = m;
    H.cols = n;
    H.ld = ld64(n);
    DMat Mo, Ko, Ro;
    Mo.ptr = base + Lo.Mo;
    Mo.rows = Mo.cols = mn;
    Mo.ld = ld64(mn);
    Ko.ptr = base + Lo.Ko;
    Ko.rows = m;
    Ko.cols = mn;
    Ko.ld = ld64(mn);
    Ro.ptr = base + Lo.Ro;
    Ro.rows = mn;
    Ro.cols = n;
    Ro.ld = ld64(n);
    const int es = codec_bytes(L.codec);
    TopResult res;
    try {
        // pack: API storage -> internal codec
        if (A->fmt == GFE_BITS64) import_bits(L, m, n, H.ptr, H.ld, (const uint64_t *)A->data, A->ld / 8);
        else import_u8(L, m, n, H.ptr, H.ld, (const uint8_t *)A->data, A->ld);
        int64_t syncs = 0;
        run_chief(L, base, ws_bytes, false, H, trafo, wantR, Mo, Ko, Ro, res, nullptr, Lo.arena, &syncs);
        const int64_t r = res.r;
        // rank, Upsilon, varrho
        std::vector<int64_t> hr(1, r), hg(res.gamma.begin(), res.gamma.end()), hp(res.rho.begin(), res.rho.end());
        if (!cuda_ok(cudaMemcpyAsync(rank_dev, hr.data(), 8, cudaMemcpyHostToDevice, L.st), "rank")) return GFE_ECUDA;
        if (pcols && r && !cuda_ok(cudaMemcpyAsync(pcols, hg.data(), 8 * r, cudaMemcpyHostToDevice, L.st), "pivot_cols"))
            return GFE_ECUDA;
        if (prows && r && !cuda_ok(cudaMemcpyAsync(prows, hp.data(), 8 * r, cudaMemcpyHostToDevice, L.st), "pivot_rows"))
            return GFE_ECUDA;
        const bool bits = A->fmt == GFE_BITS64;
        if (out) {
            if (out->R && wantR) {
                if (bits) export_bits(L, r, n - r, (uint64_t *)out->R, out->ldR / 8, Ro.ptr, Ro.ld);
                else export_u8(L, r, n - r, (uint8_t *)out->R, out->ldR, Ro.ptr, Ro.ld);
            }
            if (trafo && out->M) {
                if (bits) export_bits(L, r, r, (uint64_t *)out->M, out->ldM / 8, Mo.ptr, Mo.ld);
                else export_u8(L, r, r, (uint8_t *)out->M, out->ldM, Mo.ptr, Mo.ld);
            }
            if (trafo && out->K) {
                if (bits) export_bits(L, m - r, r, (uint64_t *)out->K, out->ldK / 8, Ko.ptr, Ko.ld);
                else export_u8(L, m - r, r, (uint8_t *)out->K, out->ldK, Ko.ptr, Ko.ld);
            }
            std::vector<int32_t> map;
            int32_t *dmap = (int32_t *)(base + Lo.maps);
            if (wantE) {
                map.assign(n, 0);
                std::vector<char> isp(n, 0);
                for (int64_t l = 0; l < r; ++l) {
                    map[res.gamma[l]] = (int32_t)l;
                    isp[res.gamma[l]] = 1;
                }
                int32_t j = 0;
                for (int64_t c = 0; c < n; ++c)
                    if (!isp[c]) map[c] = -1 - (j++);
                if (!cuda_ok(cudaMemcpyAsync(dmap, map.data(), 4 * n, cudaMemcpyHostToDevice, L.st), "map"))
                    return GFE_ECUDA;
                build_E(L, A->fmt, m, n, r, out->E, out->ldE, Ro.ptr, Ro.ld, dmap);
                if (!cuda_ok(host_wait(L.st), "sync")) return GFE_ECUDA;
            }
            if (wantT) {
                map.assign(m, 0);
                std::vector<char> isp(m, 0);
                for (int64_t s = 0; s < r; ++s) {
                    map[res.rho[s]] = (int32_t)s;
                    isp[res.rho[s]] = 1;
                }
                int32_t t = 0;
                for (int64_t x = 0; x < m; ++x)
                    if (!isp[x]) map[x] = -1 - (t++);
                if (!cuda_ok(cudaMemcpyAsync(dmap, map.data(), 4 * m, cudaMemcpyHostToDevice, L.st), "map"))
                    return GFE_ECUDA;
                build_T(L, A->fmt, m, r, out->T, out->ldT, Mo.ptr, Mo.ld, Ko.ptr, Ko.ld, dmap);
            }
        }
        (void)es;
        if (!cuda_ok(host_wait(L.st), "final sync")) return GFE_ECUDA;
        if (!cuda_ok(cudaGetLastError(), "kernel launch")) return GFE_ECUDA;
        int gave_up = 0;
        if (!cuda_ok(read_error_word(L.st, L.err, &gave_up) ? cudaSuccess : cudaErrorUnknown, "error word read"))
            return GFE_ECUDA;
        if (gave_up) {
            set_error("a tensor-core multiply-add timed out waiting on its pipeline");
            return GFE_ETIMEOUT;
        }
    } catch (const std::exception &e) {
        set_error(e.what());
        if (std::string(e.what()).find("workspace") != std::string::npos) return GFE_ENOMEM;
        return GFE_ECUDA;
    }
    return GFE_OK;
}

}  // namespace gfe

using namespace gfe;

extern "C" {

gfe_status gfe_query_workspace(const gfe_matrix *A, uint32_t flags, size_t *ws_bytes) {
    gfe_status st = check_matrix(A);
    if (st) return st;
    if (!ws_bytes) return (set_error("ws_bytes is NULL"), GFE_EINVAL);
    bool trafo = (flags & (GFE_WANT_TRANSFORM | GFE_WANT_DENSE_T)) != 0;
    return query(A, trafo, true, ws_bytes);
}

gfe_status gfe_query_result_bytes(const gfe_matrix *A, uint32_t flags, size_t *out_bytes) {
    gfe_status st = check_matrix(A);
    if (st) return st;
    if (!out_bytes) return (set_error("out_bytes is NULL"), GFE_EINVAL);
    const bool bits = A->fmt == GFE_BITS64;
    const int64_t m = A->m, n = A->n, k = std::min(m, n);
    auto row = [&](int64_t c) -> size_t { return bits ? (size_t)((c + 63) / 64) * 8 : (size_t)c; };
    size_t total = al256(8) + 2 * al256((size_t)k * 8) + al256((size_t)k * row(n));
    if (flags & (GFE_WANT_TRANSFORM | GFE_WANT_DENSE_T)) total += al256((size_t)k * row(k)) + al256((size_t)m * row(k));
    if (flags & GFE_WANT_DENSE_E) total += al256((size_t)m * row(n));
    if (flags & GFE_WANT_DENSE_T) total += al256((size_t)m * row(m));
    *out_bytes = total;
    return GFE_OK;
}

gfe_status gfe_echelon(const gfe_matrix *A, const gfe_result *out, uint32_t flags, void *ws, size_t ws_bytes,
                       void *stream) {
    if (!out || !out->rank) return (set_error("out->rank is required"), GFE_EINVAL);
    bool trafo = (flags & (GFE_WANT_TRANSFORM | GFE_WANT_DENSE_T)) != 0;
    return run(A, out, out->rank, out->pivot_cols, out->pivot_rows, flags, trafo, true, ws, ws_bytes, stream);
}

gfe_status gfe_rank(const gfe_matrix *A, int64_t *rank_dev, int64_t *pivot_cols, int64_t *pivot_rows,
                    uint32_t flags, void *ws, size_t ws_bytes, void *stream) {
    if (!rank_dev) return (set_error("rank_dev is required"), GFE_EINVAL);
    return run(A, nullptr, rank_dev, pivot_cols, pivot_rows, flags, false, false, ws, ws_bytes, stream);
}

// ---------------------------------------------------------------------------
// batched form: independent matrices on a pool of host workers, each with its
// own CUDA stream and workspace slice; ordered after prior work on `stream`
// and completed on it (events)
// ---------------------------------------------------------------------------
static int batch_workers(int32_t count) {
    int w = g_batch_workers > 0 ? g_batch_workers : 8;
    return count < w ? (count > 0 ? count : 1) : w;
}

// GFE_WAIT_AUTO: workers sleep in their waits when there are more of them
// than host threads
static int g_wait_policy = GFE_WAIT_AUTO;

static bool workers_sleep(int nw) {
    if (g_wait_policy == GFE_WAIT_BLOCK) return true;
    if (g_wait_policy == GFE_WAIT_SPIN) return false;
    const unsigned hw = std::thread::hardware_concurrency();
    return hw == 0 || (unsigned)nw > hw;
}

// The batch is split: matrices that fit the one-CTA kernel (gfe_small.cu)
// and need no dense E / T are echelonised together by ONE launch; the
// others go to the pool of workers.  Workspace: the workers' slices, then
// each small matrix's m x ldw area, then the job table.
// A matrix whose work m n min(m,n) is above the cut-off would keep one SM
// busy long after the others are done (one CTA runs it at about 2e11
// multiply-adds/s); the blocked Chief spreads it over the whole GPU.
constexpr double SMALL_WORK_DEFAULT = 4e9;
static int64_t g_batch_small_max = SMALL_MAX;
static double g_batch_small_work = SMALL_WORK_DEFAULT;

static bool batch_small(const gfe_matrix &A, uint32_t flags) {
    if (flags & (GFE_WANT_DENSE_E | GFE_WANT_DENSE_T)) return false;
    if (A.m > g_batch_small_max || A.n > g_batch_small_max) return false;
    // work in units of the wide kernel's rate: the GF(2) kernel is about 16x
    // as fast and the byte kernel for p <= 13 (rest update on int8 tensor
    // instructions) about 2.5x
    const double rate = A.fmt == GFE_BITS64 ? 16.0 : (A.p <= SMALL_MAX_P ? 2.5 : 1.0);
    const double work = (double)A.m * (double)A.n * (double)std::min(A.m, A.n) / rate;
    if (work > g_batch_small_work) return false;
    return small_eligible(A.p, A.fmt, A.m, A.n);
}

}  // extern "C"

namespace gfe {
// for the server's grouping of small requests
bool batch_takes_small(const gfe_matrix &A, uint32_t flags) { return batch_small(A, flags); }
}  // namespace gfe

extern "C" {

struct BatchPlan {
    std::vector<int32_t> small, rest;
    std::vector<size_t> small_off;  // offset of each small matrix's area
    int nw = 0;
    size_t slice = 0, small_base = 0, jobs_off = 0, total = 0;
};

static gfe_status batch_plan(const gfe_matrix *As, int32_t count, uint32_t flags, BatchPlan &P) {
    size_t best = 0;
    for (int32_t i = 0; i < count; ++i) {
        gfe_status st = check_matrix(&As[i]);
        if (st) return st;
        if (batch_small(As[i], flags)) {
            P.small.push_back(i);
            continue;
        }
        P.rest.push_back(i);
        size_t w = 0;
        st = gfe_query_workspace(&As[i], flags, &w);
        if (st) return st;
        best = std::max(best, w);
    }
    P.nw = P.rest.empty() ? 0 : batch_workers((int32_t)P.rest.size());
    P.slice = al256(best);
    size_t off = P.slice * (size_t)P.nw;
    P.small_base = off;
    for (int32_t i : P.small) {
        P.small_off.push_back(off);
        off += al256((size_t)As[i].m * (size_t)small_ldw(As[i].fmt, As[i].n));
    }
    P.jobs_off = off;
    if (!P.small.empty()) off += al256(P.small.size() * sizeof(SmallJob)) + 256;  // + the three job counters
    P.total = off;
    return GFE_OK;
}

gfe_status gfe_query_batch_workspace(const gfe_matrix *As, int32_t count, uint32_t flags, size_t *ws_bytes) {
    if (!ws_bytes || count < 0 || (count && !As)) return (set_error("bad batch arguments"), GFE_EINVAL);
    BatchPlan P;
    gfe_status st = batch_plan(As, count, flags, P);
    if (st) return st;
    *ws_bytes = P.total;
    return GFE_OK;
}

gfe_status gfe_set_batch_small_max(int32_t side, double max_work) {
    if (side < 0) return (set_error("bad small-matrix side"), GFE_EINVAL);
    g_batch_small_max = std::min<int64_t>(side, SMALL_MAX);
    g_batch_small_work = max_work > 0 ? max_work : SMALL_WORK_DEFAULT;
    return GFE_OK;
}

gfe_status gfe_batch_echelon(const gfe_matrix *As, const gfe_result *outs, int32_t count, uint32_t flags,
                             void *ws, size_t ws_bytes, void *stream) {
    if (count < 0 || (count && (!As || !outs))) return (set_error("bad batch arguments"), GFE_EINVAL);
    if (count == 0) return GFE_OK;
    BatchPlan P;
    gfe_status st = batch_plan(As, count, flags, P);
    if (st) return st;
    if (!ws || ws_bytes < P.total) {
        set_error("workspace too small: need " + std::to_string(P.total) + " bytes");
        return GFE_EINVAL;
    }
    for (int32_t i : P.small)
        if (!outs[i].rank) return (set_error("rank output is NULL"), GFE_EINVAL);
    const int nw = P.nw;
    const size_t slice = P.slice;
    const int32_t nrest = (int32_t)P.rest.size();
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return GFE_ECUDA;
    cudaEvent_t start;
    if (!cuda_ok(cudaEventCreateWithFlags(&start, cudaEventDisableTiming), "event")) return GFE_ECUDA;
    cudaEventRecord(start, (cudaStream_t)stream);
    // the small matrices: one job table, one launch per kind of kernel (bytes
    // with p <= 13, bytes with larger p, GF(2) words), each on a stream of its
    // own, the most expensive matrices first (their CTAs start first)
    cudaStream_t small_st[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t small_done[3] = {nullptr, nullptr, nullptr};
    if (!P.small.empty()) {
        std::vector<SmallJob> jobs;
        jobs.reserve(P.small.size());
        const bool tr = (flags & GFE_WANT_TRANSFORM) != 0;
        for (size_t q = 0; q < P.small.size(); ++q) {
            const gfe_matrix &A = As[P.small[q]];
            const gfe_result &o = outs[P.small[q]];
            SmallJob J;
            J.A = A.data;
            J.lda = A.ld;
            J.W = (char *)ws + P.small_off[q];
            J.ldw = small_ldw(A.fmt, A.n);
            J.m = (int32_t)A.m;
            J.n = (int32_t)A.n;
            J.p = A.p;
            J.fmt = A.fmt;
            J.rank = o.rank;
            J.pcols = o.pivot_cols;
            J.prows = o.pivot_rows;
            J.R = o.R;
            J.ldR = o.ldR;
            J.M = tr ? o.M : nullptr;
            J.ldM = o.ldM;
            J.K = tr ? o.K : nullptr;
            J.ldK = o.ldK;
            jobs.push_back(J);
        }
        std::stable_sort(jobs.begin(), jobs.end(), [](const SmallJob &a, const SmallJob &b) {
            const int ka = small_kind(a.p, a.fmt), kb = small_kind(b.p, b.fmt);
            if (ka != kb) return ka < kb;
            return (double)a.m * a.n * std::min(a.m, a.n) > (double)b.m * b.n * std::min(b.m, b.n);
        });
        int nkind[3] = {0, 0, 0};
        for (const SmallJob &J : jobs) ++nkind[small_kind(J.p, J.fmt)];
        SmallJob *djobs = (SmallJob *)((char *)ws + P.jobs_off);
        Launch L;
        launch_for(&As[P.small[0]], flags, nullptr, L);
        bool ok = cuda_ok(cudaStreamCreateWithFlags(&small_st[0], cudaStreamNonBlocking), "stream") &&
                  cuda_ok(cudaStreamWaitEvent(small_st[0], start, 0), "stream wait");
        // pageable source: the call returns once the table has been staged
        ok = ok && cuda_ok(cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(SmallJob),
                                           cudaMemcpyHostToDevice, small_st[0]),
                           "job table upload");
        cudaEvent_t up = nullptr;
        ok = ok && cuda_ok(cudaEventCreateWithFlags(&up, cudaEventDisableTiming), "event") &&
             cuda_ok(cudaEventRecord(up, small_st[0]), "event record");
        for (int k = 1; ok && k < 3; ++k)  // the other kinds beside it, once the table is on the device
            if (nkind[k])
                ok = cuda_ok(cudaStreamCreateWithFlags(&small_st[k], cudaStreamNonBlocking), "stream") &&
                     cuda_ok(cudaStreamWaitEvent(small_st[k], up, 0), "stream wait");
        if (up) cudaEventDestroy(up);
        int first = 0;
        for (int k = 0; ok && k < 3; ++k) {
            if (nkind[k]) {
                L.st = small_st[k];
                int *counters = (int *)((char *)ws + P.jobs_off + al256(P.small.size() * sizeof(SmallJob)));
                ok = cuda_ok(ech_small_batch(L, djobs + first, nkind[k], k, counters + k), "small-matrix launch") &&
                     cuda_ok(cudaEventCreateWithFlags(&small_done[k], cudaEventDisableTiming), "event") &&
                     cuda_ok(cudaEventRecord(small_done[k], small_st[k]), "event record");
            }
            first += nkind[k];
        }
        if (ok && !nkind[0]) {  // stream 0 only carried the upload: its end orders nothing else
            ok = cuda_ok(cudaEventCreateWithFlags(&small_done[0], cudaEventDisableTiming), "event") &&
                 cuda_ok(cudaEventRecord(small_done[0], small_st[0]), "event record");
        }
        if (!ok) {  // what was launched still uses the workspace: let it finish first
            for (int k = 0; k < 3; ++k) {
                if (small_st[k]) {
                    cudaStreamSynchronize(small_st[k]);
                    cudaStreamDestroy(small_st[k]);
                }
                if (small_done[k]) cudaEventDestroy(small_done[k]);
            }
            cudaEventDestroy(start);
            return GFE_ECUDA;
        }
    }
    std::atomic<int32_t> next(0);
    std::mutex mu;
    gfe_status first = GFE_OK;
    std::string first_msg;
    std::vector<cudaStream_t> streams(nw, nullptr);
    std::vector<cudaEvent_t> done(nw, nullptr);
    std::vector<std::thread> pool;
    const bool trafo = (flags & (GFE_WANT_TRANSFORM | GFE_WANT_DENSE_T)) != 0;
    const bool sleep = workers_sleep(nw);
    for (int w = 0; w < nw; ++w) {
        pool.emplace_back([&, w] {
            cudaSetDevice(dev);
            cudaStream_t s = nullptr;
            gfe_status mine = GFE_OK;
            struct WaitGuard {
                ~WaitGuard() {
                    if (g_wait_event) cudaEventDestroy(g_wait_event);
                    g_wait_event = nullptr;
                }
            } wg;
            if (sleep && cudaEventCreateWithFlags(&g_wait_event, cudaEventDisableTiming | cudaEventBlockingSync) !=
                             cudaSuccess) {
                g_wait_event = nullptr;
                mine = GFE_ECUDA;
                set_error("worker event set-up failed");
            }
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamWaitEvent(s, start, 0) != cudaSuccess) {
                mine = GFE_ECUDA;
                set_error("worker stream set-up failed");
            }
            streams[w] = s;
            while (mine == GFE_OK) {
                const int32_t q = next.fetch_add(1);
                if (q >= nrest) break;
                const int32_t i = P.rest[q];
                mine = run(&As[i], &outs[i], outs[i].rank, outs[i].pivot_cols, outs[i].pivot_rows, flags, trafo,
                           true, (char *)ws + slice * w, slice, s);
            }
            if (mine != GFE_OK) {
                std::lock_guard<std::mutex> g(mu);
                if (first == GFE_OK) {
                    first = mine;
                    first_msg = gfe_last_error();
                }
                next.store(nrest);
            }
            if (s) {
                cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming);
                cudaEventRecord(done[w], s);
            }
        });
    }
    for (auto &t : pool) t.join();
    for (int w = 0; w < nw; ++w) {
        if (done[w]) {
            cudaStreamWaitEvent((cudaStream_t)stream, done[w], 0);
            cudaEventDestroy(done[w]);
        }
        if (streams[w]) cudaStreamDestroy(streams[w]);
    }
    for (int k = 0; k < 3; ++k) {
        if (small_done[k]) {
            cudaStreamWaitEvent((cudaStream_t)stream, small_done[k], 0);
            cudaEventDestroy(small_done[k]);
        }
        if (small_st[k]) cudaStreamDestroy(small_st[k]);
    }
    cudaEventDestroy(start);
    if (first != GFE_OK) {
        set_error(first_msg);
        return first;
    }
    return GFE_OK;
}

gfe_status gfe_set_wait_policy(int32_t policy) {
    if (policy < GFE_WAIT_AUTO || policy > GFE_WAIT_BLOCK) return (set_error("bad wait policy"), GFE_EINVAL);
    g_wait_policy = policy;
    return GFE_OK;
}

gfe_status gfe_set_batch_workers(int32_t workers) {
    g_batch_workers = workers > 0 ? (workers > GFE_MAX_BATCH_WORKERS ? GFE_MAX_BATCH_WORKERS : workers) : 0;
    return GFE_OK;
}

// operands A, B and C in the codec, then 256 bytes for the call's error word
size_t gfe_mad_workspace(int32_t p, int64_t m, int64_t n, int64_t k) {
    int es = codec_bytes(codec_for(p < 2 ? 2 : p));
    return al256((size_t)m * ld64(k) * es) + al256((size_t)k * ld64(n) * es) + al256((size_t)m * ld64(n) * es) + 256;
}

gfe_status gfe_mad(int32_t p, int64_t m, int64_t n, int64_t k, const uint8_t *W, int64_t ldw, const uint8_t *A,
                   int64_t lda, const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc, uint32_t flags, void *ws,
                   size_t ws_bytes, void *stream) {
    if (!is_prime(p) || p > 251) return (set_error("p must be a prime <= 251"), GFE_EINVAL);
    if (m < 0 || n < 0 || k < 0) return (set_error("negative size"), GFE_EINVAL);
    if (m == 0 || n == 0) return GFE_OK;
    if (!C || ldc < n || (k > 0 && (!A || !B || lda < k || ldb < n)) || (W && ldw < n))
        return (set_error("bad matrix argument"), GFE_EINVAL);
    if (!ws || ws_bytes < gfe_mad_workspace(p, m, n, k)) return (set_error("workspace too small"), GFE_EINVAL);
    Launch L;
    L.st = (cudaStream_t)stream;
    L.p = p;
    L.codec = codec_for(p);
    L.impl = (flags & GFE_IMPL_PLAIN) ? 1 : 0;
    const int es = codec_bytes(L.codec);
    const int64_t lk = ld64(k), ln = ld64(n);
    char *a = (char *)ws, *b = a + al256((size_t)m * lk * es), *c = b + al256((size_t)k * ln * es);
    L.err = (int *)(c + al256((size_t)m * ln * es));
    if (!cuda_ok(cudaMemsetAsync(L.err, 0, sizeof(int), L.st), "error word")) return GFE_ECUDA;
    if (k > 0) {
        import_u8(L, m, k, a, lk, A, lda);
        import_u8(L, k, n, b, ln, B, ldb);
    }
    if (W) import_u8(L, m, n, c, ln, W, ldw);
    mad(L, m, n, k, W ? c : nullptr, ln, a, lk, b, ln, c, ln);
    export_u8(L, m, n, C, ldc, c, ln);
    if (!cuda_ok(cudaGetLastError(), "kernel launch")) return GFE_ECUDA;
    // the call returns once the product is complete on `stream`: the read of
    // its error word is a copy on that stream
    int gave_up = 0;
    if (!read_error_word(L.st, L.err, &gave_up)) return (set_error("error word read failed"), GFE_ECUDA);
    if (gave_up) return (set_error("tensor-core multiply-add timed out"), GFE_ETIMEOUT);
    return GFE_OK;
}

gfe_status gfe_set_block_policy(int64_t threshold, int64_t block) {
    if (threshold <= 0 && block <= 0) {  // back to the measured table
        g_block_threshold = g_block_big = 0;
        return GFE_OK;
    }
    const int64_t t = threshold > 0 ? threshold : block, b = block > 0 ? block : threshold;
    // a block must itself be echelonised from leaves (b <= t), else the
    // split would recurse without end
    if (t < b) return (set_error("block policy needs block <= threshold"), GFE_EINVAL);
    g_block_threshold = t;
    g_block_big = b;
    return GFE_OK;
}

int64_t gfe_auto_block(int32_t p, int64_t m, int64_t n) { return auto_block(p, m, n); }

gfe_status gfe_set_side_tiles(int32_t tiles) {
    if (tiles < 0 || tiles > 1024) return (set_error("side tiles must be in [0, 1024]"), GFE_EINVAL);
    g_side_tiles = tiles;
    return GFE_OK;
}

gfe_status gfe_set_leaf_rows(int64_t rows) {
    if (rows < 0 || rows > ECH_LEAF_ROWS) return (set_error("leaf rows must be in [0, 1024]"), GFE_EINVAL);
    g_leaf_rows = rows;
    return GFE_OK;
}

gfe_status gfe_selftest_wait_timeout(int64_t limit_us, void *stream) {
    if (limit_us < 1 || limit_us > 10000000) return (set_error("limit_us out of range"), GFE_EINVAL);
    const int gave_up = wait_selftest((cudaStream_t)stream, limit_us);
    if (gave_up < 0) return (set_error("self-test could not run"), GFE_ECUDA);
    if (!cuda_ok(cudaGetLastError(), "self-test launch")) return GFE_ECUDA;
    if (gave_up == 1) return (set_error("bounded wait gave up as designed"), GFE_ETIMEOUT);
    return (set_error("the wait completed although nothing arrived"), GFE_EINTERNAL);
}

gfe_status gfe_profile_enable(int32_t mask) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_on = mask != 0;
    g_prof_mask = mask;
    return GFE_OK;
}

gfe_status gfe_profile_read(gfe_profile *out, int32_t reset) {
    if (!out) return (set_error("out is NULL"), GFE_EINVAL);
    std::lock_guard<std::mutex> g(g_prof_mu);
    resolve_locked();
    resolve_device_locked();
    *out = g_prof;
    if (reset) std::memset(&g_prof, 0, sizeof g_prof);
    return GFE_OK;
}

static void drop_device_slots_locked() {
    if (g_dslots) {
        cudaDeviceSynchronize();
        cudaFree(g_dslots);
    }
    g_dslots = nullptr;
    g_dcap = g_dnext = g_dresolved = 0;
    g_dmeta.clear();
    g_dtimes.clear();
}

gfe_status gfe_trace_enable(int64_t capacity) {
    if (capacity < 0) return (set_error("capacity < 0"), GFE_EINVAL);
    std::lock_guard<std::mutex> g(g_prof_mu);
    resolve_locked();
    g_trace.clear();
    if (g_trace_t0) g_evpool.push_back(g_trace_t0);
    g_trace_t0 = nullptr;
    g_trace_cap = capacity;
    drop_device_slots_locked();
    if (capacity) {
        g_trace.reserve((size_t)std::min<int64_t>(capacity, 1 << 20));
        // device slots for the launches that time themselves (the
        // tensor-core multiply-add)
        if (cudaGetDevice(&g_ddev) == cudaSuccess &&
            cudaMalloc((void **)&g_dslots, (size_t)capacity * 4 * sizeof(uint64_t)) == cudaSuccess &&
            cudaMemset(g_dslots, 0, (size_t)capacity * 4 * sizeof(uint64_t)) == cudaSuccess) {
            g_dcap = capacity;
        } else {
            if (g_dslots) cudaFree(g_dslots);
            g_dslots = nullptr;
            cudaGetLastError();
        }
    }
    return GFE_OK;
}

gfe_status gfe_trace_read(gfe_trace_record *out, int64_t cap, int64_t *count, int32_t reset) {
    if (!count || cap < 0 || (cap > 0 && !out)) return (set_error("gfe_trace_read: bad arguments"), GFE_EINVAL);
    std::lock_guard<std::mutex> g(g_prof_mu);
    resolve_locked();
    resolve_device_locked();
    // device-timed records: starts relative to the earliest of them
    std::vector<gfe_trace_record> all(g_trace);
    uint64_t t0 = ~0ull;
    for (auto &tt : g_dtimes)
        if (tt.first && tt.first < t0) t0 = tt.first;
    for (size_t q = 0; q < g_dtimes.size(); ++q) {
        const DevSlot &d = g_dmeta[q];
        gfe_trace_record r{};
        r.kind = d.kind;
        r.clock = 1;  // device clock
        r.m = d.m;
        r.n = d.n;
        r.k = d.k;
        r.stream = (uint64_t)(uintptr_t)d.st;
        r.start_ms = g_dtimes[q].first >= t0 ? (double)(g_dtimes[q].first - t0) * 1e-6 : 0.0;
        r.ms = g_dtimes[q].second > g_dtimes[q].first ? (double)(g_dtimes[q].second - g_dtimes[q].first) * 1e-6 : 0.0;
        all.push_back(r);
    }
    *count = (int64_t)all.size();
    const int64_t c = std::min<int64_t>(cap, *count);
    if (c) std::memcpy(out, all.data(), (size_t)c * sizeof(gfe_trace_record));
    if (reset) {
        g_trace.clear();
        if (g_trace_t0) g_evpool.push_back(g_trace_t0);
        g_trace_t0 = nullptr;
        // keep the device buffer, start its slots over
        if (g_dslots) {
            cudaMemset(g_dslots, 0, (size_t)g_dnext * 4 * sizeof(uint64_t));
            cudaDeviceSynchronize();
        }
        g_dnext = g_dresolved = 0;
        g_dmeta.clear();
        g_dtimes.clear();
    }
    return GFE_OK;
}

const char *gfe_status_str(gfe_status s) {
    switch (s) {
    case GFE_OK: return "ok";
    case GFE_EINVAL: return "invalid argument";
    case GFE_ENOMEM: return "out of memory";
    case GFE_ETIMEOUT: return "timeout";
    case GFE_EBUSY: return "busy";
    case GFE_ECUDA: return "CUDA error";
    case GFE_EINTERNAL: return "internal error";
    case GFE_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

const char *gfe_last_error(void) { return t_err.c_str(); }
const char *gfe_version(void) { return "gfe 0.1 (sm_103a)"; }

}  // extern "C"
