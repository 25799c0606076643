// Planner simulation (test infrastructure, CPU only): the library's planner
// and C-ABI code (csrc/gfe_chief.cu, csrc/gfe_api.cu, compiled as plain C++)
// linked against
//   * stand-ins for the CUDA runtime calls they make: streams and events are
//     handles, copies happen at once, and every stream carries a vector
//     clock (event record = snapshot, stream wait = join, host
//     synchronisation = join into the calling thread's clock);
//   * CPU restatements of each job the kernels implement (MAD, leaf ECH,
//     row / column gathers, copies, pack / unpack), written from the jobs'
//     definitions, sharing no code with the CUDA kernels or the oracle.
// Every element a job reads or writes is checked to lie in a registered
// buffer, and against the last write and the reads since, per stream: an
// access that is not ordered after a conflicting one of another stream (by
// stream order or an event) is reported as a race.  Results are compared
// with the oracle by the test that drives this file.
#include "gfe_internal.h"
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>
#include <mutex>

#include <array>
#include <map>
#include <string>
#include <unordered_map>
namespace {
struct Region { const char* b; size_t n; };
std::vector<Region> g_regions;
std::mutex g_rmu;
// ---- stream race checker: vector clocks over streams, shadow per byte ----
namespace race {
constexpr int NS = 16;
struct VC { int32_t c[NS] = {0}; void join(const VC& o) { for (int i = 0; i < NS; ++i) c[i] = std::max(c[i], o.c[i]); } };
std::mutex mu;
std::map<uintptr_t, int> sid;
VC svc[NS];
thread_local VC host;
int nstreams = 0;
std::map<uintptr_t, VC> evs;
struct Op { int s; int32_t clk; std::string what; };
std::vector<Op> ops;
thread_local int cur = -1;  // current op index
thread_local VC cur_vc;
struct Sh { int32_t w = -1; int32_t r[NS]; Sh() { for (int i = 0; i < NS; ++i) r[i] = -1; } };
std::unordered_map<uintptr_t, Sh*> pages;
long races = 0;
int id_of(uintptr_t s) { auto it = sid.find(s); if (it != sid.end()) return it->second; if (nstreams >= NS) { fprintf(stderr, "too many streams\n"); abort(); } sid[s] = nstreams; return nstreams++; }
void op_begin(cudaStream_t st, const char* what) {
    std::lock_guard<std::mutex> g(mu);
    int i = id_of((uintptr_t)st);
    svc[i].join(host); svc[i].c[i]++;
    ops.push_back({i, svc[i].c[i], what});
    cur = (int)ops.size() - 1; cur_vc = svc[i];
}
bool hb(int opi) { const Op& o = ops[opi]; return cur_vc.c[o.s] >= o.clk; }
void report(const char* kind, uintptr_t a, int other) {
    if (++races <= 10) fprintf(stderr, "RACE %s at %lx: op %s (stream %d clk %d) vs %s (stream %d clk %d)\n", kind, (unsigned long)a,
        ops[cur].what.c_str(), ops[cur].s, ops[cur].clk, ops[other].what.c_str(), ops[other].s, ops[other].clk);
}
void access(const void* p, size_t n, bool write) {
    if (cur < 0) return;
    std::lock_guard<std::mutex> g(mu);
    for (size_t k = 0; k < n; ++k) {
        uintptr_t a = (uintptr_t)p + k, pg = a >> 12;
        auto it = pages.find(pg); Sh* sh;
        if (it == pages.end()) { sh = new Sh[4096]; pages[pg] = sh; } else sh = it->second;
        Sh& x = sh[a & 4095];
        if (x.w >= 0 && x.w != cur && !hb(x.w)) report(write ? "write-after-write" : "read-after-write", a, x.w);
        if (write) {
            for (int i = 0; i < NS; ++i) if (x.r[i] >= 0 && x.r[i] != cur && !hb(x.r[i])) report("write-after-read", a, x.r[i]);
            x.w = cur; for (int i = 0; i < NS; ++i) x.r[i] = -1;
        } else {
            x.r[ops[cur].s] = cur;
        }
    }
}
}  // namespace race
void chk(const void* p, size_t bytes, const char* what, bool write = false) {
    const char* c = (const char*)p;
    {
        std::lock_guard<std::mutex> g(g_rmu);
        bool ok = false;
        for (auto& r : g_regions) if (c >= r.b && c + bytes <= r.b + r.n) { ok = true; break; }
        if (!ok) { fprintf(stderr, "SIM OOB: %s at %p (%zu bytes)\n", what, p, bytes); abort(); }
    }
    race::access(p, bytes, write);
}
}
extern "C" long sim_races() { return race::races; }
extern "C" void sim_race_reset() { std::lock_guard<std::mutex> g(race::mu); race::races = 0; race::ops.clear(); for (auto& kv : race::pages) delete[] kv.second; race::pages.clear(); race::cur = -1; race::sid.clear(); race::nstreams = 0; for (auto& v : race::svc) v = race::VC(); race::evs.clear(); race::host = race::VC(); }
extern "C" void sim_register(void* p, size_t n) { std::lock_guard<std::mutex> g(g_rmu); g_regions.push_back({(const char*)p, n}); }
extern "C" void sim_clear() { g_regions.clear(); }

// ---- CUDA stubs ----
extern "C" {
static uintptr_t g_handle = 0x1000;
cudaError_t cudaStreamSynchronize(cudaStream_t s) { std::lock_guard<std::mutex> g(race::mu); race::host.join(race::svc[race::id_of((uintptr_t)s)]); return cudaSuccess; }
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t) { return "sim"; }
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind k, cudaStream_t st) {
    race::op_begin(st, "memcpy");
    if (k != cudaMemcpyHostToDevice) chk(s, n, "memcpy src");
    if (k != cudaMemcpyDeviceToHost) chk(d, n, "memcpy dst", true);
    memcpy(d, s, n); race::cur = -1; return cudaSuccess; }
cudaError_t cudaMemsetAsync(void* d, int v, size_t n, cudaStream_t st) {
    race::op_begin(st, "memset");
    chk(d, n, "memset dst", true);
    memset(d, v, n); race::cur = -1; return cudaSuccess; }
cudaError_t cudaHostAlloc(void** p, size_t n, unsigned int) { *p = malloc(n); std::lock_guard<std::mutex> g(g_rmu); g_regions.push_back({(const char*)*p, n}); return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t* e) { std::lock_guard<std::mutex> g(race::mu); *e = (cudaEvent_t)(g_handle++); return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s) { std::lock_guard<std::mutex> g(race::mu); int i = race::id_of((uintptr_t)s); race::svc[i].join(race::host); race::evs[(uintptr_t)e] = race::svc[i]; return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t e) { std::lock_guard<std::mutex> g(race::mu); race::host.join(race::evs[(uintptr_t)e]); return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t, cudaEvent_t) { *ms = 0; return cudaSuccess; }
cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned int) { return cudaEventCreate(e); }
cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned int) { std::lock_guard<std::mutex> g(race::mu); *s = (cudaStream_t)(g_handle++); return cudaSuccess; }
cudaError_t cudaStreamCreateWithPriority(cudaStream_t* s, unsigned int, int) { std::lock_guard<std::mutex> g(race::mu); *s = (cudaStream_t)(g_handle++); return cudaSuccess; }
cudaError_t cudaDeviceGetStreamPriorityRange(int* least, int* greatest) { *least = 0; *greatest = -5; return cudaSuccess; }
cudaError_t cudaHostGetDevicePointer(void** d, void* h, unsigned int) { *d = h; return cudaSuccess; }
cudaError_t cudaStreamWaitEvent(cudaStream_t s, cudaEvent_t e, unsigned int) { std::lock_guard<std::mutex> g(race::mu); int i = race::id_of((uintptr_t)s); race::svc[i].join(race::host); race::svc[i].join(race::evs[(uintptr_t)e]); return cudaSuccess; }
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaGetDevice(int* d) { *d = 0; return cudaSuccess; }
}

namespace gfe {
static thread_local int g_p; static thread_local Codec g_c;
static int cen(int r, int p) { return r > (p >> 1) ? r - p : r; }
static int res_(int c, int p) { return c < 0 ? c + p : c; }
static int dec8(uint8_t b) { int mag = b & 0x7F; if (mag < 0x38) return 0; int e = mag >> 3, mt = mag & 7; int v = ((8 + mt) << (e - 7)) >> 3; return (b & 0x80) ? -v : v; }
static uint8_t enc8(int c) { if (!c) return 0; int s = c < 0, a = s ? -c : c; int e = 31 - __builtin_clz(a); int mt = ((a << 3) >> e) - 8; return (uint8_t)((s << 7) | ((e + 7) << 3) | mt); }
static int dec16(uint16_t b) { uint32_t u = (uint32_t)b << 16; float f; memcpy(&f, &u, 4); return (int)f; }
static uint16_t enc16(int c) { float f = (float)c; uint32_t u; memcpy(&u, &f, 4); return (uint16_t)(u >> 16); }
static int es() { return g_c == CODEC_F8 ? 1 : 2; }
static int get(const void* base, int64_t idx) { const char* a = (const char*)base + idx * es(); chk(a, es(), "read", false); return g_c == CODEC_F8 ? dec8(*(const uint8_t*)a) : dec16(*(const uint16_t*)a); }
static void put(void* base, int64_t idx, int c) { char* a = (char*)base + idx * es(); chk(a, es(), "write", true); if (g_c == CODEC_F8) *(uint8_t*)a = enc8(c); else *(uint16_t*)a = enc16(c); }
static void rawcpy(void* d, const void* s) { chk(s, es(), "rcopy"); chk(d, es(), "wcopy", true); memcpy(d, s, es()); }
static void setL(const Launch& L, const char* what = "kernel") { g_p = L.p; g_c = L.codec; race::op_begin(L.st, what); }
static int modp(long x, int p) { long r = x % p; return (int)(r < 0 ? r + p : r); }


void mad_plain(const Launch& L, int64_t m, int64_t n, int64_t k, const void* W, int64_t ldw, const void* A, int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc) {
    setL(L, "mad"); int p = L.p;
    std::vector<int> out(m * n);
    for (int64_t i = 0; i < m; ++i) for (int64_t j = 0; j < n; ++j) {
        long s = W ? get(W, i * ldw + j) : 0;
        for (int64_t t = 0; t < k; ++t) s += (long)get(A, i * lda + t) * get(B, t * ldb + j);
        out[i * n + j] = cen(modp(s, p), p);
    }
    for (int64_t i = 0; i < m; ++i) for (int64_t j = 0; j < n; ++j) put(C, i * ldc + j, out[i * n + j]);
}
bool mad_tc(const Launch&, int64_t, int64_t, int64_t, const void*, int64_t, const void*, int64_t, const void*, int64_t, void*, int64_t) { return false; }
void mad(const Launch& L, int64_t m, int64_t n, int64_t k, const void* W, int64_t ldw, const void* A, int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc) {
    if (m <= 0 || n <= 0) return;
    mad_plain(L, m, n, k, W, ldw, A, lda, B, ldb, C, ldc);
}
bool read_error_word(cudaStream_t st, const int* err, int* value) {
    *value = 0;
    if (!err) return true;
    cudaMemcpyAsync(value, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return true;
}
int wait_selftest(cudaStream_t, int64_t) { return 1; }
int64_t tc_k_chunk(int) { return 1 << 20; }
int ech_leaf_cols(int p) { return p == 2 ? ECH_LEAF_COLS_GF2 : ECH_LEAF_COLS; }
static int inv(int a, int p) { for (int x = 1; x < p; ++x) if (a * x % p == 1) return x; return 0; }
void ech_leaf(const Launch& L, int64_t alpha, int64_t beta, const void* H, int64_t ldh, int32_t* info, void* M, int64_t ldm, void* K, int64_t ldk, void* R, int64_t ldr) {
    setL(L, "ech_leaf"); int p = L.p;
    const int cap = ech_leaf_cols(L.p);
    if (alpha > ECH_LEAF_ROWS || beta > cap) { fprintf(stderr, "leaf too big\n"); abort(); }
    std::vector<std::vector<int>> S(alpha, std::vector<int>(beta)), T(alpha, std::vector<int>(cap, 0));
    for (int y = 0; y < alpha; ++y) for (int c = 0; c < beta; ++c) S[y][c] = res_(get(H, y * ldh + c), p);
    std::vector<int> piv(alpha, 0), slotOf(alpha, -1), slotRow, slotCol;
    int ns = 0;
    for (int c = 0; c < beta; ++c) {
        int x = -1;
        for (int y = 0; y < alpha; ++y) if (!piv[y] && S[y][c]) { x = y; break; }
        if (x < 0) continue;
        int s = (p - inv(S[x][c], p)) % p;
        for (int cc = c; cc < beta; ++cc) S[x][cc] = S[x][cc] * s % p;
        T[x][ns] = 1;
        for (int t = 0; t <= ns; ++t) T[x][t] = T[x][t] * s % p;
        piv[x] = 1; slotOf[x] = ns; slotRow.push_back(x); slotCol.push_back(c);
        for (int y = 0; y < alpha; ++y) if (y != x && S[y][c]) { int f = S[y][c];
            for (int cc = c; cc < beta; ++cc) S[y][cc] = (S[y][cc] + f * S[x][cc]) % p;
            for (int t = 0; t <= ns; ++t) T[y][t] = (T[y][t] + f * T[x][t]) % p; }
        ++ns;
    }
    int r = ns;
    chk(info, 4 * (1 + 2 * cap), "info", true);
    info[0] = r;
    std::vector<int> sortedSlot; std::vector<int> pivpos(alpha);
    int np = 0, nn = 0;
    for (int y = 0; y < alpha; ++y) { if (piv[y]) { info[1 + np] = y; sortedSlot.push_back(slotOf[y]); pivpos[y] = np++; } else pivpos[y] = nn++; }
    for (int l = 0; l < r; ++l) info[1 + cap + l] = slotCol[l];
    std::vector<int> nonCol; { int l = 0; for (int c = 0; c < beta; ++c) { if (l < r && slotCol[l] == c) ++l; else nonCol.push_back(c); } }
    for (int l = 0; l < r; ++l) for (int s2 = 0; s2 < r; ++s2) put(M, l * ldm + s2, cen(T[slotRow[l]][sortedSlot[s2]], p));
    for (int y = 0; y < alpha; ++y) if (!piv[y]) for (int s2 = 0; s2 < r; ++s2) put(K, pivpos[y] * ldk + s2, cen(T[y][sortedSlot[s2]], p));
    for (int l = 0; l < r; ++l) for (int j = 0; j < beta - r; ++j) put(R, l * ldr + j, cen(S[slotRow[l]][nonCol[j]], p));
}
// a map passed by value (host array) has no device memory to check
static const int32_t* map_of(const IdxMap& m, int64_t n) { if (m.host) return m.host; chk(m.dev, 4 * n, "map"); return m.dev; }
void gather_rows(const Launch& L, int64_t nrows, int64_t ncols, void* dst, int64_t ldd, const void* A, int64_t lda, const void* B, int64_t ldb, const IdxMap& mp) {
    setL(L, "gather_rows"); const int32_t* map = map_of(mp, nrows);
    for (int64_t r = 0; r < nrows; ++r) { int32_t s = map[r];
        for (int64_t c = 0; c < ncols; ++c) {
            const char* src = s >= 0 ? (const char*)A + (s * lda + c) * es() : (const char*)B + ((-1 - s) * ldb + c) * es();
            rawcpy((char*)dst + (r * ldd + c) * es(), src); } }
}
void gather_cols(const Launch& L, int64_t nrows, int64_t ncols, void* dst, int64_t ldd, const void* src, int64_t lds, const IdxMap& mp) {
    setL(L, "gather_cols"); const int32_t* map = map_of(mp, ncols);
    for (int64_t r = 0; r < nrows; ++r) for (int64_t c = 0; c < ncols; ++c) {
        int32_t s = map[c];
        if (s >= 0) rawcpy((char*)dst + (r * ldd + c) * es(), (const char*)src + (r * lds + s) * es());
        else put(dst, r * ldd + c, 0); }
}
void gather_rowptr(const Launch& L, int64_t nrows, int64_t ncols, void* dst, int64_t ldd, const uint64_t* rows, const int32_t* map) {
    setL(L, "gather_rowptr"); chk(rows, 8 * nrows, "rowptr"); chk(map, 4 * ncols, "map");
    for (int64_t r = 0; r < nrows; ++r) for (int64_t c = 0; c < ncols; ++c) {
        int32_t s = map[c];
        if (s >= 0) rawcpy((char*)dst + (r * ldd + c) * es(), (const char*)rows[r] + s * es()); else put(dst, r * ldd + c, 0); }
}
void set_ones(const Launch& L, int64_t count, void* V, int64_t ldv, const IdxMap& mp) { setL(L, "set_ones"); const int32_t* pos = map_of(mp, count); for (int64_t t = 0; t < count; ++t) put(V, t * ldv + pos[t], 1); }
void copy2d(const Launch& L, int64_t rows, int64_t cols, void* dst, int64_t ldd, const void* src, int64_t lds) {
    setL(L, "copy2d"); for (int64_t r = 0; r < rows; ++r) for (int64_t c = 0; c < cols; ++c) { if (src) rawcpy((char*)dst + (r * ldd + c) * es(), (const char*)src + (r * lds + c) * es()); else put(dst, r * ldd + c, 0); }
}
void zero2d(const Launch& L, int64_t rows, int64_t cols, void* dst, int64_t ldd) { copy2d(L, rows, cols, dst, ldd, nullptr, 0); }
void import_u8(const Launch& L, int64_t rows, int64_t cols, void* dst, int64_t ldd, const uint8_t* src, int64_t lds) {
    setL(L, "import_u8"); for (int64_t r = 0; r < rows; ++r) for (int64_t c = 0; c < cols; ++c) { chk(src + r * lds + c, 1, "imp"); put(dst, r * ldd + c, cen(src[r * lds + c], L.p)); } }
void import_bits(const Launch& L, int64_t rows, int64_t cols, void* dst, int64_t ldd, const uint64_t* src, int64_t ldw) {
    setL(L, "import_bits"); for (int64_t r = 0; r < rows; ++r) for (int64_t c = 0; c < cols; ++c) { chk(src + r * ldw + (c >> 6), 8, "impb"); put(dst, r * ldd + c, (int)((src[r * ldw + (c >> 6)] >> (c & 63)) & 1)); } }
void export_u8(const Launch& L, int64_t rows, int64_t cols, uint8_t* dst, int64_t ldd, const void* src, int64_t lds) {
    setL(L, "export_u8"); for (int64_t r = 0; r < rows; ++r) for (int64_t c = 0; c < cols; ++c) { chk(dst + r * ldd + c, 1, "exp", true); dst[r * ldd + c] = (uint8_t)res_(get(src, r * lds + c), L.p); } }
void export_bits(const Launch& L, int64_t rows, int64_t cols, uint64_t* dst, int64_t ldw, const void* src, int64_t lds) {
    setL(L, "export_bits"); int64_t nw = (cols + 63) >> 6;
    for (int64_t r = 0; r < rows; ++r) for (int64_t w = 0; w < nw; ++w) { uint64_t v = 0;
        for (int b = 0; b < 64 && w * 64 + b < cols; ++b) v |= (uint64_t)(get(src, r * lds + w * 64 + b) & 1) << b;
        chk(dst + r * ldw + w, 8, "expb", true); dst[r * ldw + w] = v; } }
void build_E(const Launch& L, int fmt, int64_t m, int64_t n, int64_t r, void* dst, int64_t ldd, const void* R, int64_t ldr, const int32_t* colmap) {
    setL(L, "build_E"); int p = L.p;
    for (int64_t row = 0; row < m; ++row) for (int64_t c = 0; c < n; ++c) {
        int v = 0; if (row < r) { int32_t q = colmap[c]; v = q >= 0 ? (q == row ? p - 1 : 0) : res_(get(R, row * ldr + (-1 - q)), p); }
        if (fmt == 1) { uint64_t* w = (uint64_t*)dst + row * (ldd / 8) + (c >> 6); chk(w, 8, "E", true); if (!(c & 63)) *w = 0; *w |= (uint64_t)(v & 1) << (c & 63); }
        else { uint8_t* d = (uint8_t*)dst + row * ldd + c; chk(d, 1, "E", true); *d = (uint8_t)v; } }
}
void build_T(const Launch& L, int fmt, int64_t m, int64_t r, void* dst, int64_t ldd, const void* M, int64_t ldm, const void* K, int64_t ldk, const int32_t* rowmap) {
    setL(L, "build_T"); int p = L.p;
    for (int64_t row = 0; row < m; ++row) for (int64_t x = 0; x < m; ++x) {
        int32_t q = rowmap[x]; int v;
        if (row < r) v = q >= 0 ? res_(get(M, row * ldm + q), p) : 0; else v = q >= 0 ? res_(get(K, (row - r) * ldk + q), p) : ((-1 - q) == row - r);
        if (fmt == 1) { uint64_t* w = (uint64_t*)dst + row * (ldd / 8) + (x >> 6); chk(w, 8, "T", true); if (!(x & 63)) *w = 0; *w |= (uint64_t)(v & 1) << (x & 63); }
        else { uint8_t* d = (uint8_t*)dst + row * ldd + x; chk(d, 1, "T", true); *d = (uint8_t)v; } }
}
void any_nonzero(const Launch& L, int64_t rows, int64_t cols, const void* A, int64_t lda, int32_t* flag) {
    setL(L, "any_nonzero");
    for (int64_t r = 0; r < rows; ++r) for (int64_t c = 0; c < cols; ++c)
        if (get(A, r * lda + c) != 0) { chk(flag, 4, "flag", true); *flag = 1; return; }
}
// the one-launch small-matrix batch: every job's result from its definition
// (column-by-column Gauss-Jordan on [A | 1] with the topmost available row as
// pivot, pivots scaled to -1), written in the API storage; the workspace
// area of a job is marked written, as the kernel works in place there
cudaError_t ech_small_batch(const Launch& L, const SmallJob* jobs, int count, int, int* next) {
    setL(L, "ech_small_batch");
    chk(next, 4, "job counter", true);
    chk(jobs, sizeof(SmallJob) * count, "jobs");
    for (int q = 0; q < count; ++q) {
        const SmallJob& J = jobs[q];
        const int m = J.m, n = J.n, p = J.p;
        const bool bits = J.fmt == 1;
        chk(J.W, (size_t)m * J.ldw, "small ws", true);
        std::vector<std::vector<int>> B(m, std::vector<int>(n + m, 0));
        for (int y = 0; y < m; ++y) {
            for (int c = 0; c < n; ++c) {
                if (bits) { const uint64_t* w = (const uint64_t*)((const char*)J.A + y * J.lda) + (c >> 6); chk(w, 8, "small A"); B[y][c] = (int)((*w >> (c & 63)) & 1); }
                else { const uint8_t* b = (const uint8_t*)J.A + y * J.lda + c; chk(b, 1, "small A"); B[y][c] = *b % p; }
            }
            B[y][n + y] = 1;
        }
        std::vector<int> isp(m, 0), pr, pc;  // pivot rows / columns in pivot order
        for (int c = 0; c < n; ++c) {
            int x = -1;
            for (int y = 0; y < m; ++y) if (!isp[y] && B[y][c]) { x = y; break; }
            if (x < 0) continue;
            const int s = (p - inv(B[x][c], p)) % p;
            for (auto& v : B[x]) v = v * s % p;
            for (int y = 0; y < m; ++y) if (y != x && B[y][c]) { const int f = B[y][c]; for (int k = 0; k < n + m; ++k) B[y][k] = (B[y][k] + f * B[x][k]) % p; }
            isp[x] = 1; pr.push_back(x); pc.push_back(c);
        }
        const int r = (int)pc.size();
        std::vector<int> rho, rhob, ups = pc, upsb;
        for (int y = 0; y < m; ++y) (isp[y] ? rho : rhob).push_back(y);
        { size_t l = 0; for (int c = 0; c < n; ++c) { if (l < pc.size() && pc[l] == c) ++l; else upsb.push_back(c); } }
        chk(J.rank, 8, "rank", true); *J.rank = r;
        for (int l = 0; l < r; ++l) {
            if (J.pcols) { chk(J.pcols + l, 8, "pcols", true); J.pcols[l] = ups[l]; }
            if (J.prows) { chk(J.prows + l, 8, "prows", true); J.prows[l] = rho[l]; }
        }
        auto out = [&](void* base, int64_t ld, int row, int col, int v) {
            if (bits) {
                uint64_t* w = (uint64_t*)((char*)base + row * ld) + (col >> 6); chk(w, 8, "small out", true);
                *w = (*w & ~(1ull << (col & 63))) | ((uint64_t)(v & 1) << (col & 63));
            } else { uint8_t* b = (uint8_t*)base + row * ld + col; chk(b, 1, "small out", true); *b = (uint8_t)v; }
        };
        for (int l = 0; l < r; ++l) {  // pivot l (ascending column) sits in row pr[l]
            if (J.R) for (int t = 0; t < n - r; ++t) out(J.R, J.ldR, l, t, B[pr[l]][upsb[t]]);
            if (J.M) for (int s2 = 0; s2 < r; ++s2) out(J.M, J.ldM, l, s2, B[pr[l]][n + rho[s2]]);
        }
        if (J.K) for (int t = 0; t < m - r; ++t) for (int s2 = 0; s2 < r; ++s2) out(J.K, J.ldK, t, s2, B[rhob[t]][n + rho[s2]]);
        if (bits) {  // pad bits of every written output word are 0
            auto pad = [&](void* base, int64_t ld, int rows, int cols) {
                if (!base || cols <= 0 || !(cols & 63)) return;
                for (int y = 0; y < rows; ++y) { uint64_t* w = (uint64_t*)((char*)base + y * ld) + (cols >> 6); *w &= (1ull << (cols & 63)) - 1; }
            };
            pad(J.R, J.ldR, r, n - r); pad(J.M, J.ldM, r, r); pad(J.K, J.ldK, m - r, r);
        }
    }
    return cudaSuccess;
}
void write_i64(const Launch&, int64_t* dst, const int32_t* src, int64_t count, int64_t offset) { for (int64_t t = 0; t < count; ++t) dst[t] = src[t] + offset; }
}
