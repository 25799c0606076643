// Internal declarations of libgfe (not part of the C ABI).
//
// Element storage inside the library ("codec"): the tensor-core operand
// encoding of the centred residue c in [-(p-1)/2, (p-1)/2]:
//   CODEC_F8   p <= 31 : one e4m3 byte (|c| <= 15 is exact in e4m3)
//   CODEC_BF16 p <= 251: one bf16 (|c| <= 125 is exact in bf16)
// so the tcgen05 multiply-add reads operands straight from HBM.  Zero is the
// all-zero bit pattern in both.  This is the floating-point representation
// of field elements the paper mentions as prior art (Section 1), with the
// reduction mod p done exactly on integer accumulators.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

namespace gfe {

enum Codec { CODEC_F8 = 0, CODEC_BF16 = 1 };
// e4m3 for p <= 31 (tcgen05 kind::f8f6f4), bf16 above (kind::f16); both
// types are accepted by the tensor cores in K-major and MN-major layout.
inline Codec codec_for(int p) { return p <= 31 ? CODEC_F8 : CODEC_BF16; }
inline int codec_bytes(Codec c) { return c == CODEC_F8 ? 1 : 2; }

// A device matrix in the internal codec: rows x cols, row-major, ld elements.
struct DMat {
    void *ptr = nullptr;
    int64_t rows = 0, cols = 0, ld = 0;
};

// Kernel kinds for the profile counters (match gfe_profile in gfe.h).
enum Kind { K_MAD_TC = 0, K_MAD_PLAIN = 1, K_ECH = 2, K_ROWS = 3, K_COLS = 4, K_COPY = 5, K_CONV = 6, K_OTHER = 7 };

struct Launch {  // per-call launch context
    cudaStream_t st = nullptr;
    int p = 0;
    Codec codec = CODEC_F8;
    int impl = 0;  // 0 tensor cores, 1 plain CUDA-core multiply-add
    // tensor-core multiply-add: 0 = one persistent CTA per SM; k > 0 = enough
    // CTAs that none takes more than k tiles, so SMs come free for other
    // (higher-priority) streams every few tiles
    int tiles_per_cta = 0;
    // the call's error word (device memory, zeroed by the call): a bounded
    // wait of the tensor-core multiply-add that gives up sets it to 1.  Each
    // call owns its word, so concurrent calls never see one another's errors.
    int *err = nullptr;
};

// ---- profiling (gfe_api.cu) ----
void prof_begin(const Launch &L, Kind k, cudaEvent_t *ev0);
void prof_end(const Launch &L, Kind k, cudaEvent_t ev0, double madds, double bytes = 0, int64_t m = 0,
              int64_t n = 0, int64_t kk = 0);
void prof_sync_point();
// A device trace slot for this launch (4 words: start, end, CTA counters),
// or null: the kernel stamps %globaltimer itself, no events are recorded
uint64_t *prof_device_slot(const Launch &L, Kind k, int64_t m, int64_t n, int64_t kk);
void prof_count(Kind k);  // count a launch timed on the device
void prof_count_sync(double wait_ms);
void prof_host_ms(double ms);
extern bool g_prof_on;

// ---- kernels (gfe_kernels.cu); all asynchronous on L.st ----
// C := W + A B (mod p); W may be null or equal C; shapes m x k, k x n.
void mad(const Launch &L, int64_t m, int64_t n, int64_t k, const void *W, int64_t ldw,
         const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc);
void mad_plain(const Launch &L, int64_t m, int64_t n, int64_t k, const void *W, int64_t ldw,
               const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc);
// tcgen05 multiply-add (gfe_mma.cu); returns false if the shape is not handled
bool mad_tc(const Launch &L, int64_t m, int64_t n, int64_t k, const void *W, int64_t ldw,
            const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc);

int64_t tc_k_chunk(int p);
// runs the bounded-wait self-test on st (with an error word of its own);
// returns 1 if the wait gave up, 0 if it completed, -1 on a CUDA error
int wait_selftest(cudaStream_t st, int64_t limit_us);
// reads a call's error word on stream st (after all work queued on st) into
// *value; the copy to pageable host memory returns once it is complete
bool read_error_word(cudaStream_t st, const int *err, int *value);

// Leaf echelonisation of H (alpha <= ECH_LEAF_ROWS, beta <= ech_leaf_cols(p)).
// info[0] = r, info[1..] = rho (r), info[1+cap..] = gamma (r), cap = ech_leaf_cols(p).
constexpr int ECH_LEAF_ROWS = 1024;
constexpr int F32_LEAF_ROWS = 256;  // the fp32 leaf for 17 <= p <= 251
// rows one leaf kernel takes for this field
inline int ech_leaf_rows(int p) { return (p == 2 || p <= 13) ? ECH_LEAF_ROWS : F32_LEAF_ROWS; }
constexpr int ECH_LEAF_COLS = 64;       // p > 2: byte rows in shared memory
constexpr int ECH_LEAF_COLS_GF2 = 256;  // p = 2: 64-bit words in registers
int ech_leaf_cols(int p);
void ech_leaf(const Launch &L, int64_t alpha, int64_t beta, const void *H, int64_t ldh,
              int32_t *info, void *M, int64_t ldm, void *K, int64_t ldk, void *R, int64_t ldr);

// Batched form for small matrices (gfe_small.cu): one launch, one CTA per
// matrix, the whole echelonisation with transformation inside the CTA.
// A job reads A in the API storage, works in place in W (m rows of ldw
// bytes: one byte per entry, or GF(2) words), and writes r, Ups, rho and
// R, M, K in the API storage (any of pcols, prows, R, M, K may be null).
constexpr int SMALL_MAX = 2048;  // rows and columns of a small matrix
constexpr int SMALL_MAX_P = 13;  // byte entries with lazy reduction: (p-1)^2 + (p-1) <= 255
// the three kernels: bytes with 3 <= p <= 13, bytes with 17 <= p <= 251, GF(2) words
enum SmallKind { SMALL_BYTES = 0, SMALL_WIDE = 1, SMALL_GF2 = 2 };
struct SmallJob {
    const void *A;
    int64_t lda;  // bytes
    void *W;
    int64_t ldw;  // bytes, a multiple of 16 (small_ldw)
    int32_t m, n, p, fmt;
    int64_t *rank, *pcols, *prows;
    void *R, *M, *K;
    int64_t ldR, ldM, ldK;  // bytes
};
// fmt: 0 = one byte per entry (odd p <= 251), 1 = GF(2) words
inline bool small_eligible(int p, int fmt, int64_t m, int64_t n) {
    if (m <= 0 || n <= 0 || m > SMALL_MAX || n > SMALL_MAX) return false;
    return fmt == 1 ? p == 2 : (fmt == 0 && p >= 3 && p <= 251);
}
inline int small_kind(int p, int fmt) { return fmt == 1 ? SMALL_GF2 : (p <= SMALL_MAX_P ? SMALL_BYTES : SMALL_WIDE); }
// workspace row pitch (bytes) of a small matrix: 16-byte vectors
inline int64_t small_ldw(int fmt, int64_t n) { return fmt == 1 ? (n + 127) / 128 * 16 : (n + 15) / 16 * 16; }
// one persistent launch for count jobs of one kind (SmallKind): a CTA per SM
// takes jobs in table order through the device counter *next (zeroed here)
cudaError_t ech_small_batch(const Launch &L, const SmallJob *jobs_dev, int count, int kind, int *next);

// An index array for a gather: a device copy, or, when it has at most
// MAP_INLINE entries, the host array itself, which is then passed by value
// with the launch (no separate upload on the stream).
constexpr int MAP_INLINE = 2048;
struct IdxMap {
    const int32_t *dev = nullptr;   // device array (any length)
    const int32_t *host = nullptr;  // host array, n <= MAP_INLINE (takes precedence)
    int64_t n = 0;
};

// dst row t = map[t] >= 0 ? A row map[t] : B row (-1 - map[t])   (B may be null if unused)
void gather_rows(const Launch &L, int64_t nrows, int64_t ncols, void *dst, int64_t ldd,
                 const void *A, int64_t lda, const void *B, int64_t ldb, const IdxMap &map);
// dst col t = map[t] >= 0 ? src col map[t] : 0
void gather_cols(const Launch &L, int64_t nrows, int64_t ncols, void *dst, int64_t ldd,
                 const void *src, int64_t lds, const IdxMap &map);
// dst[t][c] = map[c] >= 0 ? rows[t][map[c]] : 0, rows[] a device array of row
// start pointers (gathers from several matrices in one launch)
void gather_rowptr(const Launch &L, int64_t nrows, int64_t ncols, void *dst, int64_t ldd,
                   const uint64_t *rows, const int32_t *map);
// V[t][pos[t]] := 1 for t < count (job ADI)
void set_ones(const Launch &L, int64_t count, void *V, int64_t ldv, const IdxMap &pos);
void copy2d(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd,
            const void *src, int64_t lds);
void zero2d(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd);

// conversions between the API storage and the codec
void import_u8(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd,
               const uint8_t *src, int64_t lds);
void import_bits(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd,
                 const uint64_t *src, int64_t ldw);
void export_u8(const Launch &L, int64_t rows, int64_t cols, uint8_t *dst, int64_t ldd,
               const void *src, int64_t lds);
void export_bits(const Launch &L, int64_t rows, int64_t cols, uint64_t *dst, int64_t ldw,
                 const void *src, int64_t lds);
// dense E: colmap[c] = l (pivot l) or -1-j (non-pivot j); rows >= r zero.
void build_E(const Launch &L, int fmt, int64_t m, int64_t n, int64_t r, void *dst, int64_t ldd,
             const void *R, int64_t ldr, const int32_t *colmap);
// dense T: rowmap[x] = s (x = rho_s) or -1-t (x = rho_bar_t).
void build_T(const Launch &L, int fmt, int64_t m, int64_t r, void *dst, int64_t ldd,
             const void *M, int64_t ldm, const void *K, int64_t ldk, const int32_t *rowmap);
void write_i64(const Launch &L, int64_t *dst, const int32_t *src, int64_t count, int64_t offset);
// *flag := 1 if A (rows x cols, codec entries) has a non-zero entry; flag is
// left alone otherwise (the caller zeroes it first)
void any_nonzero(const Launch &L, int64_t rows, int64_t cols, const void *A, int64_t lda, int32_t *flag);

// ---- the planner (gfe_chief.cu) ----
struct TopResult {
    int64_t r = 0;
    std::vector<int32_t> rho, gamma;
};
// Runs the method on the internal matrix H (destroyed).  Mo, Ko, Ro receive
// M (min x min), K (m x min), R (min x n) in the codec.  dry = only size the
// workspace (peak bytes from base_used).
void run_chief(const Launch &L, char *ws, size_t ws_bytes, bool dry, const DMat &H, bool trafo, bool wantR,
               const DMat &Mo, const DMat &Ko, const DMat &Ro, TopResult &res, size_t *peak, size_t base_used,
               int64_t *syncs);

extern int64_t g_block_threshold, g_block_big, g_leaf_rows;
extern int g_side_tiles;
// A host thread that set g_wait_event (a cudaEventBlockingSync event) sleeps
// in its waits for the GPU instead of spinning: the batched form runs more
// workers than the host has cores.  host_wait(s) waits for stream s either way.
extern thread_local cudaEvent_t g_wait_event;
cudaError_t host_wait(cudaStream_t s);
int64_t auto_leaf_rows(int p, int64_t m, int64_t n);
int64_t auto_block(int p, int64_t m, int64_t n);

// ---- error state and argument checks (gfe_api.cu) ----
void set_error(const std::string &s);
bool field_ok(int p);  // p is a prime <= 251
bool cuda_ok(cudaError_t e, const char *what);

}  // namespace gfe
