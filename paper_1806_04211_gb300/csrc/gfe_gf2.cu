// Bit-packed GF(2) block multiply-add, job MAD of Section 4.1 over GF(2):
//   C := W + A B,  A m x k, B k x n, W and C m x n, rows of 64-bit words
//   (bit c % 64 of word c / 64 is column c, LSB first).
// Over GF(2) a multiply is AND and an add is XOR, so a row of C is the XOR
// of the rows of B selected by the set bits of the row of A.
//
// Method of the Four Russians (Arlazarov, Dinic, Kronrod, Faradzev 1970; in
// the form of "M4RM", Albrecht, Bard, Hart 2010): for every 8 consecutive
// rows of B (a "slice" of k), a table of all 256 XOR combinations of those
// rows is built once in shared memory; each row of A then adds ONE table
// entry per slice, picked by its 8 bits there.  This does 1/8 of the XORs
// of the row-by-row product and reads operands from shared memory with
// 128-bit loads.
//
// CTA tile: 512 rows x 16 words (1024 columns) of C, 256 threads.  A thread
// owns 16 consecutive rows x 2 words (one uint4) in registers.  Per 64-bit
// chunk of k: A's 64 bits of every tile row are stored transposed in shared
// memory (byte s of each row contiguous over rows), the chunk's 64 rows of B
// beside them; then 8 slices, each: build the next slice's table (double
// buffered) and look the current one up for every row.  Products too small
// to fill the GPU split k across CTAs, which XOR their partial tiles into C
// atomically after C has been set to W.
#include "gfe.h"
#include "gfe_internal.h"

#include <algorithm>
#include <string>

namespace gfe {
namespace {

constexpr int G_BM = 512;         // rows of a tile
constexpr int G_BW = 16;          // 64-bit words of a tile row
constexpr int G_THREADS = 256;
constexpr int G_ROWS = 16;        // rows per thread
constexpr int G_SMEM = 2 * 256 * G_BW * 8 + 64 * G_BW * 8 + 8 * G_BM;  // tables, B chunk, A bytes

__device__ __forceinline__ void xor4(uint4 &a, const uint4 &b) {
    a.x ^= b.x;
    a.y ^= b.y;
    a.z ^= b.z;
    a.w ^= b.w;
}

// the 8 table entries h5 * 8 + l (l = 0..7) of word column w: entry e is the
// XOR of the slice's B rows b with bit b of e set
__device__ __forceinline__ void build_entries(uint64_t *T, const uint64_t *Bs, int slice, int w, int h5) {
    const uint64_t *b = Bs + (size_t)(8 * slice) * G_BW + w;
    uint64_t base = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if ((h5 >> q) & 1) base ^= b[(3 + q) * G_BW];
    const uint64_t b0 = b[0], b1 = b[G_BW], b2 = b[2 * G_BW];
    uint64_t *t = T + (size_t)(h5 * 8) * G_BW + w;
    const uint64_t v2 = base ^ b1, v4 = base ^ b2, v6 = v4 ^ b1;
    t[0 * G_BW] = base;
    t[1 * G_BW] = base ^ b0;
    t[2 * G_BW] = v2;
    t[3 * G_BW] = v2 ^ b0;
    t[4 * G_BW] = v4;
    t[5 * G_BW] = v4 ^ b0;
    t[6 * G_BW] = v6;
    t[7 * G_BW] = v6 ^ b0;
}

// grid: (row tiles, word tiles, k splits); `split` = 64-bit chunks of k per
// split; atomic = partial tiles are XORed into C (C already holds W)
__global__ void __launch_bounds__(G_THREADS, 1)
    k_mad_gf2(int64_t m, int64_t nw, int64_t k, const uint64_t *__restrict__ W, int64_t ldw,
              const uint64_t *__restrict__ A, int64_t lda, const uint64_t *__restrict__ B, int64_t ldb,
              uint64_t *C, int64_t ldc, int64_t split, bool atomic, uint64_t lastmask) {
    extern __shared__ __align__(16) unsigned char g2_smem[];
    uint64_t *Tb = (uint64_t *)g2_smem;                 // [2][256][G_BW]
    uint64_t *Bs = Tb + 2 * 256 * G_BW;                 // [64][G_BW]
    uint8_t *As = (uint8_t *)(Bs + 64 * G_BW);          // [8][G_BM]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = lane & 7, g = lane >> 3;
    const int rbase = warp * 64 + g * 16;
    const int64_t m0 = (int64_t)blockIdx.x * G_BM, w0 = (int64_t)blockIdx.y * G_BW;
    const int64_t kchunks = (k + 63) / 64;
    const int64_t ch0 = (int64_t)blockIdx.z * split, ch1 = min(kchunks, ch0 + split);
    uint4 acc[G_ROWS];
#pragma unroll
    for (int j = 0; j < G_ROWS; ++j) acc[j] = make_uint4(0, 0, 0, 0);
    // table-build items: word column bw, high 5 bits bh and bh + 16
    const int bw = tid & 15, bh = tid >> 4;
    for (int64_t ch = ch0; ch < ch1; ++ch) {
        __syncthreads();  // the previous chunk's readers are done with As, Bs and the tables
        const int64_t kc0 = ch * 64;
        const uint64_t kmask = (k - kc0 >= 64) ? ~0ull : ((1ull << (k - kc0)) - 1ull);
#pragma unroll
        for (int q = 0; q < G_BM / G_THREADS; ++q) {
            const int row = tid + q * G_THREADS;
            const uint64_t a = (m0 + row < m) ? (A[(m0 + row) * lda + ch] & kmask) : 0ull;
#pragma unroll
            for (int s = 0; s < 8; ++s) As[s * G_BM + row] = (uint8_t)(a >> (8 * s));
        }
#pragma unroll
        for (int q = 0; q < 64 * G_BW / G_THREADS; ++q) {
            const int i = tid + q * G_THREADS, row = i / G_BW, w = i % G_BW;
            Bs[i] = (kc0 + row < k && w0 + w < nw) ? B[(kc0 + row) * ldb + w0 + w] : 0ull;
        }
        __syncthreads();
        build_entries(Tb, Bs, 0, bw, bh);
        build_entries(Tb, Bs, 0, bw, bh + 16);
        for (int s = 0; s < 8; ++s) {
            __syncthreads();  // table s complete; table s+1's buffer free
            if (s < 7) {
                build_entries(Tb + ((s + 1) & 1) * 256 * G_BW, Bs, s + 1, bw, bh);
                build_entries(Tb + ((s + 1) & 1) * 256 * G_BW, Bs, s + 1, bw, bh + 16);
            }
            const uint64_t *T = Tb + (s & 1) * 256 * G_BW;
            const uint4 ab = *(const uint4 *)(As + s * G_BM + rbase);
            const uint32_t aw[4] = {ab.x, ab.y, ab.z, ab.w};
#pragma unroll
            for (int j = 0; j < G_ROWS; ++j) {
                const uint32_t byte = (aw[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                xor4(acc[j], *(const uint4 *)(T + byte * G_BW + 2 * c));
            }
        }
    }
    // epilogue: C = W ^ acc, or C ^= acc (split k); pad bits beyond n stay 0
#pragma unroll
    for (int j = 0; j < G_ROWS; ++j) {
        const int64_t row = m0 + rbase + j;
        if (row >= m) continue;
        uint64_t v[2] = {((uint64_t)acc[j].y << 32) | acc[j].x, ((uint64_t)acc[j].w << 32) | acc[j].z};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t w = w0 + 2 * c + h;
            if (w >= nw) continue;
            uint64_t x = v[h];
            if (w == nw - 1) x &= lastmask;
            if (atomic) {
                if (x) atomicXor((unsigned long long *)&C[row * ldc + w], (unsigned long long)x);
            } else {
                uint64_t o = W ? W[row * ldw + w] : 0ull;
                if (w == nw - 1) o &= lastmask;
                C[row * ldc + w] = o ^ x;
            }
        }
    }
}

// C rows := W rows (or 0), pad bits of the last word cleared
__global__ void k_set_gf2(int64_t m, int64_t nw, const uint64_t *W, int64_t ldw, uint64_t *C, int64_t ldc,
                          uint64_t lastmask) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m * nw) return;
    const int64_t row = i / nw, w = i % nw;
    uint64_t v = W ? W[row * ldw + w] : 0ull;
    if (w == nw - 1) v &= lastmask;
    C[row * ldc + w] = v;
}

// ---- peak probes: LOP3 issue rate and 128-bit shared-memory load rate ----
// every thread runs 8 independent (a & b) ^ c chains of `iters` steps
__global__ void k_lop3_probe(int iters, uint32_t seed, uint32_t *out) {
    uint32_t a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = seed * (threadIdx.x + 1) + q;
    const uint32_t b = seed ^ 0x5bd1e995u, c = seed + blockIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x6A;" : "+r"(a[q]) : "r"(b), "r"(c));  // (a & b) ^ c
    }
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s ^= a[q];
    if (s == 0x12345678u) out[blockIdx.x] = s;  // keeps the chains live
}

// every thread reads `iters` x 8 uint4 from a conflict-free 16 KB pattern
__global__ void k_lds_probe(int iters, uint32_t *out) {
    __shared__ uint4 buf[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) buf[i] = make_uint4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    uint4 acc = make_uint4(0, 0, 0, 0);
    int idx = threadIdx.x & 1023;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint4 v = buf[(idx + 128 * q) & 1023];
            xor4(acc, v);
        }
        idx = (idx + 32) & 1023;
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x12345678u) out[blockIdx.x] = acc.x;
}

bool g_gf2_attr[64] = {};

}  // namespace
}  // namespace gfe

using namespace gfe;

extern "C" {

gfe_status gfe_mad_gf2(int64_t m, int64_t n, int64_t k, const uint64_t *W, int64_t ldw, const uint64_t *A,
                       int64_t lda, const uint64_t *B, int64_t ldb, uint64_t *C, int64_t ldc, void *stream) {
    if (m < 0 || n < 0 || k < 0) return (set_error("negative size"), GFE_EINVAL);
    if (m == 0 || n == 0) return GFE_OK;
    const int64_t nw = (n + 63) / 64, kw = (k + 63) / 64;
    if (!C || ldc % 8 || ldc < 8 * nw || (W && (ldw % 8 || ldw < 8 * nw)) ||
        (k > 0 && (!A || !B || lda % 8 || lda < 8 * kw || ldb % 8 || ldb < 8 * nw)))
        return (set_error("gfe_mad_gf2: bad matrix argument (ld in bytes, a multiple of 8, >= a row)"), GFE_EINVAL);
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return GFE_ECUDA;
    if (dev >= 0 && dev < 64 && !g_gf2_attr[dev]) {
        if (!cuda_ok(cudaFuncSetAttribute(k_mad_gf2, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM), "attribute"))
            return GFE_ECUDA;
        g_gf2_attr[dev] = true;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t lastmask = (n % 64) ? ((1ull << (n % 64)) - 1ull) : ~0ull;
    const int64_t tm = (m + G_BM - 1) / G_BM, tn = (nw + G_BW - 1) / G_BW, tiles = tm * tn;
    // split k when the tiles alone would leave SMs idle (one CTA per SM)
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(kw, (sms + tiles - 1) / tiles));
    const int64_t per = (kw + splits - 1) / std::max<int64_t>(splits, 1);
    splits = kw ? (kw + per - 1) / per : 1;
    const bool atomic = splits > 1;
    if (tm > 65535 * 32 || tn > 65535 || splits > 65535) return (set_error("gfe_mad_gf2: too large"), GFE_EINVAL);
    const uint64_t *Wl = W;
    if (atomic || k == 0) {
        if (!(W == C && ldw == ldc)) {
            const int64_t cnt = m * nw;
            k_set_gf2<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(m, nw, W, ldw / 8, C, ldc / 8, lastmask);
        }
        if (k == 0) return cuda_ok(cudaGetLastError(), "gfe_mad_gf2 launch") ? GFE_OK : GFE_ECUDA;
        Wl = nullptr;
    }
    dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)splits);
    k_mad_gf2<<<grid, G_THREADS, G_SMEM, st>>>(m, nw, k, Wl, ldw / 8, A, lda / 8, B, ldb / 8, C, ldc / 8, per,
                                               atomic, lastmask);
    return cuda_ok(cudaGetLastError(), "gfe_mad_gf2 launch") ? GFE_OK : GFE_ECUDA;
}

gfe_status gfe_gf2_peaks(double *lop3_per_s, double *lds_bytes_per_s, void *stream) {
    if (!lop3_per_s || !lds_bytes_per_s) return (set_error("gfe_gf2_peaks: NULL output"), GFE_EINVAL);
    int dev = 0, sms = 148;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return GFE_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *sink = nullptr;
    if (!cuda_ok(cudaMalloc(&sink, 4 * 64 * (size_t)sms), "cudaMalloc")) return GFE_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = 8 * sms, threads = 512;
    float ms = 0.f, best = 1e30f;
    const int it1 = 1 << 14;
    for (int rep = 0; rep < 4; ++rep) {  // first launch warms up; best of the rest
        cudaEventRecord(e0, st);
        k_lop3_probe<<<blocks, threads, 0, st>>>(it1, 0x9e3779b9u + rep, sink);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) best = std::min(best, ms);
    }
    *lop3_per_s = (double)blocks * threads * it1 * 8.0 / (best * 1e-3);
    best = 1e30f;
    const int it2 = 1 << 12;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        k_lds_probe<<<blocks, threads, 0, st>>>(it2, sink);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) best = std::min(best, ms);
    }
    *lds_bytes_per_s = (double)blocks * threads * it2 * 8.0 * 16.0 / (best * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return cuda_ok(cudaGetLastError(), "peak probes") ? GFE_OK : GFE_ECUDA;
}

}  // extern "C"
