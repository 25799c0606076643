// Job kernels of libgfe on CUDA cores: the plain multiply-add (job MAD/MUL),
// the leaf echelonisation (job ECH), extracts and riffles (CEX, REX, RRF,
// CRZ, ADI) and the conversions at the API boundary.
// Jobs: arXiv 1806.04211, Section 4.1.
#include "gfe_internal.h"

#include <cstring>
#include <type_traits>

#include <climits>
#include <cuda_fp16.h>
#include <mutex>

namespace gfe {

// ---------------------------------------------------------------------------
// codecs (see gfe_internal.h)
// ---------------------------------------------------------------------------
template <int C> struct Cd;

// e4m3: sign | 4-bit exponent (bias 7) | 3-bit mantissa.  Only integers with
// |c| <= 15 are ever stored, all exact: c = 1.m * 2^(e-7) with e in [7,10].
template <> struct Cd<CODEC_F8> {
    using T = uint8_t;
    __device__ __forceinline__ static int dec(T b) {
        int mag = b & 0x7F;
        if (mag < 0x38) return 0;  // only +-0 is stored below 1.0
        int e = mag >> 3, mt = mag & 7;
        int v = ((8 + mt) << (e - 7)) >> 3;
        return (b & 0x80) ? -v : v;
    }
    __device__ __forceinline__ static T enc(int c) {
        if (c == 0) return 0;
        int s = c < 0, a = s ? -c : c;
        int e = 31 - __clz(a);
        int mt = ((a << 3) >> e) - 8;
        return (T)((s << 7) | ((e + 7) << 3) | mt);
    }
};

// bf16: the upper half of the float32; integers |c| <= 256 are exact.
template <> struct Cd<CODEC_BF16> {
    using T = uint16_t;
    __device__ __forceinline__ static int dec(T b) { return (int)__uint_as_float((uint32_t)b << 16); }
    __device__ __forceinline__ static T enc(int c) { return (T)(__float_as_uint((float)c) >> 16); }
};

__device__ __forceinline__ int cen(int r, int p) { return r > (p >> 1) ? r - p : r; }
__device__ __forceinline__ int res(int c, int p) { return c < 0 ? c + p : c; }
__device__ __forceinline__ int modp(int x, int p) {
    int r = x % p;
    return r < 0 ? r + p : r;
}

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// plain multiply-add  C := W + A B  (mod p)   -- the CUDA-core comparator
// 64 x 64 tile per CTA, 256 threads, 4 x 4 outputs per thread, int32
// accumulation of centred products (|c| <= 125): exact for k <= 2^17.
// ---------------------------------------------------------------------------
constexpr int PT = 64, PK = 16;

template <int C>
__global__ void __launch_bounds__(256) k_mad_plain(int p, int M, int N, int K,
                                                    const typename Cd<C>::T *W, int64_t ldw,
                                                    const typename Cd<C>::T *A, int64_t lda,
                                                    const typename Cd<C>::T *B, int64_t ldb,
                                                    typename Cd<C>::T *Cm, int64_t ldc) {
    using D = Cd<C>;
    __shared__ int As[PK][PT + 1];
    __shared__ int Bs[PK][PT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * PT, n0 = blockIdx.x * PT;
    int acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int k0 = 0; k0 < K; k0 += PK) {
        for (int t = threadIdx.x; t < PT * PK; t += 256) {
            int mm = t / PK, kk = t % PK, gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? D::dec(A[(int64_t)gm * lda + gk]) : 0;
            int kk2 = t / PT, nn = t % PT, gk2 = k0 + kk2, gn = n0 + nn;
            Bs[kk2][nn] = (gk2 < K && gn < N) ? D::dec(B[(int64_t)gk2 * ldb + gn]) : 0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < PK; ++kk) {
            int a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            int v = acc[i][j] % p;
            if (W) v += D::dec(W[(int64_t)gm * ldw + gn]);
            Cm[(int64_t)gm * ldc + gn] = D::enc(cen(modp(v, p), p));
        }
    }
}

void mad_plain(const Launch &L, int64_t m, int64_t n, int64_t k, const void *W, int64_t ldw,
               const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc) {
    if (m <= 0 || n <= 0) return;
    if (k <= 0) {  // C := W (or 0)
        if (!W) zero2d(L, m, n, C, ldc);
        else if (W != C) copy2d(L, m, n, C, ldc, W, ldw);
        return;
    }
    const int64_t KMAX = 1 << 17;
    const int es = codec_bytes(L.codec);
    for (int64_t k0 = 0; k0 < k; k0 += KMAX) {
        int64_t kk = k - k0 < KMAX ? k - k0 : KMAX;
        const char *Ak = (const char *)A + k0 * es;
        const char *Bk = (const char *)B + k0 * ldb * es;
        const void *Wk = k0 ? C : W;
        int64_t ldwk = k0 ? ldc : ldw;
        dim3 grid(cdiv(n, PT), cdiv(m, PT));
        cudaEvent_t ev;
        prof_begin(L, K_MAD_PLAIN, &ev);
        if (L.codec == CODEC_F8)
            k_mad_plain<CODEC_F8><<<grid, 256, 0, L.st>>>(L.p, (int)m, (int)n, (int)kk,
                (const uint8_t *)Wk, ldwk, (const uint8_t *)Ak, lda, (const uint8_t *)Bk, ldb,
                (uint8_t *)C, ldc);
        else
            k_mad_plain<CODEC_BF16><<<grid, 256, 0, L.st>>>(L.p, (int)m, (int)n, (int)kk,
                (const uint16_t *)Wk, ldwk, (const uint16_t *)Ak, lda, (const uint16_t *)Bk, ldb,
                (uint16_t *)C, ldc);
        prof_end(L, K_MAD_PLAIN, ev, (double)m * (double)n * (double)kk, 0, m, n, kk);
    }
}

void mad(const Launch &L, int64_t m, int64_t n, int64_t k, const void *W, int64_t ldw,
         const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc) {
    if (m <= 0 || n <= 0) return;
    if (L.impl == 0 && k > 0 && mad_tc(L, m, n, k, W, ldw, A, lda, B, ldb, C, ldc)) return;
    mad_plain(L, m, n, k, W, ldw, A, lda, B, ldb, C, ldc);
}

// ---------------------------------------------------------------------------
// leaf echelonisation (job ECH, Remark "echelon") of H: alpha x beta with
// beta <= 64 (256 for GF(2)), one CTA, one thread per row.  Column-by-column
// Gauss-Jordan; the pivot of column c is the topmost non-pivot row with a
// non-zero entry there, which yields the row rank profile and the column
// rank profile, i.e. the unique result of Eq. (gauss).  The transformation
// is kept in "slot" space: slot t = the t-th pivot found (= the t-th pivot
// column), so each row carries <= 64 (GF(2): 256) coefficients.
// ---------------------------------------------------------------------------
constexpr int LS = 68;  // smem row stride (bytes): 17 words -> conflict-free rows

// column c's place among the non-pivot columns: slotCol holds the r pivot
// columns in ascending order (pivots are found column by column)
__device__ __forceinline__ void place_non_pivot(const int16_t *slotCol, int r, int c, int16_t *nonCol) {
    int lo = 0, hi = r;  // first index with slotCol[] >= c
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (slotCol[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= r || slotCol[lo] != c) nonCol[c - lo] = (int16_t)c;
}

// x mod p for an integer-valued float 0 <= x < 2^24 with x / p < 2^20.
// The quotient x / p is rounded to the nearest integer by adding and
// subtracting 1.5 * 2^23 (FMA-pipe arithmetic, no conversion instruction);
// it is within one of the true quotient, so the remainder, formed exactly by
// an fma, needs one correction.  Checked against integer x mod p for every
// prime 17 <= p <= 251 and every x < 2^24, and for p <= 13 over the values a
// leaf reaches (below 64 p^2 + p), with and without the multiply and add
// contracted into one fma.
__device__ __forceinline__ float fred(float x, float p, float invp) {
    const float q = __fadd_rn(fmaf(x, invp, 12582912.0f), -12582912.0f);
    const float r = fmaf(-q, p, x);
    return r < 0.f ? r + p : r;
}

// ---------------------------------------------------------------------------
// leaf ECH of at most 256 rows for p > 2 (every leaf of 17 <= p <= 251; the
// byte leaf below takes the larger ones of p <= 13): the same
// column-by-column Gauss-Jordan and topmost-row rule.  A row's 64 entries
// and 64 slot coefficients are fp32 integers in shared memory (row y at
// Rw[y], columns then slots); columns are taken eight at a time:
//  (A) the panel: every row's eight entries in the group's columns, reduced
//      (written by the previous group's (D), else read from the rows);
//  (B) the finder: the first half of the threads, one row per lane, runs the
//      column-by-column elimination on the panel alone, one named barrier per
//      column: each warp's topmost candidate publishes its reduced entries
//      and the scale that makes its pivot -1, every row takes the new pivot
//      row from the winner, and records the multiple G[y][s] of the new pivot
//      row s added to it (one 64-bit word per row).  Then NP[s], the pivot
//      row s as a combination of the rows Q_0 .. Q_s, Q_s being row x_s as
//      it stood at the group start plus the identity of its slot;
//  (C) warp s publishes Q_s, reduced, and row x_s restarts from zero; every
//      row forms its coefficients CM_y = G[y] NP;
//  (D) rows += CM Q, i.e. row y becomes [y is no pivot of the group] * y +
//      sum_s CM_y[s] Q_s, on the tensor cores (mma.sync m16n8k8 with tf32
//      operands), over the columns from the group on and the slots up to its
//      last.
// Rows are linear in the rows they were built from, so (D) reproduces the
// column-by-column result; three block barriers per group.  Entries start
// below p and grow by less than p^2 per pivot, so after the at most 64
// pivots of a leaf they stay below 64 p^2 + p < 2^24: exact in fp32, and no
// row is reduced before the end.  At most F32_LEAF_ROWS rows.
// ---------------------------------------------------------------------------
constexpr int F32_THREADS = 2 * F32_LEAF_ROWS;
constexpr int F32_RS = 136;  // row stride of Rw and Q (floats): the tensor-core fragments fall in distinct banks
// dynamic shared memory of k_ech_leaf_f32 for rows_cap rows: the rows, then the byte
// staging of the load phase
inline int f32_leaf_smem(int rows_cap) { return rows_cap * F32_RS * 4 + rows_cap * LS; }

struct InvTable {
    uint8_t v[256];  // v[x] = x^-1 mod p (v[0] = 0)
};

template <int C>
__global__ void __launch_bounds__(F32_THREADS, 1) k_ech_leaf_f32(const __grid_constant__ InvTable it, int p,
                                                              int alpha, int beta,
                                                              const typename Cd<C>::T *H, int64_t ldh,
                                                              int32_t *info, typename Cd<C>::T *Mo,
                                                              int64_t ldm, typename Cd<C>::T *Ko,
                                                              int64_t ldk, typename Cd<C>::T *Ro,
                                                              int64_t ldr) {
    using D = Cd<C>;
    extern __shared__ __align__(16) uint8_t sm[];
    const int rows_cap = blockDim.x >> 1;        // a multiple of 32
    float *Rw = (float *)sm;                     // [rows_cap][F32_RS]  the rows
    uint8_t *S = sm + rows_cap * F32_RS * 4;     // [rows_cap][LS]  residues of H (load)
    __shared__ uint8_t inv[256];
    __shared__ uint8_t piv[F32_LEAF_ROWS];
    __shared__ int16_t slotOf[F32_LEAF_ROWS];
    __shared__ int16_t pivpos[F32_LEAF_ROWS];
    __shared__ int16_t slotRow[64], slotCol[64], sortedSlot[64], nonCol[64];
    __shared__ float panel[F32_LEAF_ROWS][9];    // the group's eight columns, reduced
    __shared__ uint64_t Gm[F32_LEAF_ROWS];       // G[y][s] in byte s
    __shared__ __align__(16) float NP[8][8];     // NP[s][s'] (zero for s' > s)
    __shared__ __align__(16) float Q[8][F32_RS]; // Q_s: 64 columns, then 64 slots
    __shared__ __align__(16) float CMs[F32_LEAF_ROWS][12];  // CM_y (stride 12: distinct banks)
    __shared__ float cbuf[2][F32_LEAF_ROWS / 32][8];  // per warp: its topmost candidate's panel entries,
    __shared__ uint64_t cgw[2][F32_LEAF_ROWS / 32];    // its multiples so far,
    __shared__ float csc[2][F32_LEAF_ROWS / 32];       // the scale that makes its pivot -1
    __shared__ uint64_t pgx[8];                        // per pivot s of the group: the multiples of x_s,
    __shared__ float psc[8];                           // and its scale
    __shared__ int wmin[2][F32_LEAF_ROWS / 32];        // and its row
    __shared__ int gnp;                          // pivots in the group
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int hf = tid >= rows_cap ? 1 : 0, y = tid - hf * rows_cap;  // half, row
    const float fp = (float)p, invp = 1.0f / (float)p;
    float *row = Rw + y * F32_RS + 32 * hf;      // this thread's 32 columns; its slots at + 64

    for (int q = tid; q < 256; q += blockDim.x) inv[q] = it.v[q];
    for (int q = tid; q < 8 * F32_RS; q += blockDim.x) Q[q / F32_RS][q % F32_RS] = 0.f;
    if (hf == 0) {
        piv[y] = 0;
        slotOf[y] = -1;
    }
    // warp w loads rows 16 w .. 16 w + 15 (lane l: entries l and 32 + l)
#pragma unroll 8
    for (int rr = 0; rr < 16; ++rr) {
        const int r = warp * 16 + rr;
        const typename D::T *hr = H + (int64_t)r * ldh;
        const bool in = r < alpha;
        S[r * LS + lane] = in && lane < beta ? (uint8_t)res(D::dec(hr[lane]), p) : 0;
        S[r * LS + 32 + lane] = in && 32 + lane < beta ? (uint8_t)res(D::dec(hr[32 + lane]), p) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; k += 4) {
        const uint32_t w = *(const uint32_t *)(S + y * LS + 32 * hf + k);
        *(float4 *)(row + k) = make_float4((float)(w & 0xFF), (float)((w >> 8) & 0xFF), (float)((w >> 16) & 0xFF),
                                           (float)(w >> 24));
        *(float4 *)(row + 64 + k) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    int ns = 0;          // pivots before the group
    bool fresh = true;   // the panel is to be read from the rows
    const int ngroups = (beta + 7) >> 3;
    for (int g = 0; g < ngroups; ++g) {
        const int c0 = 8 * g;
        // (A) the panel: the half that holds columns c0 .. c0 + 7, unless the
        // previous group's (D) has written it
        if (fresh && hf == (c0 >> 5)) {
            const float4 a = *(const float4 *)(row + (c0 & 31)), b = *(const float4 *)(row + (c0 & 31) + 4);
            panel[y][0] = fred(a.x, fp, invp);
            panel[y][1] = fred(a.y, fp, invp);
            panel[y][2] = fred(a.z, fp, invp);
            panel[y][3] = fred(a.w, fp, invp);
            panel[y][4] = fred(b.x, fp, invp);
            panel[y][5] = fred(b.y, fp, invp);
            panel[y][6] = fred(b.z, fp, invp);
            panel[y][7] = fred(b.w, fp, invp);
        }
        __syncthreads();
        // (B) the finder: the half-0 warps, one row per lane, one named
        // barrier per column.  Each warp's topmost candidate publishes its
        // reduced entries and the scale that makes its pivot -1 before the
        // barrier; after it every row takes the new pivot row from the winner.
        if (hf == 0) {
            float pan[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) pan[k] = panel[y][k];
            bool cand = y < alpha && !piv[y];
            uint64_t gw = 0;  // G[y][s] in byte s
            int s = 0;
            // one column per pass, the current one always in pan[0] (a short
            // loop body: the finder runs once per group and its code is fetched
            // each time)
#pragma unroll 1
            for (int k = 0; k < 8; ++k) {
                const int b = k & 1;
                const float v = fred(pan[0], fp, invp);
                const bool c = c0 + k < beta && cand && v != 0.f;
                const unsigned bal = __ballot_sync(0xffffffffu, c);
                if (bal && lane == __ffs(bal) - 1) {  // this warp's topmost candidate
#pragma unroll
                    for (int j = 1; j < 8; ++j) cbuf[b][warp][j] = fred(pan[j], fp, invp);
                    cgw[b][warp] = gw;
                    csc[b][warp] = (float)(p - inv[(int)v]);
                }
                if (lane == 0) wmin[b][warp] = bal ? y + __ffs(bal) - 1 : INT_MAX;
                asm volatile("bar.sync 1, %0;" ::"r"(rows_cap) : "memory");
                const int x = (int)__reduce_min_sync(0xffffffffu, (unsigned)(lane < (rows_cap >> 5) ? wmin[b][lane]
                                                                                                    : INT_MAX));
                if (x != INT_MAX) {  // uniform: else column c0 + k has no pivot
                    const int xw = x >> 5;
                    const float sc = csc[b][xw];
                    // the new pivot row's entries: lane j computes entry j & 7
                    const float npl = fred(sc * cbuf[b][xw][lane & 7], fp, invp);
                    // every other row adds its entry at column c0 + k times the new
                    // pivot row; the pivot row's earlier multiples go into NP[s]
                    const bool isx = y == x;
#pragma unroll
                    for (int j = 1; j < 8; ++j) {
                        const float nj = __shfl_sync(0xffffffffu, npl, j);
                        pan[j] = isx ? nj : fmaf(v, nj, pan[j]);
                    }
                    gw = isx ? 1ull << (8 * s) : (gw | ((uint64_t)(uint32_t)v << (8 * s)));
                    cand = cand && !isx;
                    if (tid == 0) {
                        piv[x] = 1;
                        slotOf[x] = (int16_t)(ns + s);
                        slotRow[ns + s] = (int16_t)x;
                        slotCol[ns + s] = (int16_t)(c0 + k);
                        pgx[s] = cgw[b][xw];
                        psc[s] = sc;
                    }
                    ++s;
                }
#pragma unroll
                for (int j = 1; j < 8; ++j) pan[j - 1] = pan[j];
            }
            Gm[y] = gw;
            if (tid == 0) gnp = s;
            // NP[s] = sc_s (CM_(x_s) + e_s), CM_(x_s) = sum_{s' < s} G[x_s][s'] NP[s']:
            // lane j < 8 of warp 0 forms column j
            if (warp == 0) {
                __syncwarp();
                if (lane < 8) {
                    float npc[8];
#pragma unroll
                    for (int s1 = 0; s1 < 8; ++s1) {
                        float nv = 0.f;
                        if (s1 < s) {
                            const uint64_t gx = pgx[s1];
                            float acc = 0.f;
#pragma unroll
                            for (int s2 = 0; s2 < s1; ++s2)
                                acc = fmaf((float)(uint32_t)((gx >> (8 * s2)) & 0xFF), npc[s2], acc);
                            acc = lane == s1 ? 1.f : (lane < s1 ? fred(acc, fp, invp) : 0.f);
                            nv = fred(psc[s1] * acc, fp, invp);
                        }
                        npc[s1] = nv;
                        NP[s1][lane] = nv;
                    }
                }
            }
        }
        __syncthreads();
        const int nsg = gnp;
        fresh = nsg == 0;
        if (nsg == 0) continue;  // uniform
        // (C) warp s publishes Q_s from pivot row x_s, which then restarts from
        // zero; every row forms its coefficients
        for (int sq = warp; sq < nsg; sq += nwarp) {
            const int xs = slotRow[ns + sq], own = 64 + ns + sq;  // the identity of its slot
            float *rx = Rw + xs * F32_RS + 4 * lane;
            const float4 a = *(const float4 *)rx;
            *(float4 *)(Q[sq] + 4 * lane) = make_float4(
                fred(a.x, fp, invp) + (own == 4 * lane ? 1.f : 0.f), fred(a.y, fp, invp) + (own == 4 * lane + 1 ? 1.f : 0.f),
                fred(a.z, fp, invp) + (own == 4 * lane + 2 ? 1.f : 0.f), fred(a.w, fp, invp) + (own == 4 * lane + 3 ? 1.f : 0.f));
            *(float4 *)rx = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (hf == 0) {  // CM_y = G[y] NP, reduced
            const uint64_t gy = Gm[y];
            float acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll
            for (int s2 = 0; s2 < 8; ++s2) {
                if (s2 < nsg) {
                    const float gv = (float)(uint32_t)((gy >> (8 * s2)) & 0xFF);
                    const float4 a = *(const float4 *)NP[s2], b = *(const float4 *)(NP[s2] + 4);
                    acc[0] = fmaf(gv, a.x, acc[0]);
                    acc[1] = fmaf(gv, a.y, acc[1]);
                    acc[2] = fmaf(gv, a.z, acc[2]);
                    acc[3] = fmaf(gv, a.w, acc[3]);
                    acc[4] = fmaf(gv, b.x, acc[4]);
                    acc[5] = fmaf(gv, b.y, acc[5]);
                    acc[6] = fmaf(gv, b.z, acc[6]);
                    acc[7] = fmaf(gv, b.w, acc[7]);
                }
            }
            *(float4 *)CMs[y] = make_float4(fred(acc[0], fp, invp), fred(acc[1], fp, invp), fred(acc[2], fp, invp),
                                            fred(acc[3], fp, invp));
            *(float4 *)(CMs[y] + 4) = make_float4(fred(acc[4], fp, invp), fred(acc[5], fp, invp), fred(acc[6], fp, invp),
                                                  fred(acc[7], fp, invp));
        }
        __syncthreads();
        // (D) rows += CM Q on the tensor cores (mma.sync m16n8k8, tf32 operands:
        // CM and Q are residues below 2^8, exact in tf32; the rows stay below
        // 2^24, exact in the fp32 accumulator), over the 8-column tiles from
        // the group on and the 8-slot tiles up to its last slot.  Warp w takes
        // rows 16 w .. 16 w + 15; its tile of columns c0 + 8 .. c0 + 15 also
        // writes the next group's panel.
        {
            const int gid = lane >> 2, tig = lane & 3, r0 = 16 * warp;
            const int nth = 8 - g, nt = nth + ((ns + nsg + 7) >> 3);  // column tiles, all tiles
            const uint32_t a0 = __float_as_uint(CMs[r0 + gid][tig]), a1 = __float_as_uint(CMs[r0 + gid + 8][tig]),
                           a2 = __float_as_uint(CMs[r0 + gid][tig + 4]), a3 = __float_as_uint(CMs[r0 + gid + 8][tig + 4]);
#pragma unroll 4
            for (int t2 = 0; t2 < nt; ++t2) {
                const int off = t2 < nth ? 8 * (g + t2) : 64 + 8 * (t2 - nth);
                const uint32_t b0 = __float_as_uint(Q[tig][off + gid]), b1 = __float_as_uint(Q[tig + 4][off + gid]);
                float2 *c01 = (float2 *)(Rw + (r0 + gid) * F32_RS + off + 2 * tig);
                float2 *c23 = (float2 *)(Rw + (r0 + gid + 8) * F32_RS + off + 2 * tig);
                float2 u = *c01, w = *c23;
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                    "{%0, %1, %2, %3};"
                    : "+f"(u.x), "+f"(u.y), "+f"(w.x), "+f"(w.y)
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                *c01 = u;
                *c23 = w;
                if (t2 == 1 && nth > 1) {
                    panel[r0 + gid][2 * tig] = fred(u.x, fp, invp);
                    panel[r0 + gid][2 * tig + 1] = fred(u.y, fp, invp);
                    panel[r0 + gid + 8][2 * tig] = fred(w.x, fp, invp);
                    panel[r0 + gid + 8][2 * tig + 1] = fred(w.y, fp, invp);
                }
            }
        }
        ns += nsg;
    }
    __syncthreads();  // rows were last written by the warps of their tiles
    const int r = ns;
    const bool isp = piv[y] != 0;
    // rank of each row among pivot rows (ascending) and among non-pivot rows
    // (the half-0 warps count: warp w holds rows 32 w .. 32 w + 31)
    const int isp_i = (y < alpha) && isp && hf == 0;
    unsigned bal = __ballot_sync(0xffffffffu, isp_i);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    before += __popc(bal & ((1u << lane) - 1));
    if (y < alpha && hf == 0) {
        if (isp_i) {
            pivpos[y] = (int16_t)before;
            sortedSlot[before] = slotOf[y];
            info[1 + before] = y;
        } else {
            pivpos[y] = (int16_t)(y - before);
        }
    }
    if (tid == 0) info[0] = r;
    for (int c = tid; c < beta; c += blockDim.x) place_non_pivot(slotCol, r, c, nonCol);
    if (tid < r) info[1 + ECH_LEAF_COLS + tid] = slotCol[tid];
    __syncthreads();
    // the outputs, reduced and centred, straight from the rows: lane l writes
    // output columns l and l + 32 (their row entries found once)
    using T = typename D::T;
    const int nr = beta - r;
    const int sa = lane < r ? 64 + sortedSlot[lane] : -1, sb = lane + 32 < r ? 64 + sortedSlot[lane + 32] : -1;
    const int ca = lane < nr ? nonCol[lane] : -1, cb = lane + 32 < nr ? nonCol[lane + 32] : -1;
    auto put = [&](T *dst, const float *rw, int e) {
        if (e >= 0) *dst = D::enc(cen((int)fred(rw[e], fp, invp), p));
    };
    for (int l = warp; l < r; l += nwarp) {  // M and R: the pivot rows in slot order
        const float *rw = Rw + slotRow[l] * F32_RS;
        put(Mo + (int64_t)l * ldm + lane, rw, sa);
        put(Mo + (int64_t)l * ldm + lane + 32, rw, sb);
        put(Ro + (int64_t)l * ldr + lane, rw, ca);
        put(Ro + (int64_t)l * ldr + lane + 32, rw, cb);
    }
    for (int rw = warp; rw < alpha; rw += nwarp) {  // K: the other rows
        if (piv[rw]) continue;
        T *ko = Ko + (int64_t)pivpos[rw] * ldk;
        put(ko + lane, Rw + rw * F32_RS, sa);
        put(ko + lane + 32, Rw + rw * F32_RS, sb);
    }
}

// ---------------------------------------------------------------------------
// leaf ECH for 3 <= p <= 13, 257 to 1024 rows x 64 columns (smaller leaves
// take the fp32 leaf above): the same column-by-column Gauss-Jordan and
// topmost-row rule, and the same eight-column groups as the fp32 leaf, with
// the rows as residue bytes in
// shared memory (row y at Rb[y]: 64 columns, then 64 slots), reduced after
// every group:
//  (B) the finder: one row per thread, one barrier per column; each warp's
//      topmost candidate publishes its entries and the scale that makes its
//      pivot -1, every row takes the new pivot row from the winner and
//      records the multiple G[y][s] of the new pivot row s added to it.
//      Then NP[s], pivot row s as a combination of the rows Q_0 .. Q_s, Q_s
//      being row x_s as it stood at the group start plus the identity of its
//      slot;
//  (C) warp s publishes Q_s (transposed, for the tensor-core operand) and
//      row x_s restarts from zero; every row forms CM_y = G[y] NP, reduced;
//  (D) rows += CM Q on the tensor cores (mma.sync m16n8k8, fp16 operands
//      below 13, fp32 sums below 2^11: exact), reduced to bytes again, over
//      the columns from the group on and the slots up to its last.
// A group's panel is read from the rows, which are reduced: the finder's
// values stay below 8 p^2 + p during a group.  Three barriers per group plus
// one per column.
// ---------------------------------------------------------------------------
constexpr int U8_RB = 132;  // row stride of Rb (bytes): 33 words, so 32 rows fall in 32 banks

template <int C>
__global__ void __launch_bounds__(1024, 1) k_ech_leaf_u8(const __grid_constant__ InvTable it, int p, int alpha,
                                                         int beta, const typename Cd<C>::T *H, int64_t ldh,
                                                         int32_t *info, typename Cd<C>::T *Mo, int64_t ldm,
                                                         typename Cd<C>::T *Ko, int64_t ldk,
                                                         typename Cd<C>::T *Ro, int64_t ldr) {
    using D = Cd<C>;
    using T = typename D::T;
    extern __shared__ __align__(16) uint8_t sm[];
    uint8_t *Rb = sm;                             // [rows][U8_RB]  the rows
    __shared__ uint8_t inv[256];
    __shared__ uint8_t piv[1024];
    __shared__ int16_t slotOf[1024];
    __shared__ int16_t pivpos[1024];
    __shared__ int16_t slotRow[64], slotCol[64], sortedSlot[64], nonCol[64];
    __shared__ uint64_t Gm[1024];                 // G[y][s] in byte s
    __shared__ __align__(16) __half2 CMh[1024][4];    // CM_y: (CM_y[2 t], CM_y[2 t + 1]) at [y][t]
    __shared__ __align__(16) __half QT[128][8];       // Q_s[e] at [e][s]
    __shared__ __align__(16) float NP[8][8];      // NP[s][s'] (zero for s' > s)
    __shared__ float cbuf[2][32][8];              // per warp: its topmost candidate's entries,
    __shared__ uint64_t cgw[2][32];               // its multiples so far,
    __shared__ float csc[2][32];                  // the scale that makes its pivot -1
    __shared__ int wmin[2][32];                   // and its row
    __shared__ uint64_t pgx[8];                   // per pivot s of the group: the multiples of x_s,
    __shared__ float psc[8];                      // and its scale
    __shared__ int gnp;                           // pivots in the group
    __shared__ int wsum[32];
    const int y = threadIdx.x, lane = y & 31, warp = y >> 5, nwarp = blockDim.x >> 5;
    const float fp = (float)p, invp = 1.0f / (float)p;
    uint8_t *row = Rb + y * U8_RB;

    for (int q = y; q < 256; q += blockDim.x) inv[q] = it.v[q];
    for (int q = y; q < 128 * 8; q += blockDim.x) QT[q >> 3][q & 7] = __float2half_rn(0.f);
    piv[y] = 0;
    slotOf[y] = -1;
    // warp w loads rows 32 w .. 32 w + 31 (lane l: entries l and 32 + l); every
    // thread clears its own row's slots
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
        const int r = warp * 32 + rr;
        const T *hr = H + (int64_t)r * ldh;
        const bool in = r < alpha;
        Rb[r * U8_RB + lane] = in && lane < beta ? (uint8_t)res(D::dec(hr[lane]), p) : 0;
        Rb[r * U8_RB + 32 + lane] = in && 32 + lane < beta ? (uint8_t)res(D::dec(hr[32 + lane]), p) : 0;
    }
#pragma unroll
    for (int k = 64; k < 128; k += 4) *(uint32_t *)(row + k) = 0u;
    __syncthreads();

    int ns = 0;  // pivots before the group
    const int ngroups = (beta + 7) >> 3;
    for (int g = 0; g < ngroups; ++g) {
        const int c0 = 8 * g;
        // (B) the finder
        float pan[8];
        {
            const uint32_t w0 = *(const uint32_t *)(row + c0), w1 = *(const uint32_t *)(row + c0 + 4);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pan[j] = (float)((w0 >> (8 * j)) & 0xFF);
                pan[4 + j] = (float)((w1 >> (8 * j)) & 0xFF);
            }
        }
        bool cand = y < alpha && !piv[y];
        uint64_t gw = 0;  // G[y][s] in byte s
        int s = 0;
        // one column per pass, the current one always in pan[0]
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
            const int b = k & 1;
            const float v = fred(pan[0], fp, invp);
            const bool c = c0 + k < beta && cand && v != 0.f;
            const unsigned bal = __ballot_sync(0xffffffffu, c);
            if (bal && lane == __ffs(bal) - 1) {  // this warp's topmost candidate
#pragma unroll
                for (int j = 1; j < 8; ++j) cbuf[b][warp][j] = fred(pan[j], fp, invp);
                cgw[b][warp] = gw;
                csc[b][warp] = (float)(p - inv[(int)v]);
            }
            if (lane == 0) wmin[b][warp] = bal ? y + __ffs(bal) - 1 : INT_MAX;
            __syncthreads();
            const int x = (int)__reduce_min_sync(0xffffffffu, (unsigned)(lane < nwarp ? wmin[b][lane] : INT_MAX));
            if (x != INT_MAX) {  // uniform: else column c0 + k has no pivot
                const int xw = x >> 5;
                const float sc = csc[b][xw];
                // the new pivot row's entries: lane j computes entry j & 7
                const float npl = fred(sc * cbuf[b][xw][lane & 7], fp, invp);
                // every other row adds its entry at column c0 + k times the new
                // pivot row; the pivot row's earlier multiples go into NP[s]
                const bool isx = y == x;
#pragma unroll
                for (int j = 1; j < 8; ++j) {
                    const float nj = __shfl_sync(0xffffffffu, npl, j);
                    pan[j] = isx ? nj : fmaf(v, nj, pan[j]);
                }
                gw = isx ? 1ull << (8 * s) : (gw | ((uint64_t)(uint32_t)v << (8 * s)));
                cand = cand && !isx;
                if (y == 0) {
                    piv[x] = 1;
                    slotOf[x] = (int16_t)(ns + s);
                    slotRow[ns + s] = (int16_t)x;
                    slotCol[ns + s] = (int16_t)(c0 + k);
                    pgx[s] = cgw[b][xw];
                    psc[s] = sc;
                }
                ++s;
            }
#pragma unroll
            for (int j = 1; j < 8; ++j) pan[j - 1] = pan[j];
        }
        Gm[y] = gw;
        if (y == 0) gnp = s;
        // NP[s] = sc_s (CM_(x_s) + e_s), CM_(x_s) = sum_{s' < s} G[x_s][s'] NP[s']:
        // lane j < 8 of warp 0 forms column j
        if (warp == 0) {
            __syncwarp();
            if (lane < 8) {
                float npc[8];
#pragma unroll
                for (int s1 = 0; s1 < 8; ++s1) {
                    float nv = 0.f;
                    if (s1 < s) {
                        const uint64_t gx = pgx[s1];
                        float acc = 0.f;
#pragma unroll
                        for (int s2 = 0; s2 < s1; ++s2)
                            acc = fmaf((float)(uint32_t)((gx >> (8 * s2)) & 0xFF), npc[s2], acc);
                        acc = lane == s1 ? 1.f : (lane < s1 ? fred(acc, fp, invp) : 0.f);
                        nv = fred(psc[s1] * acc, fp, invp);
                    }
                    npc[s1] = nv;
                    NP[s1][lane] = nv;
                }
            }
        }
        __syncthreads();
        const int nsg = gnp;
        if (nsg == 0) continue;  // uniform
        // (C) warp s publishes Q_s (transposed) from pivot row x_s, which then
        // restarts from zero; every row forms its coefficients
        for (int sq = warp; sq < nsg; sq += nwarp) {
            const int xs = slotRow[ns + sq], own = 64 + ns + sq;  // the identity of its slot
            uint32_t *rx = (uint32_t *)(Rb + xs * U8_RB) + lane;
            uint32_t w = *rx;
            if ((own >> 2) == lane) w += 1u << (8 * (own & 3));
#pragma unroll
            for (int i = 0; i < 4; ++i) QT[4 * lane + i][sq] = __uint2half_rn((w >> (8 * i)) & 0xFF);
            *rx = 0u;
        }
        {
            const uint64_t gy = Gm[y];
            float acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll
            for (int s2 = 0; s2 < 8; ++s2) {
                if (s2 < nsg) {
                    const float gv = (float)(uint32_t)((gy >> (8 * s2)) & 0xFF);
                    const float4 a = *(const float4 *)NP[s2], b = *(const float4 *)(NP[s2] + 4);
                    acc[0] = fmaf(gv, a.x, acc[0]);
                    acc[1] = fmaf(gv, a.y, acc[1]);
                    acc[2] = fmaf(gv, a.z, acc[2]);
                    acc[3] = fmaf(gv, a.w, acc[3]);
                    acc[4] = fmaf(gv, b.x, acc[4]);
                    acc[5] = fmaf(gv, b.y, acc[5]);
                    acc[6] = fmaf(gv, b.z, acc[6]);
                    acc[7] = fmaf(gv, b.w, acc[7]);
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t)
                CMh[y][t] = __floats2half2_rn(fred(acc[2 * t], fp, invp), fred(acc[2 * t + 1], fp, invp));
        }
        __syncthreads();
        // (D) rows += CM Q, reduced, on the tensor cores over the 8-column
        // tiles from the group on and the 8-slot tiles up to its last slot;
        // warp w takes the 16-row tiles w, w + nwarp, ...
        {
            const int gid = lane >> 2, tig = lane & 3;
            const int nth = 8 - g, nt = nth + ((ns + nsg + 7) >> 3);  // column tiles, all tiles
            const int mtiles = (blockDim.x + 15) >> 4;
            for (int mt = warp; mt < mtiles; mt += nwarp) {
                const int r0 = 16 * mt;
                const uint32_t a0 = *(const uint32_t *)&CMh[r0 + gid][tig];
                const uint32_t a1 = *(const uint32_t *)&CMh[r0 + gid + 8][tig];
                uint8_t *ra = Rb + (r0 + gid) * U8_RB, *rb = Rb + (r0 + gid + 8) * U8_RB;
#pragma unroll 2
                for (int t2 = 0; t2 < nt; ++t2) {
                    const int off = t2 < nth ? 8 * (g + t2) : 64 + 8 * (t2 - nth);
                    const uint32_t b0 = *(const uint32_t *)&QT[off + gid][2 * tig];
                    const int e = off + 2 * tig;
                    const uint32_t ua = *(const uint16_t *)(ra + e), ub = *(const uint16_t *)(rb + e);
                    float d0 = (float)(ua & 0xFF), d1 = (float)(ua >> 8), d2 = (float)(ub & 0xFF), d3 = (float)(ub >> 8);
                    asm volatile(
                        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5}, {%6}, "
                        "{%0, %1, %2, %3};"
                        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
                        : "r"(a0), "r"(a1), "r"(b0));
                    *(uint16_t *)(ra + e) = (uint16_t)((uint32_t)fred(d0, fp, invp) | ((uint32_t)fred(d1, fp, invp) << 8));
                    *(uint16_t *)(rb + e) = (uint16_t)((uint32_t)fred(d2, fp, invp) | ((uint32_t)fred(d3, fp, invp) << 8));
                }
            }
        }
        __syncthreads();
        ns += nsg;
    }
    const int r = ns;
    // rank of each row among pivot rows (ascending) and among non-pivot rows
    const int isp_i = (y < alpha) && piv[y];
    unsigned bal = __ballot_sync(0xffffffffu, isp_i);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    before += __popc(bal & ((1u << lane) - 1));
    if (y < alpha) {
        if (isp_i) {
            pivpos[y] = (int16_t)before;
            sortedSlot[before] = slotOf[y];
            info[1 + before] = y;
        } else {
            pivpos[y] = (int16_t)(y - before);
        }
    }
    if (y == 0) info[0] = r;
    for (int c = y; c < beta; c += blockDim.x) place_non_pivot(slotCol, r, c, nonCol);
    if (y < r) info[1 + ECH_LEAF_COLS + y] = slotCol[y];
    __syncthreads();
    // the outputs, centred, straight from the (reduced) rows: lane l writes
    // output columns l and l + 32
    const int nr = beta - r;
    const int sa = lane < r ? 64 + sortedSlot[lane] : -1, sb = lane + 32 < r ? 64 + sortedSlot[lane + 32] : -1;
    const int ca = lane < nr ? nonCol[lane] : -1, cb = lane + 32 < nr ? nonCol[lane + 32] : -1;
    auto put = [&](T *dst, const uint8_t *rw, int e) {
        if (e >= 0) *dst = D::enc(cen(rw[e], p));
    };
    for (int l = warp; l < r; l += nwarp) {  // M and R: the pivot rows in slot order
        const uint8_t *rw = Rb + slotRow[l] * U8_RB;
        put(Mo + (int64_t)l * ldm + lane, rw, sa);
        put(Mo + (int64_t)l * ldm + lane + 32, rw, sb);
        put(Ro + (int64_t)l * ldr + lane, rw, ca);
        put(Ro + (int64_t)l * ldr + lane + 32, rw, cb);
    }
    for (int rw = warp; rw < alpha; rw += nwarp) {  // K: the other rows
        if (piv[rw]) continue;
        T *ko = Ko + (int64_t)pivpos[rw] * ldk;
        put(ko + lane, Rb + rw * U8_RB, sa);
        put(ko + lane + 32, Rb + rw * U8_RB, sb);
    }
}


// ---------------------------------------------------------------------------
// leaf echelonisation over GF(2): the same Gauss-Jordan with the topmost-row
// rule, each thread holding its row (<= 256 columns) and its <= 256 slot
// coefficients as 64-bit words in registers, taken eight columns at a time:
//  (A) every warp publishes its rows' bits in the group's columns, one
//      32-bit word per column (a ballot each);
//  (B) one finder warp runs the column-by-column elimination on that
//      1024 x 8 bit slice alone (lane l holds warp l's words), finding the
//      group's pivot rows x_s in order and, for every row y, the set CM_y of
//      group pivots whose rows as they stood at the group start make up what
//      was added to y (also one word per pivot);
//  (C) the group's pivot rows publish their rows as they stood at the group
//      start, with the identity of their slot;
//  (D) all threads tabulate the XOR of every subset of pivots 0..3 and of
//      pivots 4..7 (two 16-entry tables);
//  (E) row y adds the two entries that make up CM_y (and a pivot row its
//      own identity).
// Rows are linear in the rows they were built from, so (E) reproduces the
// column-by-column result; four barriers per group instead of one per column.
// ---------------------------------------------------------------------------
// register-resident word arrays: select / update word i without local memory
template <int W> __device__ __forceinline__ uint64_t wpick(const uint64_t (&a)[W], int i) {
    uint64_t v = a[0];
#pragma unroll
    for (int w = 1; w < W; ++w)
        if (i == w) v = a[w];
    return v;
}
template <int W> __device__ __forceinline__ void wxor(uint64_t (&a)[W], int i, uint64_t m) {
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (i == w) a[w] ^= m;
}
// word i of eight, select tree of depth 3
__device__ __forceinline__ uint32_t sel8(const uint32_t (&a)[8], int i) {
    const uint32_t l0 = (i & 1) ? a[1] : a[0], l1 = (i & 1) ? a[3] : a[2];
    const uint32_t l2 = (i & 1) ? a[5] : a[4], l3 = (i & 1) ? a[7] : a[6];
    const uint32_t m0 = (i & 2) ? l1 : l0, m1 = (i & 2) ? l3 : l2;
    return (i & 4) ? m1 : m0;
}

template <int W, typename T>
__global__ void __launch_bounds__(1024, 1) k_ech_leaf_gf2(int alpha, int beta, const T *H, int64_t ldh,
                                                          int32_t *info, T *Mo, int64_t ldm, T *Ko,
                                                          int64_t ldk, T *Ro, int64_t ldr, T one) {
    // 1024 threads, thread y owns row y (registers: W words of the row and W
    // words of slot coefficients)
    static_assert(W == 4, "one bitmask byte per lane in the load");
    extern __shared__ uint64_t smw[];
    uint64_t *hw = smw;                  // [threads][W] rows after elimination
    uint64_t *tw = smw + blockDim.x * W; // [threads][W] slot coefficients
    __shared__ uint64_t orig[8][2 * W];    // the group's pivot rows at the group start
    __shared__ uint64_t tab[2][2 * W][16]; // XOR of every subset of pivots 0..3 / 4..7 (word-major)
    __shared__ uint32_t slc[32][8];        // bit q of slc[w][k]: column c0+k of row 32w+q
    __shared__ __align__(16) uint32_t cms[32][8];  // bit q of cms[w][s]: pivot s in CM of row 32w+q
    __shared__ int16_t gpr[8], gpc[8];     // the group's pivots: row, column
    __shared__ uint8_t gmark[1024];        // 1 + the group slot of a row that is a group pivot, else 0
    __shared__ int gnp;
    __shared__ uint8_t piv[1024];
    __shared__ int16_t slotOf[1024], pivpos[1024];
    __shared__ int16_t slotRow[64 * W], slotCol[64 * W], sortedSlot[64 * W], nonCol[64 * W];
    __shared__ int wsum[32];
    const int y = threadIdx.x, lane = y & 31, warp = y >> 5, nwarp = blockDim.x >> 5;

    // coalesced load into the rows' 32-byte bitmasks.  One-byte codes: warp w
    // reads its 32 rows two at a time, lane l 16 columns 16 (l % 16) .. of
    // row 2 i + l / 16 (16-byte loads; a byte is 1 iff it is not zero: four
    // bytes at a time by a SIMD compare and a multiply that gathers their
    // flags).  Two-byte codes: one row at a time, lane l columns 8l..8l+7.
    if constexpr (sizeof(T) == 1) {
        uint8_t *hb = (uint8_t *)hw;
        const int half = lane >> 4, ch = lane & 15, c16 = 16 * ch;
#pragma unroll 8
        for (int rr = 0; rr < 16; ++rr) {
            const int row = warp * 32 + 2 * rr + half;
            uint32_t mask = 0;
            if (row < alpha) {
                const T *rp = H + (int64_t)row * ldh + c16;
                if (c16 + 16 <= beta && ((uintptr_t)rp & 15) == 0) {
                    const uint4 v = *(const uint4 *)rp;
                    const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        mask |= (((__vcmpne4(vv[q], 0u) & 0x01010101u) * 0x01020408u) >> 24) << (4 * q);
                } else {
                    for (int q = 0; q < 16 && c16 + q < beta; ++q)
                        if (rp[q]) mask |= 1u << q;
                }
            }
            *(uint16_t *)(hb + row * 8 * W + 2 * ch) = (uint16_t)mask;
        }
    } else {
        uint8_t *hb = (uint8_t *)hw;
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            const int row = warp * 32 + rr;
            uint32_t mask = 0;
            if (row < alpha) {
                const T *rp = H + (int64_t)row * ldh + 8 * lane;
                const int c0 = 8 * lane;
                if (c0 + 8 <= beta && ((uintptr_t)rp & (8 * sizeof(T) - 1)) == 0) {
                    if constexpr (sizeof(T) == 1) {
                        const uint2 v = *(const uint2 *)rp;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            mask |= ((v.x >> (8 * q)) & 0xFF) ? 1u << q : 0u;
                            mask |= ((v.y >> (8 * q)) & 0xFF) ? 1u << (4 + q) : 0u;
                        }
                    } else {
                        const uint4 v = *(const uint4 *)rp;
                        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            mask |= (vv[q] & 0xFFFF) ? 1u << (2 * q) : 0u;
                            mask |= (vv[q] >> 16) ? 1u << (2 * q + 1) : 0u;
                        }
                    }
                } else {
                    for (int q = 0; q < 8 && c0 + q < beta; ++q)
                        if (rp[q]) mask |= 1u << q;
                }
            }
            hb[row * 8 * W + lane] = (uint8_t)mask;
        }
    }
    __syncthreads();
    uint64_t h[W], t[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h[w] = hw[y * W + w];
        t[w] = 0;
    }
    piv[y] = 0;
    slotOf[y] = -1;
    gmark[y] = 0;
    bool isp = false;
    __syncthreads();

    // the finder's state (warp 0): lane l's rows 32l..32l+31 that may still
    // become pivots
    uint32_t cand_rows = 0;
    if (warp == 0 && lane * 32 < alpha) cand_rows = alpha - lane * 32 >= 32 ? 0xffffffffu : (1u << (alpha - lane * 32)) - 1;
    int ns = 0;
    for (int c0 = 0; c0 < beta; c0 += 8) {
        // (A) this warp's rows in columns c0..c0+7 (c0 is a multiple of 8),
        // one 32-bit word per column
        {
            const uint32_t by = (uint32_t)(wpick<W>(h, c0 >> 6) >> (c0 & 63));
            uint32_t mine = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t b = __ballot_sync(0xffffffffu, (by >> k) & 1u);
                if (lane == k) mine = b;
            }
            if (lane < 8) slc[warp][lane] = mine;
        }
        __syncthreads();
        // (B) the finder: elimination on the group's columns only, bit-sliced:
        // bit q of col[k] is column c0+k of row 32*lane+q, bit q of cmb[s]
        // says group pivot s is in that row's combination
        if (warp == 0) {
            uint32_t col[8], cmb[8];
            const bool live = lane < nwarp;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                col[k] = live ? slc[lane][k] : 0u;
                cmb[k] = 0u;
            }
            int np = 0;
            // unrolled over the group's columns, so that each step touches only
            // what can still change: the columns right of k and the group's
            // pivots found so far (np <= k)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                // every lane takes its own first candidate row q and forms that
                // row's bits and combination; the lowest lane with a candidate
                // holds the pivot and broadcasts them
                const uint32_t cand = col[k] & cand_rows;
                const int q = __ffs(cand) - 1;  // -1: none here
                const int qq = q & 31;
                uint32_t mine = 0;
#pragma unroll
                for (int u = k + 1; u < 8; ++u) mine |= ((col[u] >> qq) & 1u) << u;
#pragma unroll
                for (int u = 0; u < k; ++u) mine |= ((cmb[u] >> qq) & 1u) << (8 + u);
                const unsigned bal = __ballot_sync(0xffffffffu, cand != 0u);
                if (bal == 0u) continue;  // uniform: no pivot in this column
                const int owner = __ffs(bal) - 1;
                const uint32_t v = __shfl_sync(0xffffffffu, mine, owner);
                const uint32_t pb = v & 0xFFu, pc = ((v >> 8) & 0xFFu) ^ (1u << np);
                // rows with column c0+k set, other than the pivot
                const uint32_t rows = col[k] & ~(lane == owner ? 1u << q : 0u);
#pragma unroll
                for (int u = k + 1; u < 8; ++u) col[u] ^= rows & (0u - ((pb >> u) & 1u));
#pragma unroll
                for (int u = 0; u <= k; ++u) cmb[u] ^= rows & (0u - ((pc >> u) & 1u));
                if (lane == owner) {
                    cand_rows &= ~(1u << q);
                    gpr[np] = (int16_t)(lane * 32 + q);
                    gpc[np] = (int16_t)(c0 + k);
                    gmark[lane * 32 + q] = (uint8_t)(np + 1);
                }
                ++np;
            }
            if (live) {
#pragma unroll
                for (int u = 0; u < 8; ++u) cms[lane][u] = cmb[u];
            }
            if (lane == 0) gnp = np;
        }
        __syncthreads();
        const int np = gnp;
        if (np == 0) continue;  // uniform
        // (C) the group's pivot rows as they stand now, with their identity
        const int s_me = (int)gmark[y] - 1;
        if (s_me >= 0) gmark[y] = 0;
        if (s_me >= 0) {
            const int slot = ns + s_me;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                orig[s_me][w] = h[w];
                orig[s_me][W + w] = t[w] ^ ((slot >> 6) == w ? (uint64_t)1 << (slot & 63) : 0ull);
            }
            isp = true;
            piv[y] = 1;
            slotOf[y] = (int16_t)slot;
            slotRow[slot] = (int16_t)y;
            slotCol[slot] = gpc[s_me];
        }
        __syncthreads();
        // (D) XOR of every subset of pivots 0..3 and of pivots 4..7
        for (int e = y; e < 2 * 2 * W * 16; e += blockDim.x) {
            const int half = e >> 7, w = (e >> 4) & (2 * W - 1), m = e & 15;
            uint64_t v = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (((m >> u) & 1) && 4 * half + u < np) v ^= orig[4 * half + u][w];
            tab[half][w][m] = v;
        }
        __syncthreads();
        // (E) add the rows of this row's combination; a pivot row also its identity
        int m = 0;
        {
            const uint4 ca = *(const uint4 *)&cms[warp][0], cb = *(const uint4 *)&cms[warp][4];
            const uint32_t cw[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
            for (int u = 0; u < 8; ++u) m |= (int)((cw[u] >> lane) & 1u) << u;
        }
        if (m) {
            // the group's pivot rows are zero left of column c0 and in slot
            // words past the group's last slot, and the second table is empty
            // when the group has at most four pivots: those words are skipped
            const int lo = m & 15, hi = m >> 4;
            const int hfirst = c0 >> 6, tlast = (ns + np - 1) >> 6;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (w >= hfirst) h[w] ^= tab[0][w][lo] ^ (np > 4 ? tab[1][w][hi] : 0ull);
                if (w <= tlast) t[w] ^= tab[0][W + w][lo] ^ (np > 4 ? tab[1][W + w][hi] : 0ull);
            }
        }
        if (s_me >= 0) wxor<W>(t, (ns + s_me) >> 6, (uint64_t)1 << ((ns + s_me) & 63));
        ns += np;
    }
    const int r = ns;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        hw[y * W + w] = h[w];
        tw[y * W + w] = t[w];
    }
    unsigned bal = __ballot_sync(0xffffffffu, isp);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    before += __popc(bal & ((1u << lane) - 1));
    if (y < alpha) {
        if (isp) {
            pivpos[y] = (int16_t)before;
            sortedSlot[before] = slotOf[y];
            info[1 + before] = y;
        } else {
            pivpos[y] = (int16_t)(y - before);
        }
    }
    if (y == 0) info[0] = r;
    for (int c = y; c < beta; c += blockDim.x) place_non_pivot(slotCol, r, c, nonCol);
    if (y < r) info[1 + 64 * W + y] = slotCol[y];
    __syncthreads();
    // outputs: one row per warp; lane l writes the row's entries 8l .. 8l+7
    // (r <= 256), picking each from the row's 4 words by a fixed bit index
    // (the sorted slot for M and K, the non-pivot column for R)
    // Each lane's 8 output columns read the same bit positions of every row
    // (a sorted slot for M and K, a non-pivot column for R): their 32-bit
    // word and shift are computed once, and a row costs 8 shared loads, 8
    // bit extracts and one multiply per 4 entries (bits times the code of 1).
    const int e0 = 8 * lane;
    auto emit = [&](const uint64_t *src, const int (&qw)[8], const int (&qsh)[8], int count, T *out) {
        const uint32_t *s32 = (const uint32_t *)src;
        uint32_t b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = (s32[qw[j]] >> qsh[j]) & 1u;
        if (e0 + 8 <= count && ((uintptr_t)(out + e0) & (8 * sizeof(T) - 1)) == 0) {
            if constexpr (sizeof(T) == 1) {
                uint2 pk;
                pk.x = (b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24)) * (uint32_t)one;
                pk.y = (b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24)) * (uint32_t)one;
                *(uint2 *)(out + e0) = pk;
            } else {
                uint4 pk;
                pk.x = (b[0] | (b[1] << 16)) * (uint32_t)one;
                pk.y = (b[2] | (b[3] << 16)) * (uint32_t)one;
                pk.z = (b[4] | (b[5] << 16)) * (uint32_t)one;
                pk.w = (b[6] | (b[7] << 16)) * (uint32_t)one;
                *(uint4 *)(out + e0) = pk;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (e0 + j < count) out[e0 + j] = b[j] ? one : (T)0;
        }
    };
    if (e0 < r) {
        int qw[8], qsh[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int q = e0 + j < r ? sortedSlot[e0 + j] : 0;
            qw[j] = q >> 5;
            qsh[j] = q & 31;
        }
        // M[l][s] = coefficient of pivot row rho_s in echelon row l
        for (int l = warp; l < r; l += nwarp) emit(tw + slotRow[l] * W, qw, qsh, r, Mo + (int64_t)l * ldm);
        // K[t][s] for the non-pivot rows t
        for (int row = warp; row < alpha; row += nwarp)
            if (!piv[row]) emit(tw + row * W, qw, qsh, r, Ko + (int64_t)pivpos[row] * ldk);
    }
    // R[l][j] = entry of echelon row l in the j-th non-pivot column
    const int nr = beta - r;
    if (e0 < nr) {
        int qw[8], qsh[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = e0 + j < nr ? nonCol[e0 + j] : 0;
            qw[j] = c >> 5;
            qsh[j] = c & 31;
        }
        for (int l = warp; l < r; l += nwarp) emit(hw + slotRow[l] * W, qw, qsh, nr, Ro + (int64_t)l * ldr);
    }
}

int ech_leaf_cols(int p) { return p == 2 ? ECH_LEAF_COLS_GF2 : ECH_LEAF_COLS; }

void ech_leaf(const Launch &L, int64_t alpha, int64_t beta, const void *H, int64_t ldh,
              int32_t *info, void *M, int64_t ldm, void *K, int64_t ldk, void *R, int64_t ldr) {
    // one thread per row: the CTA shrinks with the rows still to eliminate
    const int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(32, (alpha + 31) / 32 * 32));
    if (L.p == 2) {
        const int smem_max = 2 * 1024 * 4 * 8, smem = 2 * threads * 4 * 8;
        static std::once_flag once[2];
        cudaEvent_t ev;
        prof_begin(L, K_ECH, &ev);
        if (L.codec == CODEC_F8) {
            std::call_once(once[0], [&] {
                cudaFuncSetAttribute(k_ech_leaf_gf2<4, uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
            });
            k_ech_leaf_gf2<4, uint8_t><<<1, threads, smem, L.st>>>((int)alpha, (int)beta, (const uint8_t *)H, ldh, info,
                (uint8_t *)M, ldm, (uint8_t *)K, ldk, (uint8_t *)R, ldr, (uint8_t)0x38);
        } else {
            std::call_once(once[1], [&] {
                cudaFuncSetAttribute(k_ech_leaf_gf2<4, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
            });
            k_ech_leaf_gf2<4, uint16_t><<<1, threads, smem, L.st>>>((int)alpha, (int)beta, (const uint16_t *)H, ldh,
                info, (uint16_t *)M, ldm, (uint16_t *)K, ldk, (uint16_t *)R, ldr, (uint16_t)0x3F80);
        }
        prof_end(L, K_ECH, ev, (double)alpha * (double)beta * (double)(alpha < beta ? alpha : beta), 0, alpha, beta);
        return;
    }
    // the byte leaf for small p and more rows than the fp32 leaf takes
    const bool small = L.p <= 13 && alpha > F32_LEAF_ROWS;
    InvTable it{};  // inverses mod p by x^-1 = -(p / x) * (p mod x)^-1
    it.v[1] = 1;
    for (int x = 2; x < L.p; ++x) it.v[x] = (uint8_t)((L.p - (L.p / x) * it.v[L.p % x] % L.p) % L.p);
    static std::once_flag once2[4];
    cudaEvent_t ev;
    prof_begin(L, K_ECH, &ev);
#define GFE_U8(CODEC, T, IDX)                                                                                    \
    do {                                                                                                          \
        std::call_once(once2[IDX], [&] {                                                                          \
            cudaFuncSetAttribute(k_ech_leaf_u8<CODEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 1024 * U8_RB); \
        });                                                                                                       \
        k_ech_leaf_u8<CODEC><<<1, threads, threads * U8_RB, L.st>>>(it, L.p, (int)alpha, (int)beta, (const T *)H, \
                                                                 ldh, info, (T *)M, ldm, (T *)K, ldk, (T *)R, ldr); \
    } while (0)
#define GFE_F32(CODEC, T, IDX)                                                                                   \
    do {                                                                                                          \
        std::call_once(once2[IDX], [&] {                                                                          \
            cudaFuncSetAttribute(k_ech_leaf_f32<CODEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                 f32_leaf_smem(F32_LEAF_ROWS));                                                   \
        });                                                                                                       \
        /* two threads per row: 2 x (rows rounded up to 32) */                                                    \
        k_ech_leaf_f32<CODEC><<<1, 2 * threads, f32_leaf_smem(threads), L.st>>>(                                   \
            it, L.p, (int)alpha, (int)beta, (const T *)H, ldh, info, (T *)M, ldm, (T *)K, ldk, (T *)R, ldr);       \
    } while (0)
    if (L.codec == CODEC_F8) {
        if (small) GFE_U8(CODEC_F8, uint8_t, 0);
        else GFE_F32(CODEC_F8, uint8_t, 1);
    } else {
        if (small) GFE_U8(CODEC_BF16, uint16_t, 2);
        else GFE_F32(CODEC_BF16, uint16_t, 3);
    }
#undef GFE_U8
#undef GFE_F32
    prof_end(L, K_ECH, ev, (double)alpha * (double)beta * (double)(alpha < beta ? alpha : beta), 0, alpha, beta);
}

// ---------------------------------------------------------------------------
// extracts / riffles (jobs REX, RRF, CEX, CRZ, ADI) -- pure data movement
// ---------------------------------------------------------------------------
// copy one row segment: 16-byte vectors when both ends allow it
template <typename T>
__device__ __forceinline__ void copy_row(T *d, const T *src, int64_t ncols, int64_t t0, int64_t stride) {
    const int64_t bytes = ncols * (int64_t)sizeof(T);
    if ((((uintptr_t)d | (uintptr_t)src) & 15) == 0) {
        const int64_t nv = bytes >> 4;
        const uint4 *s4 = (const uint4 *)src;
        uint4 *d4 = (uint4 *)d;
        for (int64_t v = t0; v < nv; v += stride) d4[v] = s4[v];
        for (int64_t c = (nv << 4) / (int64_t)sizeof(T) + t0; c < ncols; c += stride) d[c] = src[c];
    } else {
        for (int64_t c = t0; c < ncols; c += stride) d[c] = src[c];
    }
}

// index arrays as kernel parameters: a device pointer, or the entries by value
struct MapPtr {
    const int32_t *p;
    __device__ __forceinline__ int32_t operator[](int64_t i) const { return p[i]; }
};
template <int N> struct MapVal {
    int32_t v[N];
    __device__ __forceinline__ int32_t operator[](int64_t i) const { return v[i]; }
};
// calls f with the map in the cheapest form: by value (two size classes) or
// as a device pointer
template <typename F> static void with_map(const IdxMap &m, F &&f) {
    if (m.host && m.n <= 256) {
        MapVal<256> v;
        std::memcpy(v.v, m.host, sizeof(int32_t) * (size_t)m.n);
        f(v);
    } else if (m.host && m.n <= MAP_INLINE) {
        MapVal<MAP_INLINE> v;
        std::memcpy(v.v, m.host, sizeof(int32_t) * (size_t)m.n);
        f(v);
    } else {
        f(MapPtr{m.dev});
    }
}

template <typename T, typename Map>
__global__ void k_gather_rows(int64_t nrows, int64_t ncols, T *dst, int64_t ldd, const T *A,
                              int64_t lda, const T *B, int64_t ldb, const __grid_constant__ Map map) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t row = blockIdx.y; row < nrows; row += gridDim.y) {
        int32_t s = map[row];
        const T *src = s >= 0 ? A + (int64_t)s * lda : B + (int64_t)(-1 - s) * ldb;
        copy_row(dst + row * ldd, src, ncols, t0, stride);
    }
}

// each thread: 4 consecutive output columns of a set of rows; the map is
// read once, the 4 results are stored as one vector when aligned
template <typename T, typename Map>
__global__ void k_gather_cols(int64_t nrows, int64_t ncols, T *dst, int64_t ldd, const T *src,
                              int64_t lds, const __grid_constant__ Map map) {
    const int64_t c0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (c0 >= ncols) return;
    const int nc = ncols - c0 < 4 ? (int)(ncols - c0) : 4;
    int32_t s[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] = q < nc ? map[c0 + q] : -1;
    const bool vec = nc == 4 && (((uintptr_t)(dst + c0) | (uintptr_t)(ldd * sizeof(T))) & (4 * sizeof(T) - 1)) == 0;
    for (int64_t row = blockIdx.y; row < nrows; row += gridDim.y) {
        const T *sr = src + row * lds;
        T v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = s[q] >= 0 ? sr[s[q]] : (T)0;
        T *dr = dst + row * ldd + c0;
        if (vec) {
            if constexpr (sizeof(T) == 1)
                *(uint32_t *)dr = (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16) | ((uint32_t)v[3] << 24);
            else
                *(uint2 *)dr = make_uint2((uint32_t)v[0] | ((uint32_t)v[1] << 16), (uint32_t)v[2] | ((uint32_t)v[3] << 16));
        } else {
            for (int q = 0; q < nc; ++q) dr[q] = v[q];
        }
    }
}

template <typename T>
__global__ void k_gather_rowptr(int64_t nrows, int64_t ncols, T *dst, int64_t ldd, const uint64_t *rows,
                                const int32_t *map) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int32_t s = map[c];
    for (int64_t row = blockIdx.y; row < nrows; row += gridDim.y)
        dst[row * ldd + c] = s >= 0 ? ((const T *)rows[row])[s] : (T)0;
}

template <typename T, typename Map>
__global__ void k_set_ones(int64_t count, T *V, int64_t ldv, const __grid_constant__ Map pos, T one) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) V[t * ldv + pos[t]] = one;
}

template <typename T>
__global__ void k_copy2d(int64_t rows, int64_t cols, T *dst, int64_t ldd, const T *src, int64_t lds) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        T *d = dst + row * ldd;
        if (src) {
            copy_row(d, src + row * lds, cols, t0, stride);
        } else if (((uintptr_t)d & 15) == 0) {
            const int64_t nv = (cols * (int64_t)sizeof(T)) >> 4;
            for (int64_t v = t0; v < nv; v += stride) ((uint4 *)d)[v] = make_uint4(0, 0, 0, 0);
            for (int64_t c = (nv << 4) / (int64_t)sizeof(T) + t0; c < cols; c += stride) d[c] = (T)0;
        } else {
            for (int64_t c = t0; c < cols; c += stride) d[c] = (T)0;
        }
    }
}

static dim3 grid_rc(int64_t rows, int64_t cols, int threads) {
    unsigned gx = cdiv(cols, threads);
    if (gx > 64) gx = 64;
    unsigned gy = (unsigned)(rows < 65535 ? rows : 65535);
    return dim3(gx, gy);
}

void gather_rows(const Launch &L, int64_t nrows, int64_t ncols, void *dst, int64_t ldd,
                 const void *A, int64_t lda, const void *B, int64_t ldb, const IdxMap &map) {
    if (nrows <= 0 || ncols <= 0) return;
    // one CTA row per output row (nrows <= 65535 always holds: rows <= blocks)
    const int64_t vec = (ncols * codec_bytes(L.codec) + 15) / 16;  // 16-byte vectors per row
    dim3 grid(cdiv(vec, 128) > 32 ? 32 : cdiv(vec, 128), (unsigned)(nrows < 65535 ? nrows : 65535));
    cudaEvent_t ev;
    prof_begin(L, K_ROWS, &ev);
    with_map(map, [&](const auto &mp) {
        using M = std::decay_t<decltype(mp)>;
        if (L.codec == CODEC_F8)
            k_gather_rows<uint8_t, M><<<grid, 128, 0, L.st>>>(nrows, ncols, (uint8_t *)dst, ldd,
                (const uint8_t *)A, lda, (const uint8_t *)B, ldb, mp);
        else
            k_gather_rows<uint16_t, M><<<grid, 128, 0, L.st>>>(nrows, ncols, (uint16_t *)dst, ldd,
                (const uint16_t *)A, lda, (const uint16_t *)B, ldb, mp);
    });
    prof_end(L, K_ROWS, ev, 0, 0, nrows, ncols);
}

void gather_cols(const Launch &L, int64_t nrows, int64_t ncols, void *dst, int64_t ldd,
                 const void *src, int64_t lds, const IdxMap &map) {
    if (nrows <= 0 || ncols <= 0) return;
    dim3 grid(cdiv((ncols + 3) / 4, 128), (unsigned)(nrows < 8192 ? nrows : 8192));
    cudaEvent_t ev;
    prof_begin(L, K_COLS, &ev);
    with_map(map, [&](const auto &mp) {
        using M = std::decay_t<decltype(mp)>;
        if (L.codec == CODEC_F8)
            k_gather_cols<uint8_t, M><<<grid, 128, 0, L.st>>>(nrows, ncols, (uint8_t *)dst, ldd,
                (const uint8_t *)src, lds, mp);
        else
            k_gather_cols<uint16_t, M><<<grid, 128, 0, L.st>>>(nrows, ncols, (uint16_t *)dst, ldd,
                (const uint16_t *)src, lds, mp);
    });
    prof_end(L, K_COLS, ev, 0, 0, nrows, ncols);
}

void gather_rowptr(const Launch &L, int64_t nrows, int64_t ncols, void *dst, int64_t ldd, const uint64_t *rows,
                   const int32_t *map) {
    if (nrows <= 0 || ncols <= 0) return;
    dim3 grid(cdiv(ncols, 128), (unsigned)(nrows < 8192 ? nrows : 8192));
    cudaEvent_t ev;
    prof_begin(L, K_COLS, &ev);
    if (L.codec == CODEC_F8)
        k_gather_rowptr<uint8_t><<<grid, 128, 0, L.st>>>(nrows, ncols, (uint8_t *)dst, ldd, rows, map);
    else
        k_gather_rowptr<uint16_t><<<grid, 128, 0, L.st>>>(nrows, ncols, (uint16_t *)dst, ldd, rows, map);
    prof_end(L, K_COLS, ev, 0, 0, nrows, ncols);
}

void set_ones(const Launch &L, int64_t count, void *V, int64_t ldv, const IdxMap &pos) {
    if (count <= 0) return;
    cudaEvent_t ev;
    prof_begin(L, K_COPY, &ev);
    with_map(pos, [&](const auto &mp) {
        using M = std::decay_t<decltype(mp)>;
        if (L.codec == CODEC_F8)
            k_set_ones<uint8_t, M><<<cdiv(count, 128), 128, 0, L.st>>>(count, (uint8_t *)V, ldv, mp, (uint8_t)0x38);
        else
            k_set_ones<uint16_t, M><<<cdiv(count, 128), 128, 0, L.st>>>(count, (uint16_t *)V, ldv, mp,
                                                                       (uint16_t)0x3F80);
    });
    prof_end(L, K_COPY, ev, 0, 0, count, 1);
}

void copy2d(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd, const void *src,
            int64_t lds) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid = grid_rc(rows, (cols * codec_bytes(L.codec) + 15) / 16, 256);
    cudaEvent_t ev;
    prof_begin(L, K_COPY, &ev);
    if (L.codec == CODEC_F8)
        k_copy2d<uint8_t><<<grid, 256, 0, L.st>>>(rows, cols, (uint8_t *)dst, ldd, (const uint8_t *)src, lds);
    else
        k_copy2d<uint16_t><<<grid, 256, 0, L.st>>>(rows, cols, (uint16_t *)dst, ldd, (const uint16_t *)src, lds);
    prof_end(L, K_COPY, ev, 0, 0, rows, cols);
}

void zero2d(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd) {
    copy2d(L, rows, cols, dst, ldd, nullptr, 0);
}

// ---------------------------------------------------------------------------
// conversions at the API boundary (jobs "pack and partition", output assembly)
// ---------------------------------------------------------------------------
template <int C>
__global__ void k_import_bits(int64_t rows, int64_t cols, typename Cd<C>::T *dst, int64_t ldd,
                              const uint64_t *src, int64_t ldw) {
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y)
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += (int64_t)gridDim.x * blockDim.x)
            dst[row * ldd + c] = Cd<C>::enc((int)((src[row * ldw + (c >> 6)] >> (c & 63)) & 1u));
}

// GF(2) bits -> e4m3 (0 or 1.0 = 0x38): 16 columns per thread, 16-byte stores
__global__ void k_import_bits_f8(int64_t rows, int64_t cols, uint8_t *dst, int64_t ldd, const uint64_t *src,
                                 int64_t ldw) {
    const int64_t nv = (cols + 15) >> 4;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const uint64_t *sr = src + row * ldw;
        uint8_t *dr = dst + row * ldd;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c0 = v << 4;  // a multiple of 16: inside one source word
            const uint32_t bits = (uint32_t)(sr[c0 >> 6] >> (c0 & 63)) & 0xFFFFu;
            uint32_t q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)  // nibble -> one flag per byte -> 0x38 per set byte
                q[j] = ((((bits >> (4 * j)) & 0xFu) * 0x00204081u) & 0x01010101u) * 0x38u;
            if (c0 + 16 <= cols && ((uintptr_t)(dr + c0) & 15) == 0) {
                *(uint4 *)(dr + c0) = make_uint4(q[0], q[1], q[2], q[3]);
            } else {
                for (int j = 0; j < 16 && c0 + j < cols; ++j) dr[c0 + j] = (uint8_t)(q[j >> 2] >> (8 * (j & 3)));
            }
        }
    }
}

// e4m3 GF(2) entries -> bits: a warp takes 512 columns of a row, lane l the
// 16 bytes at 16 l (one 16-byte load), four lanes make one 64-bit word
__global__ void k_export_bits_f8(int64_t rows, int64_t cols, uint64_t *dst, int64_t ldw, const uint8_t *src,
                                 int64_t lds) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nseg = (cols + 511) >> 9;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const uint8_t *sr = src + row * lds;
        for (int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); seg < nseg; seg += warps) {
            const int64_t c0 = (seg << 9) + 16 * lane;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (c0 + 16 <= cols && ((uintptr_t)(sr + c0) & 15) == 0) {
                const uint4 v = *(const uint4 *)(sr + c0);
                w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
            } else {
                for (int j = 0; j < 16 && c0 + j < cols; ++j) w[j >> 2] |= (uint32_t)sr[c0 + j] << (8 * (j & 3));
            }
            uint64_t bits = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {  // non-zero magnitude -> 1 (entries are 0 or 1.0)
                const uint32_t nz = __vcmpne4(w[j] & 0x7F7F7F7Fu, 0u) & 0x01010101u;
                bits |= (uint64_t)((nz * 0x10204080u) >> 28) << (4 * j);
            }
            bits <<= 16 * (lane & 3);
            bits |= __shfl_xor_sync(0xffffffffu, bits, 1);
            bits |= __shfl_xor_sync(0xffffffffu, bits, 2);
            const int64_t wi = (seg << 3) + (lane >> 2);
            if ((lane & 3) == 0 && (wi << 6) < cols) dst[row * ldw + wi] = bits;
        }
    }
}

// residues -> codec through a 256-entry table (enc(cen(x)) for every byte
// value x), 16 bytes per thread
template <int C>
__global__ void k_import_u8_vec(int p, int64_t rows, int64_t cols, typename Cd<C>::T *dst, int64_t ldd,
                                const uint8_t *src, int64_t lds) {
    using T = typename Cd<C>::T;
    __shared__ T tab[256];
    for (int x = threadIdx.x; x < 256; x += blockDim.x) tab[x] = Cd<C>::enc(cen(x, p));
    __syncthreads();
    const int64_t nv = (cols + 15) >> 4;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const uint8_t *sr = src + row * lds;
        T *dr = dst + row * ldd;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c0 = v << 4;
            if (c0 + 16 <= cols && ((uintptr_t)(sr + c0) & 15) == 0 && ((uintptr_t)(dr + c0) & 15) == 0) {
                const uint4 in = *(const uint4 *)(sr + c0);
                const uint32_t w[4] = {in.x, in.y, in.z, in.w};
                if constexpr (sizeof(T) == 1) {
                    uint32_t o[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        o[j] = (uint32_t)tab[w[j] & 0xFF] | ((uint32_t)tab[(w[j] >> 8) & 0xFF] << 8) |
                               ((uint32_t)tab[(w[j] >> 16) & 0xFF] << 16) | ((uint32_t)tab[w[j] >> 24] << 24);
                    *(uint4 *)(dr + c0) = make_uint4(o[0], o[1], o[2], o[3]);
                } else {
                    uint32_t o[8];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        o[2 * j] = (uint32_t)tab[w[j] & 0xFF] | ((uint32_t)tab[(w[j] >> 8) & 0xFF] << 16);
                        o[2 * j + 1] = (uint32_t)tab[(w[j] >> 16) & 0xFF] | ((uint32_t)tab[w[j] >> 24] << 16);
                    }
                    *(uint4 *)(dr + c0) = make_uint4(o[0], o[1], o[2], o[3]);
                    *(uint4 *)(dr + c0 + 8) = make_uint4(o[4], o[5], o[6], o[7]);
                }
            } else {
                for (int j = 0; j < 16 && c0 + j < cols; ++j) dr[c0 + j] = tab[sr[c0 + j]];
            }
        }
    }
}

// codec -> residues [0, p), 16 entries per thread; e4m3 bytes go through a
// 256-entry table (res(dec(b)) for every byte b), which keeps the kernel on
// HBM rather than on the integer pipe
template <int C>
__global__ void k_export_u8_vec(int p, int64_t rows, int64_t cols, uint8_t *dst, int64_t ldd,
                                const typename Cd<C>::T *src, int64_t lds) {
    using T = typename Cd<C>::T;
    __shared__ uint8_t tab[256];
    if constexpr (sizeof(T) == 1) {
        for (int x = threadIdx.x; x < 256; x += blockDim.x) tab[x] = (uint8_t)res(Cd<C>::dec((T)x), p);
        __syncthreads();
    }
    const int64_t nv = (cols + 15) >> 4;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const T *sr = src + row * lds;
        uint8_t *dr = dst + row * ldd;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c0 = v << 4;
            if (c0 + 16 <= cols && ((uintptr_t)(sr + c0) & 15) == 0 && ((uintptr_t)(dr + c0) & 15) == 0) {
                T e[16];
#pragma unroll
                for (int j = 0; j < 16 * (int)sizeof(T); j += 16)
                    *(uint4 *)((char *)e + j) = *(const uint4 *)((const char *)(sr + c0) + j);
                uint32_t o[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    o[j] = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        uint32_t r;
                        if constexpr (sizeof(T) == 1) r = tab[e[4 * j + b]];
                        else r = (uint32_t)res(Cd<C>::dec(e[4 * j + b]), p);
                        o[j] |= r << (8 * b);
                    }
                }
                *(uint4 *)(dr + c0) = make_uint4(o[0], o[1], o[2], o[3]);
            } else {
                for (int j = 0; j < 16 && c0 + j < cols; ++j) dr[c0 + j] = (uint8_t)res(Cd<C>::dec(sr[c0 + j]), p);
            }
        }
    }
}

template <int C>
__global__ void k_export_bits(int64_t rows, int64_t cols, uint64_t *dst, int64_t ldw,
                              const typename Cd<C>::T *src, int64_t lds) {
    int64_t nw = (cols + 63) >> 6;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y)
        for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
            uint64_t v = 0;
            int64_t c0 = w << 6;
            int n = cols - c0 < 64 ? (int)(cols - c0) : 64;
            for (int b = 0; b < n; ++b)
                v |= (uint64_t)(Cd<C>::dec(src[row * lds + c0 + b]) & 1) << b;
            dst[row * ldw + w] = v;
        }
}

void import_u8(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd,
               const uint8_t *src, int64_t lds) {
    if (rows <= 0 || cols <= 0) return;
    const dim3 grid = grid_rc(rows, (cols + 15) / 16, 256);
    cudaEvent_t ev;
    prof_begin(L, K_CONV, &ev);
    if (L.codec == CODEC_F8)
        k_import_u8_vec<CODEC_F8><<<grid, 256, 0, L.st>>>(L.p, rows, cols, (uint8_t *)dst, ldd, src, lds);
    else
        k_import_u8_vec<CODEC_BF16><<<grid, 256, 0, L.st>>>(L.p, rows, cols, (uint16_t *)dst, ldd, src, lds);
    prof_end(L, K_CONV, ev, 0, 0, rows, cols);
}

void import_bits(const Launch &L, int64_t rows, int64_t cols, void *dst, int64_t ldd,
                 const uint64_t *src, int64_t ldw) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid = grid_rc(rows, cols, 256);
    cudaEvent_t ev;
    prof_begin(L, K_CONV, &ev);
    if (L.codec == CODEC_F8)
        k_import_bits_f8<<<grid_rc(rows, (cols + 15) / 16, 256), 256, 0, L.st>>>(rows, cols, (uint8_t *)dst, ldd,
                                                                                 src, ldw);
    else
        k_import_bits<CODEC_BF16><<<grid, 256, 0, L.st>>>(rows, cols, (uint16_t *)dst, ldd, src, ldw);
    prof_end(L, K_CONV, ev, 0, 0, rows, cols);
}

void export_u8(const Launch &L, int64_t rows, int64_t cols, uint8_t *dst, int64_t ldd,
               const void *src, int64_t lds) {
    if (rows <= 0 || cols <= 0) return;
    const dim3 grid = grid_rc(rows, (cols + 15) / 16, 256);
    cudaEvent_t ev;
    prof_begin(L, K_CONV, &ev);
    if (L.codec == CODEC_F8)
        k_export_u8_vec<CODEC_F8><<<grid, 256, 0, L.st>>>(L.p, rows, cols, dst, ldd, (const uint8_t *)src, lds);
    else
        k_export_u8_vec<CODEC_BF16><<<grid, 256, 0, L.st>>>(L.p, rows, cols, dst, ldd, (const uint16_t *)src, lds);
    prof_end(L, K_CONV, ev, 0, 0, rows, cols);
}

void export_bits(const Launch &L, int64_t rows, int64_t cols, uint64_t *dst, int64_t ldw,
                 const void *src, int64_t lds) {
    if (rows <= 0) return;
    int64_t nw = (cols + 63) >> 6;
    if (nw <= 0) return;
    dim3 grid = grid_rc(rows, nw, 128);
    cudaEvent_t ev;
    prof_begin(L, K_CONV, &ev);
    if (L.codec == CODEC_F8)
        k_export_bits_f8<<<grid_rc(rows, (cols + 511) / 512 * 32, 128), 128, 0, L.st>>>(rows, cols, dst, ldw,
                                                                                         (const uint8_t *)src, lds);
    else
        k_export_bits<CODEC_BF16><<<grid, 128, 0, L.st>>>(rows, cols, dst, ldw, (const uint16_t *)src, lds);
    prof_end(L, K_CONV, ev, 0, 0, rows, cols);
}

// dense E and T in the API storage
template <int C>
__global__ void k_build_E_u8(int p, int64_t m, int64_t n, int64_t r, uint8_t *dst, int64_t ldd,
                             const typename Cd<C>::T *R, int64_t ldr, const int32_t *colmap) {
    for (int64_t row = blockIdx.y; row < m; row += gridDim.y)
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
            uint8_t v = 0;
            if (row < r) {
                int32_t q = colmap[c];
                if (q >= 0) v = (q == row) ? (uint8_t)(p - 1) : 0;
                else v = (uint8_t)res(Cd<C>::dec(R[row * ldr + (-1 - q)]), p);
            }
            dst[row * ldd + c] = v;
        }
}

template <int C>
__global__ void k_build_E_bits(int64_t m, int64_t n, int64_t r, uint64_t *dst, int64_t ldw,
                               const typename Cd<C>::T *R, int64_t ldr, const int32_t *colmap) {
    int64_t nw = (n + 63) >> 6;
    for (int64_t row = blockIdx.y; row < m; row += gridDim.y)
        for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
            uint64_t v = 0;
            if (row < r) {
                int64_t c0 = w << 6;
                int nb = n - c0 < 64 ? (int)(n - c0) : 64;
                for (int b = 0; b < nb; ++b) {
                    int32_t q = colmap[c0 + b];
                    int bit = q >= 0 ? (q == row) : (Cd<C>::dec(R[row * ldr + (-1 - q)]) & 1);
                    v |= (uint64_t)bit << b;
                }
            }
            dst[row * ldw + w] = v;
        }
}

template <int C>
__global__ void k_build_T_u8(int p, int64_t m, int64_t r, uint8_t *dst, int64_t ldd,
                             const typename Cd<C>::T *M, int64_t ldm, const typename Cd<C>::T *K,
                             int64_t ldk, const int32_t *rowmap) {
    for (int64_t row = blockIdx.y; row < m; row += gridDim.y)
        for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < m; x += (int64_t)gridDim.x * blockDim.x) {
            int32_t q = rowmap[x];
            int v;
            if (row < r) v = q >= 0 ? res(Cd<C>::dec(M[row * ldm + q]), p) : 0;
            else v = q >= 0 ? res(Cd<C>::dec(K[(row - r) * ldk + q]), p) : ((-1 - q) == row - r ? 1 : 0);
            dst[row * ldd + x] = (uint8_t)v;
        }
}

template <int C>
__global__ void k_build_T_bits(int64_t m, int64_t r, uint64_t *dst, int64_t ldw,
                               const typename Cd<C>::T *M, int64_t ldm, const typename Cd<C>::T *K,
                               int64_t ldk, const int32_t *rowmap) {
    int64_t nw = (m + 63) >> 6;
    for (int64_t row = blockIdx.y; row < m; row += gridDim.y)
        for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
            uint64_t v = 0;
            int64_t x0 = w << 6;
            int nb = m - x0 < 64 ? (int)(m - x0) : 64;
            for (int b = 0; b < nb; ++b) {
                int32_t q = rowmap[x0 + b];
                int bit;
                if (row < r) bit = q >= 0 ? (Cd<C>::dec(M[row * ldm + q]) & 1) : 0;
                else bit = q >= 0 ? (Cd<C>::dec(K[(row - r) * ldk + q]) & 1) : ((-1 - q) == row - r);
                v |= (uint64_t)bit << b;
            }
            dst[row * ldw + w] = v;
        }
}

void build_E(const Launch &L, int fmt, int64_t m, int64_t n, int64_t r, void *dst, int64_t ldd,
             const void *R, int64_t ldr, const int32_t *colmap) {
    if (m <= 0 || n <= 0) return;
    cudaEvent_t ev;
    prof_begin(L, K_CONV, &ev);
    if (fmt == 1) {
        int64_t nw = (n + 63) >> 6;
        if (L.codec == CODEC_F8)
            k_build_E_bits<CODEC_F8><<<grid_rc(m, nw, 128), 128, 0, L.st>>>(m, n, r, (uint64_t *)dst, ldd / 8,
                                                                             (const uint8_t *)R, ldr, colmap);
        else
            k_build_E_bits<CODEC_BF16><<<grid_rc(m, nw, 128), 128, 0, L.st>>>(m, n, r, (uint64_t *)dst, ldd / 8,
                                                                               (const uint16_t *)R, ldr, colmap);
    } else if (L.codec == CODEC_F8) {
        k_build_E_u8<CODEC_F8><<<grid_rc(m, n, 256), 256, 0, L.st>>>(L.p, m, n, r, (uint8_t *)dst, ldd,
                                                                      (const uint8_t *)R, ldr, colmap);
    } else {
        k_build_E_u8<CODEC_BF16><<<grid_rc(m, n, 256), 256, 0, L.st>>>(L.p, m, n, r, (uint8_t *)dst, ldd,
                                                                        (const uint16_t *)R, ldr, colmap);
    }
    prof_end(L, K_CONV, ev, 0, 0, m, n);
}

void build_T(const Launch &L, int fmt, int64_t m, int64_t r, void *dst, int64_t ldd, const void *M,
             int64_t ldm, const void *K, int64_t ldk, const int32_t *rowmap) {
    if (m <= 0) return;
    cudaEvent_t ev;
    prof_begin(L, K_CONV, &ev);
    if (fmt == 1) {
        int64_t nw = (m + 63) >> 6;
        if (L.codec == CODEC_F8)
            k_build_T_bits<CODEC_F8><<<grid_rc(m, nw, 128), 128, 0, L.st>>>(m, r, (uint64_t *)dst, ldd / 8,
                (const uint8_t *)M, ldm, (const uint8_t *)K, ldk, rowmap);
        else
            k_build_T_bits<CODEC_BF16><<<grid_rc(m, nw, 128), 128, 0, L.st>>>(m, r, (uint64_t *)dst, ldd / 8,
                (const uint16_t *)M, ldm, (const uint16_t *)K, ldk, rowmap);
    } else if (L.codec == CODEC_F8) {
        k_build_T_u8<CODEC_F8><<<grid_rc(m, m, 256), 256, 0, L.st>>>(L.p, m, r, (uint8_t *)dst, ldd,
            (const uint8_t *)M, ldm, (const uint8_t *)K, ldk, rowmap);
    } else {
        k_build_T_u8<CODEC_BF16><<<grid_rc(m, m, 256), 256, 0, L.st>>>(L.p, m, r, (uint8_t *)dst, ldd,
            (const uint16_t *)M, ldm, (const uint16_t *)K, ldk, rowmap);
    }
    prof_end(L, K_CONV, ev, 0, 0, m, m);
}

__global__ void k_write_i64(int64_t *dst, const int32_t *src, int64_t count, int64_t offset) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) dst[t] = (int64_t)src[t] + offset;
}

// any non-zero entry (either codec: zero is the all-zero pattern, and -0 is
// never stored), 16 bytes per thread where aligned
__global__ void k_any_nonzero(int64_t rows, int64_t bytes, const uint8_t *A, int64_t ldb, int32_t *flag) {
    bool nz = false;
    for (int64_t row = blockIdx.y; row < rows && !nz; row += gridDim.y) {
        const uint8_t *r = A + row * ldb;
        const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
        if (((uintptr_t)r & 15) == 0) {
            const int64_t nv = bytes >> 4;
            for (int64_t v = t0; v < nv && !nz; v += st) {
                const uint4 q = ((const uint4 *)r)[v];
                nz = (q.x | q.y | q.z | q.w) != 0;
            }
            for (int64_t c = (nv << 4) + t0; c < bytes && !nz; c += st) nz = r[c] != 0;
        } else {
            for (int64_t c = t0; c < bytes && !nz; c += st) nz = r[c] != 0;
        }
    }
    if (nz) *flag = 1;
}

void any_nonzero(const Launch &L, int64_t rows, int64_t cols, const void *A, int64_t lda, int32_t *flag) {
    if (rows <= 0 || cols <= 0) return;
    const int es = codec_bytes(L.codec);
    const int64_t bytes = cols * es;
    k_any_nonzero<<<grid_rc(rows, (bytes + 15) / 16, 128), 128, 0, L.st>>>(rows, bytes, (const uint8_t *)A,
                                                                             lda * es, flag);
}

void write_i64(const Launch &L, int64_t *dst, const int32_t *src, int64_t count, int64_t offset) {
    if (count <= 0) return;
    cudaEvent_t ev;
    prof_begin(L, K_OTHER, &ev);
    k_write_i64<<<cdiv(count, 256), 256, 0, L.st>>>(dst, src, count, offset);
    prof_end(L, K_OTHER, ev, 0, 0, count, 1);
}

}  // namespace gfe
