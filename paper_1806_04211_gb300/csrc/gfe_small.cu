// Batched form for small matrices: ONE persistent launch per kind of kernel
// echelonises a whole list of independent matrices (rows and columns up to
// SMALL_MAX); a CTA per SM takes the matrices one after the other from a
// device counter and runs the entire method on each.  For matrices this small the
// blocked scheme's work is dominated by its per-block launches and host
// round trips; here each matrix costs no launch of its own and no host
// synchronisation at all.
//
// What a CTA computes is the unique result of Section 3.1 (Eq. "echelon"):
// r, the row rank profile rho, the column rank profile Ups, R, and the
// transformation blocks M = -C[rho,Ups]^-1 and K = C[rho_bar,Ups] M, in the
// negative normalisation (pivots -1, Section 2.2), the same output as the
// Chief's.  The route is column-greedy Gauss-Jordan with the topmost-row rule
// (a column's pivot is the first row, top to bottom, that is not yet a pivot
// row and has a non-zero there), which selects exactly the row rank profile,
// in the style of the single-block ECH of Section 2.3 done on one matrix:
//   * in place: once column c has been cleared against pivot row i it holds
//     no information, so it stores column i of the transformation T (T A = E)
//     instead, and every later row operation updates it with the rest of the
//     row (the classical in-place Gauss-Jordan inverse).  The workspace is
//     then just the m x n matrix;
//   * GF(p), 3 <= p <= 13, one byte per entry, blocked by panels of BK
//     columns (the delayed update of the paper's blocked scheme, inside one
//     CTA): the panel is eliminated in shared memory, one thread per row,
//     with bytes reduced lazily (every klazy pivot steps, while
//     p-1 + klazy (p-1)^2 <= 255 keeps every byte below 256); its pivot
//     columns then hold the coefficients with which each row combines the
//     panel's pivot rows, and the rest of every row is updated in ONE pass
//     as a rank-kp multiply-add (two entries per 32-bit word in 16-bit
//     lanes, exact reduction at the end), so each row is read and written
//     once per panel instead of once per pivot;
//   * GF(p), 17 <= p <= 251: the same route with the panel in 16-bit lanes,
//     reduced after every pivot step, and the rest update in 32-bit lanes;
//   * GF(2): 64 columns per word, panels of one word per row; eliminating
//     with pivot row i is an XOR of row i, minus its bit c, into every row
//     with bit c set (that bit then holds the transformation entry, 1); the
//     rest of a row is updated once per panel by XORs of the panel's pivot
//     rows, four at a time through 16-entry tables of their combinations;
//   * the search for the next column's pivot row is fused into the update of
//     the rows (each thread tests the entry it has just written), so a pivot
//     step is one pass and three CTA barriers.
// The matrix lives in the workspace (HBM / L2).
#include "gfe.h"
#include "gfe_internal.h"

#include <atomic>
#include <climits>

namespace gfe {

namespace {

// the GF(2) kernel's CTA and shared memory (dynamic)
constexpr int G2_THREADS = 1024;
constexpr int G2_WARPS = G2_THREADS / 32;
constexpr int G2_WORDS = SMALL_MAX / 64;  // words of the longest row

struct G2Shared {
    int16_t piv_of_col[SMALL_MAX];  // pivot row of column c, -1: none
    int16_t col_of_row[SMALL_MAX];  // the column row j is the pivot of, -1: none
    int16_t ups[SMALL_MAX], upsbar[SMALL_MAX], rho[SMALL_MAX], rhobar[SMALL_MAX];
    uint64_t P[SMALL_MAX];            // the panel: word pw of every row
    uint64_t OLD[64][G2_WORDS];       // this panel's pivot rows before its update
    uint64_t T[16][16][G2_WORDS];     // T[g][t]: XOR of OLD rows 4g + b over the set bits b of t
    int16_t piv_row[64], piv_pc[64];  // this panel's pivots: row, bit in the panel word
    int wmin[G2_WARPS];
    int r, kp;
};

// minimum of v over the CTA of WARPS warps (every thread calls it, every
// thread gets it); wmin holds WARPS ints of shared memory
template <int WARPS>
__device__ __forceinline__ int cta_min(int v, int *wmin) {
    v = __reduce_min_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    int r = wmin[0];
#pragma unroll
    for (int w = 1; w < WARPS; ++w) r = min(r, wmin[w]);
    __syncthreads();
    return r;
}

// warp 0 / warp 1: split 0..len-1 by flag[x] >= 0 into yes (ascending) and
// no (ascending) lists; returns the number of yes entries (on every lane)
__device__ int split_list(const int16_t *flag, int len, int16_t *yes, int16_t *no) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int base = 0; base < len; base += 32) {
        const int x = base + lane;
        const bool f = x < len && flag[x] >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (x < len) {
            if (f) yes[cnt + before] = (int16_t)x;
            else no[x - cnt - before] = (int16_t)x;
        }
        cnt += __popc(bal);
    }
    return cnt;
}

__device__ __forceinline__ uint32_t red4(uint32_t w, const uint8_t *red) {
    return (uint32_t)red[w & 0xFF] | ((uint32_t)red[(w >> 8) & 0xFF] << 8) | ((uint32_t)red[(w >> 16) & 0xFF] << 16) |
           ((uint32_t)red[w >> 24] << 24);
}

// byte q (0..15) of a 16-byte vector
__device__ __forceinline__ uint32_t byte_of(const uint4 &v, int q) {
    const uint32_t x = q < 4 ? v.x : (q < 8 ? v.y : (q < 12 ? v.z : v.w));
    return (x >> (8 * (q & 3))) & 0xFFu;
}

// x with its byte q - base cleared when base <= q < base + 4
__device__ __forceinline__ uint32_t clear_byte(uint32_t x, int q, int base) {
    return (q >= base && q < base + 4) ? x & ~(0xFFu << (8 * (q - base))) : x;
}

// The outputs of one byte matrix from its final in-place state W (exact
// residues): r, Ups, rho, and R, M, K gathered through the index lists.
// Every thread of the CTA calls it.
template <int THREADS, class Sh>
__device__ void write_outputs_u8(const SmallJob &J, Sh &S, const uint8_t *W, int ldw) {
    constexpr int WARPS = THREADS / 32;
    const int m = J.m, n = J.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        const int r = split_list(S.piv_of_col, n, S.ups, S.upsbar);
        if (lane == 0) S.r = r;
    } else if (warp == 1) {
        split_list(S.col_of_row, m, S.rho, S.rhobar);
    }
    __syncthreads();
    const int r = S.r;
    if (tid == 0) *J.rank = r;
    for (int l = tid; l < r; l += THREADS) {
        if (J.pcols) J.pcols[l] = S.ups[l];
        if (J.prows) J.prows[l] = S.rho[l];
    }
    uint8_t *R = (uint8_t *)J.R, *M = (uint8_t *)J.M, *K = (uint8_t *)J.K;
    for (int l = warp; l < r; l += WARPS) {
        const uint8_t *src = W + S.piv_of_col[S.ups[l]] * ldw;
        if (R)
            for (int t = lane; t < n - r; t += 32) R[l * J.ldR + t] = src[S.upsbar[t]];
        if (M)
            for (int s2 = lane; s2 < r; s2 += 32) M[l * J.ldM + s2] = src[S.col_of_row[S.rho[s2]]];
    }
    if (K)
        for (int t = warp; t < m - r; t += WARPS) {
            const uint8_t *src = W + S.rhobar[t] * ldw;
            for (int s2 = lane; s2 < r; s2 += 32) K[t * J.ldK + s2] = src[S.col_of_row[S.rho[s2]]];
        }
}

// ---- GF(p), 3 <= p <= 13: one byte per entry, panels of BK columns --------
constexpr int BK = 32;             // panel width: two 16-byte vectors per row
constexpr int U8_THREADS = 1024;   // one thread per row (two rows above 1024) in the panel
constexpr int U8_WARPS = U8_THREADS / 32;

constexpr int OT = 36;             // pitch (bytes) of a column of OLDT: 32 pivots + 4 (bank spread)
struct U8Shared {
    uint8_t P[SMALL_MAX * BK];        // the panel, row j at BK j
    // this panel's pivot rows before the update, transposed: column k of the
    // matrix at OT k holds pivot rows 0..31 (zero past kp and past ldw)
    alignas(16) uint8_t OLDT[(SMALL_MAX + BK) * OT];
    alignas(16) uint8_t stage[U8_WARPS][16 * BK];  // per warp: a 16 x 32 tile of products mod p
    int16_t piv_of_col[SMALL_MAX];    // pivot row of column c, -1: none
    int16_t col_of_row[SMALL_MAX];    // the column row j is the pivot of, -1: none
    int16_t ups[SMALL_MAX], upsbar[SMALL_MAX], rho[SMALL_MAX], rhobar[SMALL_MAX];
    alignas(16) uint8_t prow[BK];     // the scaled pivot row, panel part
    alignas(16) uint8_t coef[U8_WARPS][BK];  // per warp: the row's coefficients of the pivot rows
    int16_t piv_row[BK], piv_pc[BK];  // this panel's pivots: row, panel column
    uint8_t red[256];                 // x mod p
    uint8_t inv[16];                  // a^-1 mod p
    int wmin[U8_WARPS];
    int r, kp;
};

// x mod p in both 16-bit lanes of w (lanes < 2^16); rcp = ceil(2^32 / p)
__device__ __forceinline__ uint32_t mod_lanes(uint32_t w, uint32_t p, uint32_t rcp) {
    uint32_t lo = w & 0xFFFFu, hi = w >> 16;
    lo -= p * __umulhi(lo, rcp);
    hi -= p * __umulhi(hi, rcp);
    return lo | (hi << 16);
}

__device__ void small_u8(const SmallJob &J, U8Shared &S) {
    const int m = J.m, n = J.n, p = J.p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint8_t *W = (uint8_t *)J.W;
    const int ldw = (int)J.ldw;  // multiple of 16, >= n, <= SMALL_MAX
    const uint8_t *A = (const uint8_t *)J.A;
    const uint32_t rcp = (uint32_t)((0x100000000ull + (uint64_t)p - 1) / (uint64_t)p);
    for (int x = tid; x < 256; x += U8_THREADS) S.red[x] = (uint8_t)(x % p);
    if (tid < 16) {
        int v = 0;
        for (int y = 1; y < p; ++y)
            if ((tid % p) * y % p == 1) v = y;
        S.inv[tid] = (uint8_t)v;
    }
    for (int c = tid; c < n; c += U8_THREADS) S.piv_of_col[c] = -1;
    for (int j = tid; j < m; j += U8_THREADS) S.col_of_row[j] = -1;
    __syncthreads();
    // A -> W, residues in [0, p), zero padding up to ldw
    const int vpr = ldw >> 4;
    for (int v = tid; v < m * vpr; v += U8_THREADS) {
        const int j = v / vpr, k0 = (v - j * vpr) << 4;
        uint32_t o[4] = {0u, 0u, 0u, 0u};
        const uint8_t *a = A + (int64_t)j * J.lda;
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (k0 + q < n) o[q >> 2] |= (uint32_t)S.red[a[k0 + q]] << (8 * (q & 3));
        *(uint4 *)(W + j * ldw + k0) = make_uint4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();

    const int klazy = (255 - (p - 1)) / ((p - 1) * (p - 1));
    for (int c0 = 0; c0 < n; c0 += BK) {
        const int kw = min(BK, n - c0);
        // panel load (its second vector may lie past the row pitch: zeros)
        for (int v = tid; v < 2 * m; v += U8_THREADS) {
            const int j = v >> 1, k = c0 + 16 * (v & 1);
            *(uint4 *)(S.P + j * BK + 16 * (v & 1)) =
                k < ldw ? *(const uint4 *)(W + j * ldw + k) : make_uint4(0u, 0u, 0u, 0u);
        }
        if (tid == 0) S.kp = 0;
        __syncthreads();
        // panel elimination, column by column
        int steps = 0, known = INT_MAX;
        bool have_known = false;
        for (int cc = 0; cc < kw; ++cc) {
            int i;
            if (have_known) {
                i = known;
            } else {
                int best = INT_MAX;
                for (int j = tid; j < m; j += U8_THREADS)
                    if (S.col_of_row[j] < 0 && S.red[S.P[j * BK + cc]]) {
                        best = j;
                        break;
                    }
                i = cta_min<U8_WARPS>(best, S.wmin);
            }
            have_known = false;
            if (i == INT_MAX) continue;
            const int s = p - S.inv[S.red[S.P[i * BK + cc]]];
            if (tid < BK)
                S.prow[tid] = tid == cc ? (uint8_t)s : (tid < kw ? S.red[s * S.red[S.P[i * BK + tid]]] : (uint8_t)0);
            if (tid == 0) {
                S.piv_of_col[c0 + cc] = (int16_t)i;
                S.col_of_row[i] = (int16_t)(c0 + cc);
                S.piv_row[S.kp] = (int16_t)i;
                S.piv_pc[S.kp] = (int16_t)cc;
                S.kp = S.kp + 1;
            }
            __syncthreads();
            const bool reduce = ++steps >= klazy;
            if (reduce) steps = 0;
            const int c1 = cc + 1;
            int best = INT_MAX;
            const uint4 pv0 = *(const uint4 *)(S.prow), pv1 = *(const uint4 *)(S.prow + 16);
            for (int j = tid; j < m; j += U8_THREADS) {
                uint4 *row = (uint4 *)(S.P + j * BK);
                if (j == i) {
                    row[0] = pv0;
                    row[1] = pv1;
                    continue;
                }
                const uint32_t f = S.red[S.P[j * BK + cc]];
                const bool cand = S.col_of_row[j] < 0 && c1 < kw;
                if (f == 0 && !reduce) {
                    if (cand && S.red[S.P[j * BK + c1]]) best = min(best, j);
                    continue;
                }
                uint4 w0 = row[0], w1 = row[1];
                w0.x = clear_byte(w0.x, cc, 0);
                w0.y = clear_byte(w0.y, cc, 4);
                w0.z = clear_byte(w0.z, cc, 8);
                w0.w = clear_byte(w0.w, cc, 12);
                w1.x = clear_byte(w1.x, cc, 16);
                w1.y = clear_byte(w1.y, cc, 20);
                w1.z = clear_byte(w1.z, cc, 24);
                w1.w = clear_byte(w1.w, cc, 28);
                w0.x += f * pv0.x;
                w0.y += f * pv0.y;
                w0.z += f * pv0.z;
                w0.w += f * pv0.w;
                w1.x += f * pv1.x;
                w1.y += f * pv1.y;
                w1.z += f * pv1.z;
                w1.w += f * pv1.w;
                if (reduce) {
                    w0.x = red4(w0.x, S.red);
                    w0.y = red4(w0.y, S.red);
                    w0.z = red4(w0.z, S.red);
                    w0.w = red4(w0.w, S.red);
                    w1.x = red4(w1.x, S.red);
                    w1.y = red4(w1.y, S.red);
                    w1.z = red4(w1.z, S.red);
                    w1.w = red4(w1.w, S.red);
                }
                row[0] = w0;
                row[1] = w1;
                if (cand && (c1 < 16 ? S.red[byte_of(w0, c1)] : S.red[byte_of(w1, c1 - 16)])) best = min(best, j);
            }
            const int nx = cta_min<U8_WARPS>(best, S.wmin);
            if (nx != INT_MAX) {
                known = nx;
                have_known = true;
            }
        }
        // the panel exactly reduced
        for (int v = tid; v < 2 * m; v += U8_THREADS) {
            uint4 *q = (uint4 *)(S.P + 16 * v);
            uint4 w = *q;
            w.x = red4(w.x, S.red);
            w.y = red4(w.y, S.red);
            w.z = red4(w.z, S.red);
            w.w = red4(w.w, S.red);
            *q = w;
        }
        const int kp = S.kp;  // written before the last barrier of the loop
        if (kp > 0) {
            // the pivot rows as they were before this panel's operations,
            // transposed (warp: 16 columns; lane q: pivot row q), zero past kp
            // and past ldw up to a whole 32-column block
            const int ncols = (ldw + BK - 1) / BK * BK;
            for (int k0 = warp * 16; k0 < ncols; k0 += U8_WARPS * 16) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (lane < kp && k0 < ldw) v = *(const uint4 *)(W + S.piv_row[lane] * ldw + k0);
                const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int t = 0; t < 16; ++t) S.OLDT[(k0 + t) * OT + lane] = (uint8_t)(vv[t >> 2] >> (8 * (t & 3)));
            }
            __syncthreads();
            // every row: rest += sum_q coef_q * OLD_q, coef_q = P[j][pivot column q] - [j = pivot row q],
            // as a product (rows x 32) (32 x columns) on the tensor cores: int8 mma.sync m16n8k32 with
            // int32 accumulation (at most 32 * 12 * 12 < 2^13), then mod p, then + the row's entry mod p.
            // A warp takes 16 rows and every 32-column block but the panel's own (those come from P).
            const int gid = lane >> 2, tig = lane & 3;
            const uint32_t pppp = (uint32_t)p * 0x01010101u;
            uint8_t *st = S.stage[warp];
            for (int r0 = warp * 16; r0 < m; r0 += U8_WARPS * 16) {
                // A fragment: rows r0 + gid (a0, a2) and r0 + gid + 8 (a1, a3), coefficients
                // q = 4 tig .. 4 tig + 3 (a0, a1) and 16 + 4 tig .. (a2, a3)
                uint32_t a[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int j = r0 + gid + ((h & 1) ? 8 : 0);
                    const int qb = ((h & 2) ? 16 : 0) + 4 * tig;
                    uint32_t w = 0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int q = qb + i;
                        uint32_t cq = 0;
                        if (j < m && q < kp) {
                            cq = S.P[j * BK + S.piv_pc[q]];
                            if (S.piv_row[q] == j) cq = cq ? cq - 1 : (uint32_t)(p - 1);
                        }
                        w |= cq << (8 * i);
                    }
                    a[h] = w;
                }
                if (!__any_sync(0xffffffffu, (a[0] | a[1] | a[2] | a[3]) != 0u)) continue;
                for (int cb = 0; cb < ncols; cb += BK) {
                    if (cb == c0) continue;  // the panel's own columns
                    // four n8 steps of the 16 x 32 tile; the products mod p staged as bytes
#pragma unroll
                    for (int s8 = 0; s8 < 4; ++s8) {
                        const uint8_t *bcol = S.OLDT + (cb + 8 * s8 + gid) * OT + 4 * tig;
                        const uint32_t b0 = *(const uint32_t *)bcol, b1 = *(const uint32_t *)(bcol + 16);
                        int d0 = 0, d1 = 0, d2 = 0, d3 = 0;
                        asm volatile(
                            "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                            "{%8,%9}, {%0,%1,%2,%3};"
                            : "+r"(d0), "+r"(d1), "+r"(d2), "+r"(d3)
                            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
                        // d0, d1: row gid, columns 8 s8 + 2 tig + {0, 1}; d2, d3: row gid + 8
                        const uint32_t e0 = (uint32_t)d0 - (uint32_t)p * __umulhi((uint32_t)d0, rcp);
                        const uint32_t e1 = (uint32_t)d1 - (uint32_t)p * __umulhi((uint32_t)d1, rcp);
                        const uint32_t e2 = (uint32_t)d2 - (uint32_t)p * __umulhi((uint32_t)d2, rcp);
                        const uint32_t e3 = (uint32_t)d3 - (uint32_t)p * __umulhi((uint32_t)d3, rcp);
                        *(uint16_t *)(st + gid * BK + 8 * s8 + 2 * tig) = (uint16_t)(e0 | (e1 << 8));
                        *(uint16_t *)(st + (gid + 8) * BK + 8 * s8 + 2 * tig) = (uint16_t)(e2 | (e3 << 8));
                    }
                    __syncwarp();
                    // lane: row r0 + lane / 2, 16 columns from cb + 16 (lane & 1)
                    const int j = r0 + (lane >> 1), k = cb + 16 * (lane & 1);
                    if (j < m && k < ldw) {
                        const uint4 pr = *(const uint4 *)(st + (lane >> 1) * BK + 16 * (lane & 1));
                        uint4 *wp = (uint4 *)(W + j * ldw + k);
                        uint4 w = *wp;
                        // entries and products are below p: their sum is below 2p, one correction
                        uint32_t x[4] = {w.x + pr.x, w.y + pr.y, w.z + pr.z, w.w + pr.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) x[h] -= __vcmpgeu4(x[h], pppp) & pppp;
                        *wp = make_uint4(x[0], x[1], x[2], x[3]);
                    }
                    __syncwarp();
                }
            }
        }
        // the panel back into W
        for (int v = tid; v < 2 * m; v += U8_THREADS) {
            const int j = v >> 1, k = c0 + 16 * (v & 1);
            if (k < ldw) *(uint4 *)(W + j * ldw + k) = *(const uint4 *)(S.P + j * BK + 16 * (v & 1));
        }
        __syncthreads();
    }
    write_outputs_u8<U8_THREADS>(J, S, W, ldw);
}

// ---- GF(p), 17 <= p <= 251: one byte per entry, panels of BK columns held
// as 16-bit lanes (a product (p-1)^2 no longer fits a byte) -----------------
// Same route as k_ech_small_u8.  In the panel every pivot step is reduced at
// once ((p-1) + (p-1)^2 < 2^16); the rest update accumulates the kp products
// of an entry in a 32-bit lane ((p-1) + 32 (p-1)^2 < 2^21) and reduces once.
constexpr int WP_THREADS = 1024;
constexpr int WP_WARPS = WP_THREADS / 32;

struct WShared {
    uint16_t P[SMALL_MAX * BK];       // the panel, row j at BK j, exact residues
    uint8_t OLD[BK * SMALL_MAX];      // this panel's pivot rows before the update (ldw apart)
    int16_t piv_of_col[SMALL_MAX];
    int16_t col_of_row[SMALL_MAX];
    int16_t ups[SMALL_MAX], upsbar[SMALL_MAX], rho[SMALL_MAX], rhobar[SMALL_MAX];
    alignas(16) uint16_t prow[BK];
    alignas(16) uint8_t coef[WP_WARPS][BK];
    int16_t piv_row[BK], piv_pc[BK];
    uint8_t inv[256];
    int wmin[WP_WARPS];
    int r, kp;
};

// x mod p for x < 2^21 (rcp = ceil(2^32 / p))
__device__ __forceinline__ uint32_t mod_small(uint32_t x, uint32_t p, uint32_t rcp) {
    return x - p * __umulhi(x, rcp);
}

__device__ void small_w(const SmallJob &J, WShared &S) {
    const int m = J.m, n = J.n, p = J.p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint8_t *W = (uint8_t *)J.W;
    const int ldw = (int)J.ldw;
    const uint8_t *A = (const uint8_t *)J.A;
    const uint32_t up = (uint32_t)p;
    const uint32_t rcp = (uint32_t)((0x100000000ull + (uint64_t)p - 1) / (uint64_t)p);
    for (int a = tid; a < 256; a += WP_THREADS) {
        int v = 0;
        if (a > 0 && a < p)
            for (int y = 1; y < p; ++y)
                if (a * y % p == 1) {
                    v = y;
                    break;
                }
        S.inv[a] = (uint8_t)v;
    }
    for (int c = tid; c < n; c += WP_THREADS) S.piv_of_col[c] = -1;
    for (int j = tid; j < m; j += WP_THREADS) S.col_of_row[j] = -1;
    __syncthreads();
    const int vpr = ldw >> 4;
    for (int v = tid; v < m * vpr; v += WP_THREADS) {
        const int j = v / vpr, k0 = (v - j * vpr) << 4;
        uint32_t o[4] = {0u, 0u, 0u, 0u};
        const uint8_t *a = A + (int64_t)j * J.lda;
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (k0 + q < n) o[q >> 2] |= mod_small(a[k0 + q], up, rcp) << (8 * (q & 3));
        *(uint4 *)(W + j * ldw + k0) = make_uint4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();

    for (int c0 = 0; c0 < n; c0 += BK) {
        const int kw = min(BK, n - c0);
        // panel load: 16 bytes -> 16 lanes of 16 bits (past the row pitch: zeros)
        for (int v = tid; v < 2 * m; v += WP_THREADS) {
            const int j = v >> 1, k = c0 + 16 * (v & 1);
            uint4 b = k < ldw ? *(const uint4 *)(W + j * ldw + k) : make_uint4(0u, 0u, 0u, 0u);
            uint4 *dst = (uint4 *)(S.P + j * BK + 16 * (v & 1));
            dst[0] = make_uint4(__byte_perm(b.x, 0, 0x4140), __byte_perm(b.x, 0, 0x4342), __byte_perm(b.y, 0, 0x4140),
                                __byte_perm(b.y, 0, 0x4342));
            dst[1] = make_uint4(__byte_perm(b.z, 0, 0x4140), __byte_perm(b.z, 0, 0x4342), __byte_perm(b.w, 0, 0x4140),
                                __byte_perm(b.w, 0, 0x4342));
        }
        if (tid == 0) S.kp = 0;
        __syncthreads();
        int known = INT_MAX;
        bool have_known = false;
        for (int cc = 0; cc < kw; ++cc) {
            int i;
            if (have_known) {
                i = known;
            } else {
                int best = INT_MAX;
                for (int j = tid; j < m; j += WP_THREADS)
                    if (S.col_of_row[j] < 0 && S.P[j * BK + cc]) {
                        best = j;
                        break;
                    }
                i = cta_min<WP_WARPS>(best, S.wmin);
            }
            have_known = false;
            if (i == INT_MAX) continue;
            const uint32_t s = up - S.inv[S.P[i * BK + cc]];
            if (tid < BK)
                S.prow[tid] = tid == cc ? (uint16_t)s : (tid < kw ? (uint16_t)mod_small(s * S.P[i * BK + tid], up, rcp) : 0);
            if (tid == 0) {
                S.piv_of_col[c0 + cc] = (int16_t)i;
                S.col_of_row[i] = (int16_t)(c0 + cc);
                S.piv_row[S.kp] = (int16_t)i;
                S.piv_pc[S.kp] = (int16_t)cc;
                S.kp = S.kp + 1;
            }
            __syncthreads();
            const int c1 = cc + 1;
            int best = INT_MAX;
            const uint4 *pv = (const uint4 *)S.prow;
            for (int j = tid; j < m; j += WP_THREADS) {
                uint4 *row = (uint4 *)(S.P + j * BK);
                if (j == i) {
#pragma unroll
                    for (int h = 0; h < 4; ++h) row[h] = pv[h];
                    continue;
                }
                const uint32_t f = S.P[j * BK + cc];
                const bool cand = S.col_of_row[j] < 0 && c1 < kw;
                if (f == 0) {
                    if (cand && S.P[j * BK + c1]) best = min(best, j);
                    continue;
                }
#pragma unroll
                for (int h = 0; h < 4; ++h) {  // lanes 8h .. 8h+7
                    uint4 w = row[h];
                    const uint4 q = pv[h];
                    const int l = cc - 8 * h;  // lane of column cc in this vector, if 0 <= l < 8
                    w.x = (l == 0) ? w.x & 0xFFFF0000u : ((l == 1) ? w.x & 0x0000FFFFu : w.x);
                    w.y = (l == 2) ? w.y & 0xFFFF0000u : ((l == 3) ? w.y & 0x0000FFFFu : w.y);
                    w.z = (l == 4) ? w.z & 0xFFFF0000u : ((l == 5) ? w.z & 0x0000FFFFu : w.z);
                    w.w = (l == 6) ? w.w & 0xFFFF0000u : ((l == 7) ? w.w & 0x0000FFFFu : w.w);
                    w.x = mod_lanes(w.x + f * q.x, up, rcp);
                    w.y = mod_lanes(w.y + f * q.y, up, rcp);
                    w.z = mod_lanes(w.z + f * q.z, up, rcp);
                    w.w = mod_lanes(w.w + f * q.w, up, rcp);
                    row[h] = w;
                }
                if (cand && S.P[j * BK + c1]) best = min(best, j);
            }
            const int nx = cta_min<WP_WARPS>(best, S.wmin);
            if (nx != INT_MAX) {
                known = nx;
                have_known = true;
            }
        }
        const int kp = S.kp;
        if (kp > 0) {
            for (int v = tid; v < kp * vpr; v += WP_THREADS) {
                const int q = v / vpr, k0 = (v - q * vpr) << 4;
                *(uint4 *)(S.OLD + q * ldw + k0) = *(const uint4 *)(W + S.piv_row[q] * ldw + k0);
            }
            __syncthreads();
            for (int j = warp; j < m; j += WP_WARPS) {
                uint32_t cq = 0;
                if (lane < kp) {
                    cq = S.P[j * BK + S.piv_pc[lane]];
                    if (S.piv_row[lane] == j) cq = cq ? cq - 1 : up - 1;
                    S.coef[warp][lane] = (uint8_t)cq;
                }
                if (!__any_sync(0xffffffffu, cq != 0)) continue;
                __syncwarp();
                uint8_t *row = W + j * ldw;
                for (int k0 = lane << 3; k0 < ldw; k0 += 256) {
                    if (k0 >= c0 && k0 < c0 + BK) continue;
                    const uint2 w = *(const uint2 *)(row + k0);
                    uint32_t acc[8];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        acc[e] = (w.x >> (8 * e)) & 0xFFu;
                        acc[4 + e] = (w.y >> (8 * e)) & 0xFFu;
                    }
                    for (int q4 = 0; q4 < kp; q4 += 4) {
                        const uint32_t c4 = *(const uint32_t *)(&S.coef[warp][q4]);
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const uint32_t c = (c4 >> (8 * t)) & 0xFFu;
                            if (q4 + t < kp && c) {
                                const uint2 v = *(const uint2 *)(S.OLD + (q4 + t) * ldw + k0);
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    acc[e] += c * ((v.x >> (8 * e)) & 0xFFu);
                                    acc[4 + e] += c * ((v.y >> (8 * e)) & 0xFFu);
                                }
                            }
                        }
                    }
                    uint2 out = make_uint2(0u, 0u);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        out.x |= mod_small(acc[e], up, rcp) << (8 * e);
                        out.y |= mod_small(acc[4 + e], up, rcp) << (8 * e);
                    }
                    *(uint2 *)(row + k0) = out;
                }
                __syncwarp();
            }
        }
        // the panel back into W as bytes
        for (int v = tid; v < 2 * m; v += WP_THREADS) {
            const int j = v >> 1, k = c0 + 16 * (v & 1);
            if (k < ldw) {
                const uint4 *src = (const uint4 *)(S.P + j * BK + 16 * (v & 1));
                const uint4 a = src[0], b = src[1];
                *(uint4 *)(W + j * ldw + k) = make_uint4(__byte_perm(a.x, a.y, 0x6420), __byte_perm(a.z, a.w, 0x6420),
                                                         __byte_perm(b.x, b.y, 0x6420), __byte_perm(b.z, b.w, 0x6420));
            }
        }
        __syncthreads();
    }
    write_outputs_u8<WP_THREADS>(J, S, W, ldw);
}

// ---- GF(2), 64 columns per word ---------------------------------------------
__device__ void small_gf2(const SmallJob &J, G2Shared &S) {
    const int m = J.m, n = J.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t *W = (uint64_t *)J.W;
    const int ldq = (int)(J.ldw >> 3);  // words per workspace row, >= nw, <= G2_WORDS
    const int nw = (n + 63) >> 6;
    const uint64_t *A = (const uint64_t *)J.A;
    const int64_t ldaq = J.lda >> 3;
    for (int c = tid; c < n; c += G2_THREADS) S.piv_of_col[c] = -1;
    for (int j = tid; j < m; j += G2_THREADS) S.col_of_row[j] = -1;
    for (int v = tid; v < m * ldq; v += G2_THREADS) {
        const int j = v / ldq, q = v - j * ldq;
        uint64_t x = 0;
        if (q < nw) {
            x = A[j * ldaq + q];
            if (q == nw - 1 && (n & 63)) x &= (1ull << (n & 63)) - 1ull;  // input pad bits are ignored
        }
        W[(int64_t)j * ldq + q] = x;
    }
    __syncthreads();
    // panels of 64 columns: word pw of every row
    for (int pw = 0; pw < nw; ++pw) {
        const int c0 = pw << 6, kw = min(64, n - c0);
        for (int j = tid; j < m; j += G2_THREADS) S.P[j] = W[(int64_t)j * ldq + pw];
        if (tid == 0) S.kp = 0;
        __syncthreads();
        int known = INT_MAX;
        bool have_known = false;
        for (int cc = 0; cc < kw; ++cc) {
            const uint64_t cb = 1ull << cc;
            int i;
            if (have_known) {
                i = known;
            } else {
                int best = INT_MAX;
                for (int j = tid; j < m; j += G2_THREADS)
                    if (S.col_of_row[j] < 0 && (S.P[j] & cb)) {
                        best = j;
                        break;
                    }
                i = cta_min<G2_WARPS>(best, S.wmin);
            }
            have_known = false;
            if (i == INT_MAX) continue;
            // -a^-1 = 1: row i minus its bit cc (which then holds the transformation entry 1)
            const uint64_t pr = S.P[i] & ~cb;
            if (tid == 0) {
                S.piv_of_col[c0 + cc] = (int16_t)i;
                S.col_of_row[i] = (int16_t)(c0 + cc);
                S.piv_row[S.kp] = (int16_t)i;
                S.piv_pc[S.kp] = (int16_t)cc;
                S.kp = S.kp + 1;
            }
            __syncthreads();
            const int c1 = cc + 1;
            const uint64_t c1b = c1 < 64 ? 1ull << c1 : 0ull;
            int best = INT_MAX;
            for (int j = tid; j < m; j += G2_THREADS) {
                if (j == i) continue;
                uint64_t x = S.P[j];
                if (x & cb) {
                    x ^= pr;
                    S.P[j] = x;
                }
                if (c1 < kw && S.col_of_row[j] < 0 && (x & c1b)) best = min(best, j);
            }
            const int nx = cta_min<G2_WARPS>(best, S.wmin);
            if (nx != INT_MAX) {
                known = nx;
                have_known = true;
            }
        }
        const int kp = S.kp;
        if (kp > 0) {
            for (int v = tid; v < kp * nw; v += G2_THREADS) {
                const int q = v / nw, w = v - q * nw;
                S.OLD[q][w] = W[(int64_t)S.piv_row[q] * ldq + w];
            }
            __syncthreads();
            const int ng = (kp + 3) >> 2;
            for (int v = tid; v < ng * 16 * nw; v += G2_THREADS) {
                const int g = v / (16 * nw), rem = v - g * 16 * nw, t = rem / nw, w = rem - t * nw;
                uint64_t x = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (((t >> b) & 1) && 4 * g + b < kp) x ^= S.OLD[4 * g + b][w];
                S.T[g][t][w] = x;
            }
            __syncthreads();
            // every row: rest ^= sum of the pivot rows its coefficient bits select
            // (coefficient q: bit piv_pc[q] of its panel word, minus 1 on pivot row q itself)
            for (int j = warp; j < m; j += G2_WARPS) {
                const uint64_t pj = S.P[j];
                const bool b0 = lane < kp && ((((pj >> S.piv_pc[lane]) & 1ull) != 0) != (S.piv_row[lane] == j));
                const bool b1 =
                    lane + 32 < kp && ((((pj >> S.piv_pc[lane + 32]) & 1ull) != 0) != (S.piv_row[lane + 32] == j));
                const uint64_t cbits =
                    (uint64_t)__ballot_sync(0xffffffffu, b0) | ((uint64_t)__ballot_sync(0xffffffffu, b1) << 32);
                if (!cbits) continue;
                if (lane < nw && lane != pw) {
                    uint64_t x = W[(int64_t)j * ldq + lane];
                    for (int g = 0; g < ng; ++g) {
                        const int t = (int)((cbits >> (4 * g)) & 15ull);
                        if (t) x ^= S.T[g][t][lane];
                    }
                    W[(int64_t)j * ldq + lane] = x;
                }
            }
        }
        for (int j = tid; j < m; j += G2_THREADS) W[(int64_t)j * ldq + pw] = S.P[j];
        __syncthreads();
    }
    if (warp == 0) {
        const int r = split_list(S.piv_of_col, n, S.ups, S.upsbar);
        if (lane == 0) S.r = r;
    } else if (warp == 1) {
        split_list(S.col_of_row, m, S.rho, S.rhobar);
    }
    __syncthreads();
    const int r = S.r;
    if (tid == 0) *J.rank = r;
    for (int l = tid; l < r; l += G2_THREADS) {
        if (J.pcols) J.pcols[l] = S.ups[l];
        if (J.prows) J.prows[l] = S.rho[l];
    }
    // bit t of output word o gathers column idx[64 o + t] of the source row
    auto gather = [&](const uint64_t *src, const int16_t *idx, int len, uint64_t *dst, bool viaRho) {
        for (int o = lane; o < (len + 63) >> 6; o += 32) {
            uint64_t v = 0;
            const int lim = min(64, len - 64 * o);
            for (int t = 0; t < lim; ++t) {
                int col = idx[64 * o + t];
                if (viaRho) col = S.col_of_row[col];
                v |= ((src[col >> 6] >> (col & 63)) & 1ull) << t;
            }
            dst[o] = v;
        }
    };
    uint64_t *R = (uint64_t *)J.R, *M = (uint64_t *)J.M, *K = (uint64_t *)J.K;
    for (int l = warp; l < r; l += G2_WARPS) {
        const uint64_t *src = W + (int64_t)S.piv_of_col[S.ups[l]] * ldq;
        if (R) gather(src, S.upsbar, n - r, R + l * (J.ldR >> 3), false);
        if (M) gather(src, S.rho, r, M + l * (J.ldM >> 3), true);
    }
    if (K)
        for (int t = warp; t < m - r; t += G2_WARPS)
            gather(W + (int64_t)S.rhobar[t] * ldq, S.rho, r, K + t * (J.ldK >> 3), true);
}

// One persistent launch per kernel kind: a CTA per SM claims the next matrix
// of the table (largest first) from an atomic counter until none is left.
template <class Sh, void (*JOB)(const SmallJob &, Sh &)>
__device__ __forceinline__ void run_jobs(const SmallJob *jobs, int count, int *next) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sh &S = *reinterpret_cast<Sh *>(smem_raw);
    __shared__ int job;
    for (;;) {
        if (threadIdx.x == 0) job = atomicAdd(next, 1);
        __syncthreads();
        const int q = job;
        if (q >= count) break;
        const SmallJob J = jobs[q];
        if (J.m > 0 && J.n > 0) JOB(J, S);
        __syncthreads();  // the shared state and `job` are reused by the next matrix
    }
}

__global__ void __launch_bounds__(U8_THREADS, 1) k_ech_small_u8(const SmallJob *jobs, int count, int *next) {
    run_jobs<U8Shared, small_u8>(jobs, count, next);
}
__global__ void __launch_bounds__(WP_THREADS, 1) k_ech_small_w(const SmallJob *jobs, int count, int *next) {
    run_jobs<WShared, small_w>(jobs, count, next);
}
__global__ void __launch_bounds__(G2_THREADS, 1) k_ech_small_gf2(const SmallJob *jobs, int count, int *next) {
    run_jobs<G2Shared, small_gf2>(jobs, count, next);
}

}  // namespace

cudaError_t ech_small_batch(const Launch &L, const SmallJob *jobs_dev, int count, int kind, int *next) {
    if (count <= 0) return cudaSuccess;
    // dynamic shared memory and the SM count, once per device
    static std::atomic<int> sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev].load()) {
        cudaFuncSetAttribute(k_ech_small_u8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(U8Shared));
        cudaFuncSetAttribute(k_ech_small_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WShared));
        cudaFuncSetAttribute(k_ech_small_gf2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(G2Shared));
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        sms[dev].store(n);
    }
    const int grid = count < sms[dev].load() ? count : sms[dev].load();  // one CTA per SM (their shared memory)
    cudaEvent_t ev;
    prof_begin(L, K_ECH, &ev);
    e = cudaMemsetAsync(next, 0, sizeof(int), L.st);
    if (e != cudaSuccess) return e;
    if (kind == SMALL_GF2) k_ech_small_gf2<<<grid, G2_THREADS, sizeof(G2Shared), L.st>>>(jobs_dev, count, next);
    else if (kind == SMALL_BYTES) k_ech_small_u8<<<grid, U8_THREADS, sizeof(U8Shared), L.st>>>(jobs_dev, count, next);
    else k_ech_small_w<<<grid, WP_THREADS, sizeof(WShared), L.st>>>(jobs_dev, count, next);
    e = cudaGetLastError();
    prof_end(L, K_ECH, ev, 0, 0, count, 0);
    return e;
}

}  // namespace gfe
