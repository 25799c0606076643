// Batched form for small matrices: ONE launch echelonises a whole list of
// independent matrices (rows and columns up to SMALL_MAX), one CTA per
// matrix, the entire method inside the CTA.  For matrices this small the
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
//   * GF(p), 3 <= p <= 13: one byte per entry, four entries per 32-bit word,
//     one integer multiply-add updates four; entries are reduced lazily
//     (every klazy pivot steps, while p-1 + klazy (p-1)^2 <= 255 keeps every
//     byte below 256), and every test of an entry for zero reduces it first;
//   * GF(2): 64 columns per word; eliminating with pivot row i is an XOR of
//     row i, minus its bit c, into every row with bit c set (that bit then
//     holds the transformation entry, 1);
//   * the search for the next column's pivot row is fused into the update of
//     the rows (each warp tests the entry it has just written), so a pivot
//     step is one pass over the matrix and three CTA barriers.
// The matrix lives in the workspace (HBM / L2); one warp updates one row
// with 16-byte accesses (bytes) or one word per lane (GF(2)).
#include "gfe.h"
#include "gfe_internal.h"

#include <climits>

namespace gfe {

namespace {

constexpr int SM_THREADS = 512;
constexpr int SM_WARPS = SM_THREADS / 32;

struct SmallShared {
    int16_t piv_of_col[SMALL_MAX];  // pivot row of column c, -1: none
    int16_t col_of_row[SMALL_MAX];  // the column row j is the pivot of, -1: none
    int16_t ups[SMALL_MAX], upsbar[SMALL_MAX], rho[SMALL_MAX], rhobar[SMALL_MAX];
    alignas(16) uint8_t prow[SMALL_MAX];  // the scaled pivot row (GF(2): its words)
    uint8_t red[256];                     // x mod p
    uint8_t inv[16];                      // a^-1 mod p
    int wmin[SM_WARPS];
    int r;
};

// minimum of v over the CTA (every thread calls it, every thread gets it)
__device__ __forceinline__ int cta_min(int v, SmallShared &S) {
    v = __reduce_min_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) S.wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    int r = S.wmin[0];
#pragma unroll
    for (int w = 1; w < SM_WARPS; ++w) r = min(r, S.wmin[w]);
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

// ---- GF(p), 3 <= p <= 13, one byte per entry -------------------------------
__device__ void small_u8(const SmallJob &J, SmallShared &S) {
    const int m = J.m, n = J.n, p = J.p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint8_t *W = (uint8_t *)J.W;
    const int64_t ldw = J.ldw;  // multiple of 16, >= n, <= SMALL_MAX
    const uint8_t *A = (const uint8_t *)J.A;
    for (int x = tid; x < 256; x += SM_THREADS) S.red[x] = (uint8_t)(x % p);
    if (tid < 16) {
        int v = 0;
        for (int y = 1; y < p; ++y)
            if ((tid % p) * y % p == 1) v = y;
        S.inv[tid] = (uint8_t)v;
    }
    for (int c = tid; c < n; c += SM_THREADS) S.piv_of_col[c] = -1;
    for (int j = tid; j < m; j += SM_THREADS) S.col_of_row[j] = -1;
    __syncthreads();
    // A -> W, residues in [0, p), zero padding up to ldw
    const int vpr = (int)(ldw >> 4);
    for (int v = tid; v < m * vpr; v += SM_THREADS) {
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
    int steps = 0;
    int known = INT_MAX;  // pivot row of column c found while updating for c - 1
    bool have_known = false;
    for (int c = 0; c < n; ++c) {
        int i;
        if (have_known) {
            i = known;
        } else {
            int best = INT_MAX;
            for (int j = tid; j < m; j += SM_THREADS)
                if (S.col_of_row[j] < 0 && S.red[W[j * ldw + c]]) {
                    best = j;
                    break;
                }
            i = cta_min(best, S);
        }
        have_known = false;
        if (i == INT_MAX) continue;  // no pivot in column c
        // pivot row scaled so that its pivot is -1; position c keeps the
        // transformation entry s = -a^-1
        const uint8_t *wi = W + i * ldw;
        const int s = p - S.inv[S.red[wi[c]]];
        for (int k = tid; k < ldw; k += SM_THREADS)
            S.prow[k] = k == c ? (uint8_t)s : (k < n ? S.red[s * S.red[wi[k]]] : (uint8_t)0);
        if (tid == 0) {
            S.piv_of_col[c] = (int16_t)i;
            S.col_of_row[i] = (int16_t)c;
        }
        __syncthreads();
        const bool reduce = ++steps >= klazy;
        if (reduce) steps = 0;
        const int c1 = c + 1;
        int best = INT_MAX;  // topmost non-pivot row with a non-zero in column c1
        for (int j = warp; j < m; j += SM_WARPS) {
            uint8_t *row = W + j * ldw;
            if (j == i) {
                for (int k0 = lane << 4; k0 < ldw; k0 += 512) *(uint4 *)(row + k0) = *(const uint4 *)(S.prow + k0);
                continue;
            }
            const uint32_t f = __shfl_sync(0xffffffffu, lane == 0 ? (uint32_t)S.red[row[c]] : 0u, 0);
            const bool cand = S.col_of_row[j] < 0 && c1 < n;
            if (f == 0 && !reduce) {
                if (lane == 0 && cand && S.red[row[c1]]) best = min(best, j);
                continue;
            }
            for (int k0 = lane << 4; k0 < ldw; k0 += 512) {
                uint4 w = *(const uint4 *)(row + k0);
                const uint4 pv = *(const uint4 *)(S.prow + k0);
                const int q = c - k0;
                w.x = clear_byte(w.x, q, 0);
                w.y = clear_byte(w.y, q, 4);
                w.z = clear_byte(w.z, q, 8);
                w.w = clear_byte(w.w, q, 12);
                w.x += f * pv.x;
                w.y += f * pv.y;
                w.z += f * pv.z;
                w.w += f * pv.w;
                if (reduce) {
                    w.x = red4(w.x, S.red);
                    w.y = red4(w.y, S.red);
                    w.z = red4(w.z, S.red);
                    w.w = red4(w.w, S.red);
                }
                *(uint4 *)(row + k0) = w;
                if (cand && c1 >= k0 && c1 < k0 + 16 && S.red[byte_of(w, c1 - k0)]) best = min(best, j);
            }
        }
        const int nx = cta_min(best, S);
        if (nx != INT_MAX) {
            known = nx;
            have_known = true;
        }
    }
    if (steps > 0) {  // last lazy round: every entry to [0, p)
        for (int v = tid; v < m * vpr; v += SM_THREADS) {
            uint4 *q = (uint4 *)(W + (int64_t)v * 16);
            uint4 w = *q;
            w.x = red4(w.x, S.red);
            w.y = red4(w.y, S.red);
            w.z = red4(w.z, S.red);
            w.w = red4(w.w, S.red);
            *q = w;
        }
    }
    __syncthreads();
    if (warp == 0) {
        const int r = split_list(S.piv_of_col, n, S.ups, S.upsbar);
        if (lane == 0) S.r = r;
    } else if (warp == 1) {
        split_list(S.col_of_row, m, S.rho, S.rhobar);
    }
    __syncthreads();
    const int r = S.r;
    if (tid == 0) *J.rank = r;
    for (int l = tid; l < r; l += SM_THREADS) {
        if (J.pcols) J.pcols[l] = S.ups[l];
        if (J.prows) J.prows[l] = S.rho[l];
    }
    uint8_t *R = (uint8_t *)J.R, *M = (uint8_t *)J.M, *K = (uint8_t *)J.K;
    for (int l = warp; l < r; l += SM_WARPS) {
        const uint8_t *src = W + S.piv_of_col[S.ups[l]] * ldw;
        if (R)
            for (int t = lane; t < n - r; t += 32) R[l * J.ldR + t] = src[S.upsbar[t]];
        if (M)
            for (int s2 = lane; s2 < r; s2 += 32) M[l * J.ldM + s2] = src[S.col_of_row[S.rho[s2]]];
    }
    if (K)
        for (int t = warp; t < m - r; t += SM_WARPS) {
            const uint8_t *src = W + S.rhobar[t] * ldw;
            for (int s2 = lane; s2 < r; s2 += 32) K[t * J.ldK + s2] = src[S.col_of_row[S.rho[s2]]];
        }
}

// ---- GF(2), 64 columns per word ---------------------------------------------
__device__ void small_gf2(const SmallJob &J, SmallShared &S) {
    const int m = J.m, n = J.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t *W = (uint64_t *)J.W;
    const int ldq = (int)(J.ldw >> 3);  // words per workspace row, >= nw, <= 32
    const int nw = (n + 63) >> 6;
    const uint64_t *A = (const uint64_t *)J.A;
    const int64_t ldaq = J.lda >> 3;
    uint64_t *prow = (uint64_t *)S.prow;
    for (int c = tid; c < n; c += SM_THREADS) S.piv_of_col[c] = -1;
    for (int j = tid; j < m; j += SM_THREADS) S.col_of_row[j] = -1;
    for (int v = tid; v < m * ldq; v += SM_THREADS) {
        const int j = v / ldq, q = v - j * ldq;
        uint64_t x = 0;
        if (q < nw) {
            x = A[j * ldaq + q];
            if (q == nw - 1 && (n & 63)) x &= (1ull << (n & 63)) - 1ull;  // input pad bits are ignored
        }
        W[(int64_t)j * ldq + q] = x;
    }
    __syncthreads();
    int known = INT_MAX;
    bool have_known = false;
    for (int c = 0; c < n; ++c) {
        const int cw = c >> 6;
        const uint64_t cb = 1ull << (c & 63);
        int i;
        if (have_known) {
            i = known;
        } else {
            int best = INT_MAX;
            for (int j = tid; j < m; j += SM_THREADS)
                if (S.col_of_row[j] < 0 && (W[(int64_t)j * ldq + cw] & cb)) {
                    best = j;
                    break;
                }
            i = cta_min(best, S);
        }
        have_known = false;
        if (i == INT_MAX) continue;
        // -a^-1 = 1: the pivot row is row i; bit c keeps the transformation entry 1
        if (tid < nw) prow[tid] = W[(int64_t)i * ldq + tid] & (tid == cw ? ~cb : ~0ull);
        if (tid == 0) {
            S.piv_of_col[c] = (int16_t)i;
            S.col_of_row[i] = (int16_t)c;
        }
        __syncthreads();
        const int c1 = c + 1, c1w = c1 >> 6;
        const uint64_t c1b = 1ull << (c1 & 63);
        int best = INT_MAX;
        for (int j = warp; j < m; j += SM_WARPS) {
            if (j == i) continue;
            uint64_t *row = W + (int64_t)j * ldq;
            const uint64_t x = lane < nw ? row[lane] : 0ull;
            const bool f = (__shfl_sync(0xffffffffu, x, cw) & cb) != 0;
            const bool cand = S.col_of_row[j] < 0 && c1 < n;
            uint64_t y = x;
            if (f && lane < nw) {
                y = x ^ prow[lane];
                row[lane] = y;
            }
            if (cand && lane == c1w && (y & c1b)) best = min(best, j);
        }
        const int nx = cta_min(best, S);
        if (nx != INT_MAX) {
            known = nx;
            have_known = true;
        }
    }
    __syncthreads();
    if (warp == 0) {
        const int r = split_list(S.piv_of_col, n, S.ups, S.upsbar);
        if (lane == 0) S.r = r;
    } else if (warp == 1) {
        split_list(S.col_of_row, m, S.rho, S.rhobar);
    }
    __syncthreads();
    const int r = S.r;
    if (tid == 0) *J.rank = r;
    for (int l = tid; l < r; l += SM_THREADS) {
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
    for (int l = warp; l < r; l += SM_WARPS) {
        const uint64_t *src = W + (int64_t)S.piv_of_col[S.ups[l]] * ldq;
        if (R) gather(src, S.upsbar, n - r, R + l * (J.ldR >> 3), false);
        if (M) gather(src, S.rho, r, M + l * (J.ldM >> 3), true);
    }
    if (K)
        for (int t = warp; t < m - r; t += SM_WARPS)
            gather(W + (int64_t)S.rhobar[t] * ldq, S.rho, r, K + t * (J.ldK >> 3), true);
}

__global__ void __launch_bounds__(SM_THREADS) k_ech_small(const SmallJob *jobs) {
    __shared__ SmallShared S;
    const SmallJob J = jobs[blockIdx.x];
    if (J.m <= 0 || J.n <= 0) return;
    if (J.fmt == GFE_BITS64) small_gf2(J, S);
    else small_u8(J, S);
}

}  // namespace

void ech_small_batch(const Launch &L, const SmallJob *jobs_dev, int count) {
    if (count <= 0) return;
    cudaEvent_t ev;
    prof_begin(L, K_ECH, &ev);
    k_ech_small<<<count, SM_THREADS, 0, L.st>>>(jobs_dev);
    prof_end(L, K_ECH, ev, 0, 0, count, 0);
}

}  // namespace gfe
