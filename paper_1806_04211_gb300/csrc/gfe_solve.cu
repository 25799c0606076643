// Solving and null spaces from the echelon result (arXiv 1806.04211: the
// transformation matrix is what makes these available, Section 1, variant
// list; Eq. (echelon), Section 3.1):
//
//   T = (M 0; K 1) P_rho,  T A = E = (-1 R; 0 0) in the columns (Ups Ups_bar)
//
//   left null space  {y : y A = 0}: the rows r.. of T, i.e. (K 1) P_rho --
//       row t holds K[t, s] at column rho_s and 1 at column rho_bar_t;
//   right null space {x : A x = 0}: E_top x = 0 (T is invertible), row l of
//       E_top reads -x[Ups_l] + sum_j R[l, j] x[Ups_bar_j] = 0, so basis
//       vector j is 1 at Ups_bar_j and R[l, j] at Ups_l;
//   A X = B: E X = T B; column b is consistent iff (T b)[r..] =
//       K b[rho] + b[rho_bar] = 0, and then X[Ups_l] = -(M b[rho])[l] with
//       every non-pivot variable 0.
//
// Pivot sets stay on the device: a kernel finds where an index sits in the
// ascending rho / Ups by binary search, so the null spaces need no host
// round trip; solve reads only the rank, to size its multiply-adds.
#include "gfe.h"
#include "gfe_internal.h"

#include <algorithm>
#include <string>

namespace gfe {
namespace {

// s with a[s] == v, else -1 - (number of entries < v); a ascending, length r
__device__ __forceinline__ int64_t find_sorted(const int64_t *a, int64_t r, int64_t v) {
    int64_t lo = 0, hi = r;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return (lo < r && a[lo] == v) ? lo : -1 - lo;
}

// the t-th (0-based) index of 0, 1, ... that is not in the ascending a[0..r):
// t plus the number of s with a[s] - s <= t (a[s] - s counts the missing
// indices below a[s] and does not decrease)
__device__ __forceinline__ int64_t nth_missing(const int64_t *a, int64_t r, int64_t t) {
    int64_t lo = 0, hi = r;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] - mid <= t) lo = mid + 1;
        else hi = mid;
    }
    return t + lo;
}

__device__ __forceinline__ int bit_of(const uint64_t *row, int64_t c) { return (int)((row[c >> 6] >> (c & 63)) & 1u); }

constexpr int NT = 256;

// ---- left null space: N[t][x], t < m - r, x < m ----
__global__ void k_null_left_u8(int64_t m, const int64_t *rank, const int64_t *rho, const uint8_t *K, int64_t ldk,
                               uint8_t *N, int64_t ldn) {
    const int64_t r = *rank, rows = m - r;
    const int64_t x = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (x >= m) return;
    const int64_t f = find_sorted(rho, r, x);
    const int64_t nonidx = f >= 0 ? -1 : x - (-1 - f);  // index of x among the non-pivot rows
    for (int64_t t = blockIdx.y; t < rows; t += gridDim.y)
        N[t * ldn + x] = f >= 0 ? K[t * ldk + f] : (uint8_t)(nonidx == t);
}

__global__ void k_null_left_bits(int64_t m, const int64_t *rank, const int64_t *rho, const uint64_t *K, int64_t ldk,
                                 uint64_t *N, int64_t ldn, int64_t words) {
    __shared__ int64_t where[64];
    const int64_t r = *rank, rows = m - r;
    const int64_t w = blockIdx.x;
    if (threadIdx.x < 64) {
        const int64_t x = w * 64 + threadIdx.x;
        int64_t v = INT64_MIN;  // beyond m: no bit
        if (x < m) {
            const int64_t f = find_sorted(rho, r, x);
            v = f >= 0 ? f : -1 - (x - (-1 - f));  // s >= 0, or -1 - (non-pivot index)
        }
        where[threadIdx.x] = v;
    }
    __syncthreads();
    if (w >= words) return;
    for (int64_t t = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; t < rows; t += (int64_t)gridDim.y * blockDim.x) {
        const uint64_t *kr = K + t * ldk;
        uint64_t o = 0;
        for (int b = 0; b < 64; ++b) {
            const int64_t v = where[b];
            if (v == INT64_MIN) break;
            const int bit = v >= 0 ? bit_of(kr, v) : (-1 - v == t);
            o |= (uint64_t)bit << b;
        }
        N[t * ldn + w] = o;
    }
}

// ---- right null space: N[j][c], j < n - r, c < n ----
__global__ void k_null_right_u8(int64_t n, const int64_t *rank, const int64_t *ups, const uint8_t *R, int64_t ldr,
                                uint8_t *N, int64_t ldn) {
    const int64_t r = *rank, rows = n - r;
    const int64_t c = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (c >= n) return;
    const int64_t f = find_sorted(ups, r, c);
    const int64_t freeidx = f >= 0 ? -1 : c - (-1 - f);
    for (int64_t j = blockIdx.y; j < rows; j += gridDim.y)
        N[j * ldn + c] = f >= 0 ? R[f * ldr + j] : (uint8_t)(freeidx == j);
}

__global__ void k_null_right_bits(int64_t n, const int64_t *rank, const int64_t *ups, const uint64_t *R, int64_t ldr,
                                  uint64_t *N, int64_t ldn, int64_t words) {
    __shared__ int64_t where[64];
    const int64_t r = *rank, rows = n - r;
    const int64_t w = blockIdx.x;
    if (threadIdx.x < 64) {
        const int64_t c = w * 64 + threadIdx.x;
        int64_t v = INT64_MIN;
        if (c < n) {
            const int64_t f = find_sorted(ups, r, c);
            v = f >= 0 ? f : -1 - (c - (-1 - f));
        }
        where[threadIdx.x] = v;
    }
    __syncthreads();
    if (w >= words) return;
    for (int64_t j = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.y * blockDim.x) {
        uint64_t o = 0;
        for (int b = 0; b < 64; ++b) {
            const int64_t v = where[b];
            if (v == INT64_MIN) break;
            const int bit = v >= 0 ? bit_of(R + v * ldr, j) : (-1 - v == j);
            o |= (uint64_t)bit << b;
        }
        N[j * ldn + w] = o;
    }
}

// ---- solve ----
// out row t := B row (pivots ? rho[t] : rho_bar[t]), `bytes` bytes per row
__global__ void k_gather_rows_bytes(int64_t rows, int64_t bytes, const uint8_t *B, int64_t ldb, const int64_t *rho,
                                    int64_t r, bool pivots, uint8_t *out, int64_t ldo) {
    for (int64_t t = blockIdx.y; t < rows; t += gridDim.y) {
        const int64_t src = pivots ? rho[t] : nth_missing(rho, r, t);
        for (int64_t c = blockIdx.x * (int64_t)NT + threadIdx.x; c < bytes; c += (int64_t)gridDim.x * NT)
            out[t * ldo + c] = B[src * ldb + c];
    }
}

// X row c := Ups row l of -Y (c = Ups_l), else 0; u8 residues
__global__ void k_solve_x_u8(int64_t n, int64_t k, int p, const int64_t *ups, int64_t r, const uint8_t *Y,
                             int64_t ldy, uint8_t *X, int64_t ldx) {
    for (int64_t c = blockIdx.y; c < n; c += gridDim.y) {
        const int64_t f = find_sorted(ups, r, c);
        for (int64_t j = blockIdx.x * (int64_t)NT + threadIdx.x; j < k; j += (int64_t)gridDim.x * NT) {
            uint8_t v = 0;
            if (f >= 0) {
                const int y = Y[f * ldy + j];
                v = (uint8_t)(y ? p - y : 0);
            }
            X[c * ldx + j] = v;
        }
    }
}

// the same over GF(2) words (-1 = 1)
__global__ void k_solve_x_bits(int64_t n, int64_t words, const int64_t *ups, int64_t r, const uint64_t *Y,
                               int64_t ldy, uint64_t *X, int64_t ldx) {
    for (int64_t c = blockIdx.y; c < n; c += gridDim.y) {
        const int64_t f = find_sorted(ups, r, c);
        for (int64_t a = blockIdx.x * (int64_t)NT + threadIdx.x; a < words; a += (int64_t)gridDim.x * NT)
            X[c * ldx + a] = f >= 0 ? Y[f * ldy + a] : 0ull;
    }
}

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
    const int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (i < n) a[i] = v;
}

// ok[j] := 0 where column j of Z (rows x k) has a non-zero entry
__global__ void k_consistent_u8(int64_t rows, int64_t k, const uint8_t *Z, int64_t ldz, int32_t *ok) {
    for (int64_t t = blockIdx.y; t < rows; t += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)NT + threadIdx.x; j < k; j += (int64_t)gridDim.x * NT)
            if (Z[t * ldz + j]) ok[j] = 0;
}

__global__ void k_consistent_bits(int64_t rows, int64_t k, int64_t words, const uint64_t *Z, int64_t ldz,
                                  int32_t *ok) {
    for (int64_t t = blockIdx.y; t < rows; t += gridDim.y)
        for (int64_t a = blockIdx.x * (int64_t)NT + threadIdx.x; a < words; a += (int64_t)gridDim.x * NT) {
            uint64_t v = Z[t * ldz + a];
            while (v) {
                const int b = __ffsll((long long)v) - 1;
                v &= v - 1;
                if (a * 64 + b < k) ok[a * 64 + b] = 0;
            }
        }
}

inline unsigned gy(int64_t rows) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, 65535)); }
inline unsigned gx(int64_t cols) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((cols + NT - 1) / NT, 1 << 20)); }
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
inline int64_t ld64(int64_t x) { return x > 0 ? (x + 63) / 64 * 64 : 64; }
inline int64_t words_of(int64_t cols) { return (cols + 63) / 64; }
// row pitch in bytes of an API-storage scratch matrix of `cols` columns
inline int64_t api_ld(int fmt, int64_t cols) {
    return fmt == GFE_BITS64 ? std::max<int64_t>(16, (words_of(cols) + 1) / 2 * 16) : std::max<int64_t>(16, (cols + 15) / 16 * 16);
}

struct SolveLayout {
    size_t bp_api, bn_api, bp, bn, mc, kc, y, y_api, err, total;
};

SolveLayout solve_layout(int p, int fmt, int64_t m, int64_t n, int64_t k) {
    const int es = codec_bytes(codec_for(p));
    const int64_t mn = std::min(m, n), lk = ld64(k);
    SolveLayout S;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += al256(std::max<size_t>(bytes, 256));
        return o;
    };
    S.bp_api = take((size_t)mn * api_ld(fmt, k));
    S.bn_api = take((size_t)m * api_ld(fmt, k));
    S.bp = take((size_t)mn * lk * es);
    S.bn = take((size_t)m * lk * es);
    S.mc = take((size_t)mn * ld64(mn) * es);
    S.kc = take((size_t)m * ld64(mn) * es);
    S.y = take((size_t)mn * lk * es);
    S.y_api = take((size_t)mn * api_ld(fmt, k));
    S.err = take(256);
    S.total = off;
    return S;
}

bool shape_ok(const gfe_matrix *A) {
    if (!A || !field_ok(A->p) || A->m < 0 || A->n < 0) return false;
    if (A->fmt == GFE_BITS64) return A->p == 2;
    return A->fmt == GFE_U8;
}

}  // namespace
}  // namespace gfe

using namespace gfe;

extern "C" {

gfe_status gfe_nullspace(const gfe_matrix *A, const gfe_result *res, int32_t side, void *N, int64_t ldn,
                         void *stream) {
    if (!shape_ok(A)) return (set_error("gfe_nullspace: bad matrix description"), GFE_EINVAL);
    if (side != GFE_LEFT && side != GFE_RIGHT) return (set_error("gfe_nullspace: side must be GFE_LEFT or GFE_RIGHT"), GFE_EINVAL);
    if (!res || !res->rank) return (set_error("gfe_nullspace: the result's rank is required"), GFE_EINVAL);
    const bool left = side == GFE_LEFT, bits = A->fmt == GFE_BITS64;
    const int64_t len = left ? A->m : A->n;  // columns of N, and most rows it can have
    if (len == 0) return GFE_OK;
    const int64_t *piv = left ? res->pivot_rows : res->pivot_cols;
    const void *src = left ? res->K : res->R;
    const int64_t lds = left ? res->ldK : res->ldR;
    if (!piv || !src || !N) return (set_error("gfe_nullspace: pivots, K (left) or R (right), and N are required"), GFE_EINVAL);
    const int64_t words = words_of(len);
    if (ldn < (bits ? 8 * words : len) || (bits && (ldn % 8 || lds % 8)))
        return (set_error("gfe_nullspace: ldn too small or not a whole number of words"), GFE_EINVAL);
    cudaStream_t st = (cudaStream_t)stream;
    // rows past n - r (m - r) exit early on the device: the launch needs no rank
    const unsigned rows = gy(std::min<int64_t>(len, 4096));
    if (bits) {
        dim3 grid((unsigned)words, std::max(1u, rows / 64));
        if (left)
            k_null_left_bits<<<grid, 64, 0, st>>>(len, res->rank, piv, (const uint64_t *)src, lds / 8, (uint64_t *)N,
                                                  ldn / 8, words);
        else
            k_null_right_bits<<<grid, 64, 0, st>>>(len, res->rank, piv, (const uint64_t *)src, lds / 8, (uint64_t *)N,
                                                   ldn / 8, words);
    } else {
        dim3 grid(gx(len), rows);
        if (left)
            k_null_left_u8<<<grid, NT, 0, st>>>(len, res->rank, piv, (const uint8_t *)src, lds, (uint8_t *)N, ldn);
        else
            k_null_right_u8<<<grid, NT, 0, st>>>(len, res->rank, piv, (const uint8_t *)src, lds, (uint8_t *)N, ldn);
    }
    return cuda_ok(cudaGetLastError(), "null-space launch") ? GFE_OK : GFE_ECUDA;
}

size_t gfe_solve_workspace(const gfe_matrix *A, int64_t k) {
    if (!shape_ok(A) || k < 0) return 0;
    return solve_layout(A->p, A->fmt, A->m, A->n, k).total;
}

gfe_status gfe_solve(const gfe_matrix *A, const gfe_result *res, const void *B, int64_t ldb, int64_t k, void *X,
                     int64_t ldx, int32_t *consistent, void *ws, size_t ws_bytes, void *stream) {
    if (!shape_ok(A) || k < 0) return (set_error("gfe_solve: bad matrix description or k"), GFE_EINVAL);
    const int64_t m = A->m, n = A->n;
    const bool bits = A->fmt == GFE_BITS64;
    if (!res || !res->rank || (k > 0 && (!res->pivot_rows || !res->pivot_cols)))
        return (set_error("gfe_solve: the result's rank and pivots are required"), GFE_EINVAL);
    if (k == 0) return GFE_OK;
    const int64_t kb = bits ? 8 * words_of(k) : k;  // bytes of a row of B and X
    if ((m > 0 && (!B || ldb < kb)) || (n > 0 && (!X || ldx < kb)) || !consistent || (bits && (ldb % 8 || ldx % 8)))
        return (set_error("gfe_solve: B, X (ld >= a row) and consistent are required"), GFE_EINVAL);
    const SolveLayout S = solve_layout(A->p, A->fmt, m, n, k);
    if (!ws || ws_bytes < S.total) return (set_error("gfe_solve: workspace too small: need " + std::to_string(S.total)), GFE_EINVAL);
    Launch L;
    L.st = (cudaStream_t)stream;
    L.p = A->p;
    L.codec = codec_for(A->p);
    char *base = (char *)ws;
    L.err = (int *)(base + S.err);
    // the rank sizes the multiply-adds: the one host read of this call
    int64_t r = 0;
    if (!cuda_ok(cudaMemcpyAsync(&r, res->rank, 8, cudaMemcpyDeviceToHost, L.st), "rank read") ||
        !cuda_ok(host_wait(L.st), "rank read"))
        return GFE_ECUDA;
    if (r < 0 || r > std::min(m, n)) return (set_error("gfe_solve: the result's rank is out of range"), GFE_EINVAL);
    if (r > 0 && (!res->M || (m - r > 0 && !res->K))) return (set_error("gfe_solve: M and K are required"), GFE_EINVAL);
    if (!cuda_ok(cudaMemsetAsync(L.err, 0, sizeof(int), L.st), "error word")) return GFE_ECUDA;
    const int es = codec_bytes(L.codec);
    const int64_t lk = ld64(k), lmn = ld64(std::min(m, n)), la = api_ld(A->fmt, k);
    uint8_t *bp_api = (uint8_t *)(base + S.bp_api), *bn_api = (uint8_t *)(base + S.bn_api);
    char *bp = base + S.bp, *bn = base + S.bn, *mc = base + S.mc, *kc = base + S.kc, *y = base + S.y;
    uint8_t *y_api = (uint8_t *)(base + S.y_api);
    const int64_t nr = m - r;
    // b[rho] and b[rho_bar] in the API storage, then in the codec
    if (r > 0)
        k_gather_rows_bytes<<<dim3(gx(kb), gy(r)), NT, 0, L.st>>>(r, kb, (const uint8_t *)B, ldb, res->pivot_rows, r,
                                                                   true, bp_api, la);
    if (nr > 0)
        k_gather_rows_bytes<<<dim3(gx(kb), gy(nr)), NT, 0, L.st>>>(nr, kb, (const uint8_t *)B, ldb, res->pivot_rows, r,
                                                                    false, bn_api, la);
    auto import = [&](int64_t rows, int64_t cols, void *dst, int64_t ldd, const void *src, int64_t lds) {
        if (rows <= 0 || cols <= 0) return;
        if (bits) import_bits(L, rows, cols, dst, ldd, (const uint64_t *)src, lds / 8);
        else import_u8(L, rows, cols, dst, ldd, (const uint8_t *)src, lds);
    };
    auto export_ = [&](int64_t rows, int64_t cols, void *dst, int64_t ldd, const void *src, int64_t lds) {
        if (rows <= 0 || cols <= 0) return;
        if (bits) export_bits(L, rows, cols, (uint64_t *)dst, ldd / 8, src, lds);
        else export_u8(L, rows, cols, (uint8_t *)dst, ldd, src, lds);
    };
    import(r, k, bp, lk, bp_api, la);
    import(nr, k, bn, lk, bn_api, la);
    import(r, r, mc, lmn, res->M, res->ldM);
    import(nr, r, kc, lmn, res->K, res->ldK);
    // (T b)[..r] = M b[rho];  (T b)[r..] = K b[rho] + b[rho_bar]
    if (r > 0) mad(L, r, k, r, nullptr, 0, mc, lmn, bp, lk, y, lk);
    if (nr > 0) mad(L, nr, k, r, bn, lk, kc, lmn, bp, lk, bn, lk);
    export_(r, k, y_api, la, y, lk);
    export_(nr, k, bn_api, la, bn, lk);  // (T b)[r..] back in the API storage, over b[rho_bar]
    k_fill_i32<<<(unsigned)((k + NT - 1) / NT), NT, 0, L.st>>>(consistent, k, 1);
    if (nr > 0) {
        if (bits)
            k_consistent_bits<<<dim3(gx(words_of(k)), gy(nr)), NT, 0, L.st>>>(nr, k, words_of(k),
                                                                              (const uint64_t *)bn_api, la / 8,
                                                                              consistent);
        else
            k_consistent_u8<<<dim3(gx(k), gy(nr)), NT, 0, L.st>>>(nr, k, bn_api, la, consistent);
    }
    if (n > 0) {
        if (bits)
            k_solve_x_bits<<<dim3(gx(words_of(k)), gy(n)), NT, 0, L.st>>>(n, words_of(k), res->pivot_cols, r,
                                                                          (const uint64_t *)y_api, la / 8,
                                                                          (uint64_t *)X, ldx / 8);
        else
            k_solve_x_u8<<<dim3(gx(k), gy(n)), NT, 0, L.st>>>(n, k, A->p, res->pivot_cols, r, y_api, la,
                                                              (uint8_t *)X, ldx);
    }
    if (!cuda_ok(cudaGetLastError(), "solve launch")) return GFE_ECUDA;
    int gave_up = 0;
    if (!read_error_word(L.st, L.err, &gave_up)) return (set_error("error word read failed"), GFE_ECUDA);
    if (gave_up) return (set_error("tensor-core multiply-add timed out"), GFE_ETIMEOUT);
    return GFE_OK;
}

}  // extern "C"
