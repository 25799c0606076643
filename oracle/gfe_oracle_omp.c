/*
 * gfe_oracle_omp.c -- Gauss-Jordan elimination with transformation over
 * GF(2), bit-packed, on all host cores with OpenMP.  TIMING BASELINE ONLY:
 * the benchmark reports it beside the single-threaded oracle (gfe_oracle.c);
 * the tests check that it returns the oracle's result; the product library
 * never loads it.  It shares no code with the CUDA path.
 *
 * It computes the same unique result as the oracle (arXiv 1806.04211,
 * Eq. (echelon), Section 3.1, with rho the row rank profile and the pivot
 * of a row its first non-zero entry, Section 1) by the textbook elimination
 * taken pivot by pivot, each pivot's elimination parallel over rows.  Every
 * row carries its transformation row [A_x | e_x].  For each column c, left
 * to right:
 *   1. the pivot row is the topmost row that is not yet a pivot row and has
 *      bit c set (none: c is not a pivot column).  That rule selects the row
 *      rank profile: a row becomes a pivot row exactly when it is not in the
 *      span of the rows above it.
 *   2. every other row with bit c set adds the pivot row (XOR) -- in
 *      parallel over rows.  Rows that are not pivot rows are zero left of c,
 *      and so is the pivot row, so only words from c/64 on change in the A
 *      half.
 * At the end the pivot rows, by ascending column, are E_top (over GF(2),
 * -1 = 1) and their transformation halves restricted to rho are M; the
 * other rows' transformation halves restricted to rho are K.
 * Outputs as orc_echelon_gf2 (rank, rho, Ups, M, K, R; bit-packed rows).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

static inline int obit(const uint64_t *row, int64_t c) { return (int)((row[c >> 6] >> (c & 63)) & 1u); }
static inline void oset(uint64_t *row, int64_t c) { row[c >> 6] |= (uint64_t)1 << (c & 63); }

int orc_omp_threads(void) { return omp_get_max_threads(); }

int orc_echelon_gf2_omp(int64_t m, int64_t n, const uint64_t *A, int64_t ldw,
                        int64_t *rank, int64_t *prow, int64_t *pcol,
                        uint64_t *M, int64_t ldm, uint64_t *K, int64_t ldk,
                        uint64_t *R, int64_t ldr)
{
    if (m < 0 || n < 0) return -1;
    const int64_t rmax = m < n ? m : n;
    const int64_t wn = (n + 63) / 64, wm = (m + 63) / 64, w = wn + wm;
    uint64_t *rows = (uint64_t *)calloc((size_t)(m > 0 ? m : 1) * (size_t)(w > 0 ? w : 1), 8);
    int64_t *pr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rmax + 1));  /* by column */
    int64_t *pc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rmax + 1));
    int64_t *rho = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rmax + 1)); /* ascending */
    char *isp = (char *)calloc((size_t)(m + 1), 1);
    char *ispc = (char *)calloc((size_t)(n + 1), 1);
    if (!rows || !pr || !pc || !rho || !isp || !ispc) {
        free(rows); free(pr); free(pc); free(rho); free(isp); free(ispc);
        return -1;
    }
    const uint64_t lastmask = (n & 63) ? (((uint64_t)1 << (n & 63)) - 1) : ~(uint64_t)0;
    for (int64_t x = 0; x < m; ++x) {
        uint64_t *row = rows + x * w;
        for (int64_t a = 0; a < wn; ++a) row[a] = A[x * ldw + a];
        if (wn) row[wn - 1] &= lastmask;
        oset(row + wn, x);
    }
    int64_t r = 0;
    for (int64_t c = 0; c < n && r < m; ++c) {
        int64_t x = -1;
        for (int64_t y = 0; y < m; ++y)
            if (!isp[y] && obit(rows + y * w, c)) { x = y; break; }
        if (x < 0) continue;
        isp[x] = 1;
        ispc[c] = 1;
        pr[r] = x;
        pc[r] = c;
        ++r;
        const uint64_t *e = rows + x * w;
        const int64_t a0 = c >> 6;
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < m; ++y) {
            if (y == x) continue;
            uint64_t *row = rows + y * w;
            if (!obit(row, c)) continue;
            for (int64_t a = a0; a < w; ++a) row[a] ^= e[a];
        }
    }
    int64_t q = 0;
    for (int64_t x = 0; x < m; ++x) if (isp[x]) rho[q++] = x;
    *rank = r;
    if (prow) for (int64_t s = 0; s < r; ++s) prow[s] = rho[s];
    if (pcol) for (int64_t l = 0; l < r; ++l) pcol[l] = pc[l];
    const int64_t wr = (r + 63) / 64;
    if (M)
        for (int64_t l = 0; l < r; ++l) {
            const uint64_t *t = rows + pr[l] * w + wn;
            uint64_t *o = M + l * ldm;
            memset(o, 0, 8 * (size_t)wr);
            for (int64_t s = 0; s < r; ++s) if (obit(t, rho[s])) oset(o, s);
        }
    if (K) {
        int64_t a = 0;
        for (int64_t x = 0; x < m; ++x) {
            if (isp[x]) continue;
            const uint64_t *t = rows + x * w + wn;
            uint64_t *o = K + a * ldk;
            memset(o, 0, 8 * (size_t)wr);
            for (int64_t s = 0; s < r; ++s) if (obit(t, rho[s])) oset(o, s);
            ++a;
        }
    }
    if (R) {
        const int64_t wq = (n - r + 63) / 64;
        for (int64_t l = 0; l < r; ++l) {
            const uint64_t *e = rows + pr[l] * w;
            uint64_t *o = R + l * ldr;
            memset(o, 0, 8 * (size_t)wq);
            int64_t j = 0;
            for (int64_t c = 0; c < n; ++c) {
                if (ispc[c]) continue;
                if (obit(e, c)) oset(o, j);
                ++j;
            }
        }
    }
    free(rows); free(pr); free(pc); free(rho); free(isp); free(ispc);
    return 0;
}
