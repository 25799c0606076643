/*
 * gfe_oracle.c -- plain, slow, obviously-correct CPU oracle for echelonisation
 * with transformation matrix over GF(p), p prime, p <= 251.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (Linton, Nebe, Niemeyer, Parker, Thackray, arXiv 1806.04211):
 *   Eq. (gauss) / Eq. (echelon), Section 3.1: for C in F^{m x n} of rank r,
 *     (M 0; K 1) (rho; rho_bar) C (Ups^tr Ups_bar^tr) = (-1 R; 0 0)
 *   with the pivot of a row being its first non-zero entry (Section 1) and
 *   the "negative" echelon form (Remark "echelon", Section 2.2).
 *   Readings fixed here (the paper leaves them implicit):
 *     - rho (varrho) is the row rank profile: row x is a pivot row iff it is
 *       not in the span of rows 0..x-1;
 *     - Ups is the column rank profile (pivot columns of the RREF);
 *     - rows of M and of E_top are ordered by ascending pivot column,
 *       columns of M and K by ascending pivot row, rows of K ascending;
 *     - indices are 0-based.
 *   These make M = -C[rho,Ups]^{-1}, K = C[rho_bar,Ups] M, R = M C[rho,Ups_bar]
 *   unique.
 *
 * Algorithm: row-greedy Gauss-Jordan with transformation (textbook).  Rows are
 * taken top to bottom; each is reduced against the already-found pivot rows,
 * which are kept fully reduced with -1 (= p-1) in their pivot column.  A row
 * that reduces to zero is a non-pivot row and its transformation row is a row
 * of K; otherwise its first non-zero entry becomes a pivot, it is scaled so
 * that entry is -1, and every earlier pivot row is cleared in that column.
 * Cost m*r*(n+m) multiply-adds.  Every entry is kept in [0,p) after every
 * step except in the one clearly marked lazily-reduced accumulation.
 *
 * GF(2) has its own bit-packed version (XOR instead of multiply-add): bit
 * (c % 64) of 64-bit word c/64 of a row is column c.
 *
 * Certificates (used where the oracle itself is too slow): exact structure
 * checks plus Freivalds' randomized check of T*C = E (Freivalds 1977).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* field helpers                                                             */
/* ------------------------------------------------------------------------ */

/* inverse by brute force: the x with a*x = 1 mod p (p prime, a != 0) */
static int orc_inv(int p, int a)
{
    for (int x = 1; x < p; ++x)
        if ((a * x) % p == 1) return x;
    return 0;
}

int orc_is_prime(int p)
{
    if (p < 2) return 0;
    for (int d = 2; d * d <= p; ++d)
        if (p % d == 0) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* uint8 GF(p)                                                               */
/* ------------------------------------------------------------------------ */

/*
 * orc_echelon_u8: row-greedy Gauss-Jordan with transformation over GF(p).
 *   A      : m x n, row-major, leading dimension lda (bytes), entries in [0,p)
 *   rank   : out, r
 *   prow   : out, r entries, pivot rows (rho) ascending          (may be NULL)
 *   pcol   : out, r entries, pivot columns (Ups) ascending       (may be NULL)
 *   M      : out, r x r, row-major, ld = ldm                      (may be NULL)
 *   K      : out, (m-r) x r, row-major, ld = ldk                  (may be NULL)
 *   R      : out, r x (n-r), row-major, ld = ldr                  (may be NULL)
 *   E      : out, m x n dense echelon form, ld = lde              (may be NULL)
 *   T      : out, m x m dense transformation (T*A = E), ld = ldt  (may be NULL)
 *   Buffers must be sized for the worst case r = min(m,n).
 * Returns 0, or -1 on bad arguments / out of memory.
 */
int orc_echelon_u8(int p, int64_t m, int64_t n, const uint8_t *A, int64_t lda,
                   int64_t *rank, int64_t *prow, int64_t *pcol,
                   uint8_t *M, int64_t ldm, uint8_t *K, int64_t ldk,
                   uint8_t *R, int64_t ldr, uint8_t *E, int64_t lde,
                   uint8_t *T, int64_t ldt)
{
    if (!orc_is_prime(p) || p > 251 || m < 0 || n < 0) return -1;
    int64_t rmax = m < n ? m : n;
    /* pivot store: for pivot q, its reduced row e_q (n) and transformation t_q (m) */
    int64_t w = n + m;                            /* e and t side by side */
    uint8_t *piv = (uint8_t *)calloc((size_t)(rmax > 0 ? rmax : 1) * (size_t)(w > 0 ? w : 1), 1);
    int64_t *pr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rmax + 1));
    int64_t *pc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rmax + 1));
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(w > 0 ? w : 1));
    /* transformation rows of the non-pivot rows (only kept if K or T wanted) */
    size_t kbytes = (K || T) ? (size_t)(m > 0 ? m : 1) * (size_t)(m > 0 ? m : 1) : 1;
    uint8_t *krows = (uint8_t *)calloc(kbytes, 1);
    int64_t *nonpiv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!piv || !pr || !pc || !acc || !krows || !nonpiv) {
        free(piv); free(pr); free(pc); free(acc); free(krows); free(nonpiv);
        return -1;
    }
    /* largest number of products (<= (p-1)^2 each) a uint32 can absorb */
    uint32_t maxacc = (uint32_t)((0xFFFFFFFFu - (uint32_t)(p - 1)) / (uint32_t)((p - 1) * (p - 1) > 0 ? (p - 1) * (p - 1) : 1));
    int64_t r = 0, nk = 0;

    for (int64_t x = 0; x < m; ++x) {
        /* v = A[x,:], t = unit vector at x */
        for (int64_t c = 0; c < n; ++c) acc[c] = A[x * lda + c];
        for (int64_t c = 0; c < m; ++c) acc[n + c] = 0;
        acc[n + x] = 1;
        /* Reduce against every pivot.  The pivot rows are fully reduced, so
         * adding s*e_q changes v in no other pivot column: every coefficient
         * s_q = v[c_q] is read from the (reduced-so-far) row directly.
         * Lazily reduced: acc holds sums of at most maxacc products. */
        uint32_t pending = 0;
        for (int64_t q = 0; q < r; ++q) {
            uint32_t s = acc[pc[q]] % (uint32_t)p;
            if (s == 0) continue;
            const uint8_t *eq = piv + q * w;
            for (int64_t c = 0; c < w; ++c) acc[c] += s * eq[c];
            if (++pending == maxacc) {
                for (int64_t c = 0; c < w; ++c) acc[c] %= (uint32_t)p;
                pending = 0;
            }
        }
        for (int64_t c = 0; c < w; ++c) acc[c] %= (uint32_t)p;
        int64_t lead = -1;
        for (int64_t c = 0; c < n; ++c)
            if (acc[c]) { lead = c; break; }
        if (lead < 0) {
            /* non-pivot row: its transformation row (restricted later to rho) */
            if (K || T) {
                uint8_t *kr = krows + nk * m;
                for (int64_t c = 0; c < m; ++c) kr[c] = (uint8_t)acc[n + c];
            }
            nonpiv[nk++] = x;
            continue;
        }
        /* new pivot: scale so that v[lead] = -1 */
        int s = (p - orc_inv(p, (int)acc[lead])) % p;
        uint8_t *e = piv + r * w;
        for (int64_t c = 0; c < w; ++c) e[c] = (uint8_t)((acc[c] * (uint32_t)s) % (uint32_t)p);
        /* clear the new pivot column in every earlier pivot row:
         * e_q += u * e with u = e_q[lead] (since e[lead] = -1) */
        for (int64_t q = 0; q < r; ++q) {
            uint8_t *eq = piv + q * w;
            uint32_t u = eq[lead];
            if (u == 0) continue;
            for (int64_t c = 0; c < w; ++c) eq[c] = (uint8_t)((eq[c] + u * e[c]) % (uint32_t)p);
        }
        pr[r] = x;
        pc[r] = lead;
        ++r;
    }

    /* order of pivots by column (rows of M / E_top) -- pivots were found in
     * row order; sort indices by pc (insertion sort, r small enough) */
    int64_t *byc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(r + 1));
    for (int64_t q = 0; q < r; ++q) byc[q] = q;
    for (int64_t a = 1; a < r; ++a) {
        int64_t v = byc[a], b = a - 1;
        while (b >= 0 && pc[byc[b]] > pc[v]) { byc[b + 1] = byc[b]; --b; }
        byc[b + 1] = v;
    }
    /* pr is ascending already (rows taken in order) */
    int64_t *colpos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t c = 0; c < n; ++c) colpos[c] = -1;
    for (int64_t l = 0; l < r; ++l) colpos[pc[byc[l]]] = l;

    *rank = r;
    if (prow) for (int64_t q = 0; q < r; ++q) prow[q] = pr[q];
    if (pcol) for (int64_t l = 0; l < r; ++l) pcol[l] = pc[byc[l]];
    if (M) {
        for (int64_t l = 0; l < r; ++l) {
            const uint8_t *t = piv + byc[l] * w + n;
            for (int64_t s2 = 0; s2 < r; ++s2) M[l * ldm + s2] = t[pr[s2]];
        }
    }
    if (K) {
        for (int64_t a = 0; a < nk; ++a) {
            const uint8_t *t = krows + a * m;
            for (int64_t s2 = 0; s2 < r; ++s2) K[a * ldk + s2] = t[pr[s2]];
        }
    }
    if (R) {
        for (int64_t l = 0; l < r; ++l) {
            const uint8_t *e = piv + byc[l] * w;
            int64_t j = 0;
            for (int64_t c = 0; c < n; ++c)
                if (colpos[c] < 0) R[l * ldr + (j++)] = e[c];
        }
    }
    if (E) {
        for (int64_t l = 0; l < m; ++l) memset(E + l * lde, 0, (size_t)n);
        for (int64_t l = 0; l < r; ++l) memcpy(E + l * lde, piv + byc[l] * w, (size_t)n);
    }
    if (T) {
        /* T = (M 0; K 1) P_rho: row l < r is t of pivot l; row r+a is the
         * transformation row of non-pivot row a (1 at its own position). */
        for (int64_t l = 0; l < m; ++l) memset(T + l * ldt, 0, (size_t)m);
        for (int64_t l = 0; l < r; ++l) memcpy(T + l * ldt, piv + byc[l] * w + n, (size_t)m);
        for (int64_t a = 0; a < nk; ++a) memcpy(T + (r + a) * ldt, krows + a * m, (size_t)m);
    }
    free(byc); free(colpos);
    free(piv); free(pr); free(pc); free(acc); free(krows); free(nonpiv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* bit-packed GF(2)                                                          */
/* ------------------------------------------------------------------------ */

static inline int bit_get(const uint64_t *row, int64_t c) { return (int)((row[c >> 6] >> (c & 63)) & 1u); }
static inline void bit_set(uint64_t *row, int64_t c) { row[c >> 6] |= (uint64_t)1 << (c & 63); }

/*
 * orc_echelon_gf2: the same algorithm over GF(2), rows bit-packed.
 *   A : m rows of ldw 64-bit words (ldw >= ceil(n/64)); bits >= n ignored.
 *   Outputs are bit-packed rows with the given word strides; each output row
 *   has its bits beyond the row length cleared.  Over GF(2), -1 = 1.
 */
int orc_echelon_gf2(int64_t m, int64_t n, const uint64_t *A, int64_t ldw,
                    int64_t *rank, int64_t *prow, int64_t *pcol,
                    uint64_t *M, int64_t ldm, uint64_t *K, int64_t ldk,
                    uint64_t *R, int64_t ldr, uint64_t *E, int64_t lde,
                    uint64_t *T, int64_t ldt)
{
    if (m < 0 || n < 0) return -1;
    int64_t rmax = m < n ? m : n;
    int64_t wn = (n + 63) / 64, wm = (m + 63) / 64, w = wn + wm;
    uint64_t *piv = (uint64_t *)calloc((size_t)(rmax > 0 ? rmax : 1) * (size_t)(w > 0 ? w : 1), 8);
    int64_t *pr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rmax + 1));
    int64_t *pc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rmax + 1));
    uint64_t *v = (uint64_t *)malloc(8 * (size_t)(w > 0 ? w : 1));
    size_t kbytes = (K || T) ? (size_t)(m > 0 ? m : 1) * (size_t)(wm > 0 ? wm : 1) : 1;
    uint64_t *krows = (uint64_t *)calloc(kbytes, 8);
    if (!piv || !pr || !pc || !v || !krows) {
        free(piv); free(pr); free(pc); free(v); free(krows);
        return -1;
    }
    uint64_t lastmask = (n & 63) ? (((uint64_t)1 << (n & 63)) - 1) : ~(uint64_t)0;
    int64_t r = 0, nk = 0;
    for (int64_t x = 0; x < m; ++x) {
        memset(v, 0, 8 * (size_t)w);
        for (int64_t a = 0; a < wn; ++a) v[a] = A[x * ldw + a];
        if (wn) v[wn - 1] &= lastmask;
        bit_set(v + wn, x);
        /* reduce against every (fully reduced) pivot whose column is set */
        for (int64_t q = 0; q < r; ++q) {
            if (!bit_get(v, pc[q])) continue;
            const uint64_t *eq = piv + q * w;
            for (int64_t a = 0; a < w; ++a) v[a] ^= eq[a];
        }
        int64_t lead = -1;
        for (int64_t a = 0; a < wn; ++a)
            if (v[a]) { lead = a * 64 + __builtin_ctzll(v[a]); break; }
        if (lead < 0) {
            if (K || T) memcpy(krows + nk * wm, v + wn, 8 * (size_t)wm);
            ++nk;
            continue;
        }
        uint64_t *e = piv + r * w;
        memcpy(e, v, 8 * (size_t)w);
        for (int64_t q = 0; q < r; ++q) {
            uint64_t *eq = piv + q * w;
            if (!bit_get(eq, lead)) continue;
            for (int64_t a = 0; a < w; ++a) eq[a] ^= e[a];
        }
        pr[r] = x;
        pc[r] = lead;
        ++r;
    }
    int64_t *byc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(r + 1));
    for (int64_t q = 0; q < r; ++q) byc[q] = q;
    for (int64_t a = 1; a < r; ++a) {
        int64_t t = byc[a], b = a - 1;
        while (b >= 0 && pc[byc[b]] > pc[t]) { byc[b + 1] = byc[b]; --b; }
        byc[b + 1] = t;
    }
    char *ispc = (char *)calloc((size_t)(n + 1), 1);
    for (int64_t q = 0; q < r; ++q) ispc[pc[q]] = 1;

    *rank = r;
    if (prow) for (int64_t q = 0; q < r; ++q) prow[q] = pr[q];
    if (pcol) for (int64_t l = 0; l < r; ++l) pcol[l] = pc[byc[l]];
    if (M) {
        int64_t wr = (r + 63) / 64;
        for (int64_t l = 0; l < r; ++l) {
            const uint64_t *t = piv + byc[l] * w + wn;
            uint64_t *o = M + l * ldm;
            memset(o, 0, 8 * (size_t)wr);
            for (int64_t s = 0; s < r; ++s) if (bit_get(t, pr[s])) bit_set(o, s);
        }
    }
    if (K) {
        int64_t wr = (r + 63) / 64;
        for (int64_t a = 0; a < nk; ++a) {
            const uint64_t *t = krows + a * wm;
            uint64_t *o = K + a * ldk;
            memset(o, 0, 8 * (size_t)wr);
            for (int64_t s = 0; s < r; ++s) if (bit_get(t, pr[s])) bit_set(o, s);
        }
    }
    if (R) {
        int64_t wr = (n - r + 63) / 64;
        for (int64_t l = 0; l < r; ++l) {
            const uint64_t *e = piv + byc[l] * w;
            uint64_t *o = R + l * ldr;
            memset(o, 0, 8 * (size_t)wr);
            int64_t j = 0;
            for (int64_t c = 0; c < n; ++c) {
                if (ispc[c]) continue;
                if (bit_get(e, c)) bit_set(o, j);
                ++j;
            }
        }
    }
    if (E) {
        for (int64_t l = 0; l < m; ++l) memset(E + l * lde, 0, 8 * (size_t)wn);
        for (int64_t l = 0; l < r; ++l) memcpy(E + l * lde, piv + byc[l] * w, 8 * (size_t)wn);
    }
    if (T) {
        for (int64_t l = 0; l < m; ++l) memset(T + l * ldt, 0, 8 * (size_t)wm);
        for (int64_t l = 0; l < r; ++l) memcpy(T + l * ldt, piv + byc[l] * w + wn, 8 * (size_t)wm);
        for (int64_t a = 0; a < nk; ++a) memcpy(T + (r + a) * ldt, krows + a * wm, 8 * (size_t)wm);
    }
    free(byc); free(ispc);
    free(piv); free(pr); free(pc); free(v); free(krows);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* certificates                                                              */
/* ------------------------------------------------------------------------ */

/* SplitMix64 output function (Steele, Lea, Flood 2014), used only to draw the
 * Freivalds test vectors. */
static uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/*
 * orc_certify_u8: checks a claimed result (r, rho, Ups, M, K, R) for A over GF(p)
 * without recomputing it:
 *   1  rho, Ups strictly ascending, in range;
 *   2  E_top = (-1 | R) in permuted columns is in reduced echelon form:
 *      R[l, j] = 0 for every non-pivot column j left of Ups[l];
 *   3  K[t,s] = 0 whenever rho[s] > rho_bar[t]  (rows are combinations of
 *      earlier rows only);
 *   4  Freivalds, nvec random vectors x:  M (A[rho,:] x) == E_top x  and
 *      K (A[rho,:] x) + A[rho_bar,:] x == 0.
 * Together these force the result to equal the unique output defined above
 * (with false-accept probability <= p^-nvec for check 4).
 * Returns 0 if all pass, else the number of the first failing check.
 */
int orc_certify_u8(int p, int64_t m, int64_t n, const uint8_t *A, int64_t lda,
                   int64_t r, const int64_t *prow, const int64_t *pcol,
                   const uint8_t *M, int64_t ldm, const uint8_t *K, int64_t ldk,
                   const uint8_t *R, int64_t ldr, int nvec, uint64_t seed)
{
    if (r < 0 || r > m || r > n) return 1;
    for (int64_t q = 0; q < r; ++q) {
        if (prow[q] < 0 || prow[q] >= m || pcol[q] < 0 || pcol[q] >= n) return 1;
        if (q && (prow[q] <= prow[q - 1] || pcol[q] <= pcol[q - 1])) return 1;
    }
    char *isr = (char *)calloc((size_t)m + 1, 1), *isc = (char *)calloc((size_t)n + 1, 1);
    int64_t *nonr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *nonc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t q = 0; q < r; ++q) { isr[prow[q]] = 1; isc[pcol[q]] = 1; }
    int64_t nr = 0, nc = 0;
    for (int64_t x = 0; x < m; ++x) if (!isr[x]) nonr[nr++] = x;
    for (int64_t c = 0; c < n; ++c) if (!isc[c]) nonc[nc++] = c;
    int rc = 0;
    /* 2 */
    for (int64_t l = 0; l < r && !rc; ++l)
        for (int64_t j = 0; j < nc && nonc[j] < pcol[l]; ++j)
            if (R[l * ldr + j]) { rc = 2; break; }
    /* 3 */
    for (int64_t t = 0; t < nr && !rc; ++t)
        for (int64_t s = 0; s < r; ++s)
            if (prow[s] > nonr[t] && K[t * ldk + s]) { rc = 3; break; }
    /* 4 */
    uint32_t *x = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    uint32_t *ax = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m + 1));
    for (int v = 0; v < nvec && !rc; ++v) {
        for (int64_t c = 0; c < n; ++c)
            x[c] = (uint32_t)(((orc_mix64(seed * 0x9E3779B97F4A7C15ull + (uint64_t)(v * n + c) + 1) >> 32) * (uint64_t)p) >> 32);
        for (int64_t i = 0; i < m; ++i) {
            uint64_t s = 0;
            for (int64_t c = 0; c < n; ++c) s += (uint64_t)A[i * lda + c] * x[c];
            ax[i] = (uint32_t)(s % (uint64_t)p);
        }
        for (int64_t l = 0; l < r && !rc; ++l) {
            uint64_t lhs = 0, rhs = 0;
            for (int64_t s = 0; s < r; ++s) lhs += (uint64_t)M[l * ldm + s] * ax[prow[s]];
            rhs = (uint64_t)(p - 1) * x[pcol[l]];
            for (int64_t j = 0; j < nc; ++j) rhs += (uint64_t)R[l * ldr + j] * x[nonc[j]];
            if (lhs % (uint64_t)p != rhs % (uint64_t)p) rc = 4;
        }
        for (int64_t t = 0; t < nr && !rc; ++t) {
            uint64_t s2 = ax[nonr[t]];
            for (int64_t s = 0; s < r; ++s) s2 += (uint64_t)K[t * ldk + s] * ax[prow[s]];
            if (s2 % (uint64_t)p) rc = 4;
        }
    }
    free(x); free(ax); free(isr); free(isc); free(nonr); free(nonc);
    return rc;
}

/* GF(2) bit-packed certificate: the same four checks; check 4 runs 64 random
 * vectors at once, one per bit of a 64-bit word. */
int orc_certify_gf2(int64_t m, int64_t n, const uint64_t *A, int64_t ldw,
                    int64_t r, const int64_t *prow, const int64_t *pcol,
                    const uint64_t *M, int64_t ldm, const uint64_t *K, int64_t ldk,
                    const uint64_t *R, int64_t ldr, uint64_t seed)
{
    if (r < 0 || r > m || r > n) return 1;
    for (int64_t q = 0; q < r; ++q) {
        if (prow[q] < 0 || prow[q] >= m || pcol[q] < 0 || pcol[q] >= n) return 1;
        if (q && (prow[q] <= prow[q - 1] || pcol[q] <= pcol[q - 1])) return 1;
    }
    char *isr = (char *)calloc((size_t)m + 1, 1), *isc = (char *)calloc((size_t)n + 1, 1);
    int64_t *nonr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *nonc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t q = 0; q < r; ++q) { isr[prow[q]] = 1; isc[pcol[q]] = 1; }
    int64_t nr = 0, nc = 0;
    for (int64_t x = 0; x < m; ++x) if (!isr[x]) nonr[nr++] = x;
    for (int64_t c = 0; c < n; ++c) if (!isc[c]) nonc[nc++] = c;
    int rc = 0;
    for (int64_t l = 0; l < r && !rc; ++l)
        for (int64_t j = 0; j < nc && nonc[j] < pcol[l]; ++j)
            if (bit_get(R + l * ldr, j)) { rc = 2; break; }
    for (int64_t t = 0; t < nr && !rc; ++t)
        for (int64_t s = 0; s < r; ++s)
            if (prow[s] > nonr[t] && bit_get(K + t * ldk, s)) { rc = 3; break; }
    /* x[c]: 64 random bits = column c of the 64 test vectors */
    uint64_t *x = (uint64_t *)malloc(8 * (size_t)(n + 1));
    uint64_t *ax = (uint64_t *)malloc(8 * (size_t)(m + 1));
    for (int64_t c = 0; c < n; ++c) x[c] = orc_mix64(seed * 0x9E3779B97F4A7C15ull + (uint64_t)c + 1);
    if (!rc) {
        for (int64_t i = 0; i < m; ++i) {
            uint64_t s = 0;
            for (int64_t c = 0; c < n; ++c) if (bit_get(A + i * ldw, c)) s ^= x[c];
            ax[i] = s;
        }
        for (int64_t l = 0; l < r && !rc; ++l) {
            uint64_t lhs = 0, rhs = x[pcol[l]];
            for (int64_t s = 0; s < r; ++s) if (bit_get(M + l * ldm, s)) lhs ^= ax[prow[s]];
            for (int64_t j = 0; j < nc; ++j) if (bit_get(R + l * ldr, j)) rhs ^= x[nonc[j]];
            if (lhs != rhs) rc = 4;
        }
        for (int64_t t = 0; t < nr && !rc; ++t) {
            uint64_t s2 = ax[nonr[t]];
            for (int64_t s = 0; s < r; ++s) if (bit_get(K + t * ldk, s)) s2 ^= ax[prow[s]];
            if (s2) rc = 4;
        }
    }
    free(x); free(ax); free(isr); free(isc); free(nonr); free(nonc);
    return rc;
}
