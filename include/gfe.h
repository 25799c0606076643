/*
 * gfe.h -- C ABI of libgfe: exact Gaussian elimination with transformation
 * matrix over small prime fields GF(p), p <= 251, on one GB300 (sm_103a).
 *
 * Method: Linton, Nebe, Niemeyer, Parker, Thackray, "A parallel algorithm for
 * Gaussian elimination over finite fields", arXiv 1806.04211.  For an input
 * C in GF(p)^{m x n} of rank r the library computes, Eq. (echelon) (Section 3.1):
 *
 *     (M 0; K 1) (rho; rho_bar) C (Ups^tr Ups_bar^tr) = (-1 R; 0 0)
 *
 * with rho (varrho) the pivot rows, Ups (Upsilon) the pivot columns and the
 * paper's negative normalisation: every pivot entry of the echelon form is
 * -1 (= p-1).  The pivot of a row is its first non-zero entry (Section 1);
 * rho is then the row rank profile and Ups the column rank profile, which
 * makes every output unique.  Ordering: rows of M and R by ascending pivot
 * column, columns of M and K by ascending pivot row, rows of K ascending
 * (rho_bar).  All indices are 0-based (the paper's are 1-based).
 *
 * Storage (argument "fmt"):
 *   GFE_U8     one byte per entry, value in [0,p), row-major, ld in bytes.
 *   GFE_BITS64 GF(2) only: rows of 64-bit words, bit (c % 64) of word c/64 is
 *              column c (LSB first); ld in bytes (multiple of 8); pad bits
 *              of the input are ignored, pad bits of outputs are written 0.
 *
 * Memory: every pointer in this header is DEVICE memory unless stated
 * otherwise.  Inputs are never modified.  Outputs and the workspace are
 * owned by the caller; the library keeps no pointer after a call returns
 * except for the requests of a gfe_server (see there).  Calls are asynchronous on the
 * given CUDA stream (a cudaStream_t passed as void*; NULL = legacy default
 * stream) EXCEPT that gfe_echelon / gfe_rank synchronise that stream
 * internally once per block echelonisation (the host plans the data-dependent
 * shapes); they return when all work has been queued and the result is
 * complete on the device.
 *
 * Errors: every function returns a gfe_status.  GFE_EINVAL: bad argument
 * (p not prime or > 251, fmt/p mismatch, negative sizes, NULL where a buffer
 * is required, ld too small, workspace too small).  GFE_ECUDA: a CUDA call
 * failed (gfe_last_error() gives its text).  No call aborts the process.
 */
#ifndef GFE_H
#define GFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GFE_OK = 0,
    GFE_EINVAL = 1,
    GFE_ENOMEM = 2,
    GFE_ETIMEOUT = 3,
    GFE_EBUSY = 4,
    GFE_ECUDA = 5,
    GFE_EINTERNAL = 6,
    GFE_ENOTSUP = 7
} gfe_status;

typedef enum { GFE_U8 = 0, GFE_BITS64 = 1 } gfe_storage;

/* flags */
#define GFE_WANT_TRANSFORM 0x1u  /* compute M and K (Task UpdateRowTrafo, Steps 2-3 on M) */
#define GFE_WANT_DENSE_E   0x2u  /* also write dense E = (-RREF(C); 0), m x n        */
#define GFE_WANT_DENSE_T   0x4u  /* also write dense T = (M 0; K 1) P_rho, m x m     */
#define GFE_IMPL_PLAIN     0x100u /* block multiply-add on CUDA cores (the plain     */
                                  /* comparator) instead of the tensor cores        */
#define GFE_IMPL_TENSOR    0x200u /* force the tcgen05 tensor-core multiply-add     */

/* A matrix argument: m x n over GF(p), stored as described above. */
typedef struct {
    int32_t p;
    int64_t m, n;
    int32_t fmt;          /* gfe_storage */
    const void *data;     /* device */
    int64_t ld;           /* bytes between consecutive rows */
} gfe_matrix;

/*
 * Result buffers (device, caller-allocated, sized for the worst case
 * r = min(m,n); the first r / m-r rows and r / n-r columns are written).
 * Same storage format as the input.  Any pointer may be NULL to skip that
 * output, except rank.
 */
typedef struct {
    int64_t *rank;        /* 1 int64: r */
    int64_t *pivot_cols;  /* Ups: r int64, ascending            (min(m,n) entries) */
    int64_t *pivot_rows;  /* rho: r int64, ascending            (min(m,n) entries) */
    void *R; int64_t ldR; /* r x (n-r)    (min(m,n) rows, n cols)                   */
    void *M; int64_t ldM; /* r x r        (min(m,n) rows, min(m,n) cols)            */
    void *K; int64_t ldK; /* (m-r) x r    (m rows, min(m,n) cols)                   */
    void *E; int64_t ldE; /* m x n dense echelon form   (GFE_WANT_DENSE_E)          */
    void *T; int64_t ldT; /* m x m dense transformation (GFE_WANT_DENSE_T)          */
} gfe_result;

/* Workspace (bytes, device) that gfe_echelon / gfe_rank need for A and flags.
 * Depends only on (p, m, n, flags). */
gfe_status gfe_query_workspace(const gfe_matrix *A, uint32_t flags, size_t *ws_bytes);

/* Bytes of the gfe_result buffers gfe_echelon writes for A and flags (the
 * outputs of Eq. (echelon), Section 3.1), each sized for the worst case
 * r = k = min(m, n) with rows packed tight and every buffer rounded up to 256
 * bytes: rank (8 bytes), pivot_cols and pivot_rows (k int64 each), R (k rows
 * of n entries); with GFE_WANT_TRANSFORM or GFE_WANT_DENSE_T also M (k x k)
 * and K (m x k); E (m x n) with GFE_WANT_DENSE_E, T (m x m) with
 * GFE_WANT_DENSE_T.  A row of c entries takes c bytes (GFE_U8) or
 * ceil(c / 64) 8-byte words (GFE_BITS64).  Host only: no device call, and
 * A->data is checked as for gfe_echelon but never read.  GFE_EINVAL for a
 * bad matrix or a NULL out_bytes. */
gfe_status gfe_query_result_bytes(const gfe_matrix *A, uint32_t flags, size_t *out_bytes);

/*
 * gfe_echelon -- the whole method: Step 1 (Tasks ClearDown, Extend,
 * UpdateRow, UpdateRowTrafo), Step 2 (Task RowLengthen) and Step 3 (Tasks
 * Copy, PreClearUp, ClearUp) of "The Chief" (Section 3, Algorithm "The
 * Chief"), with the single-block echelonisation ECH done recursively by the
 * same scheme (Section 2.3.2).  M and K are written only with
 * GFE_WANT_TRANSFORM (dense T needs it).
 */
gfe_status gfe_echelon(const gfe_matrix *A, const gfe_result *out, uint32_t flags,
                       void *ws, size_t ws_bytes, void *stream);

/* gfe_rank -- Step 1 without UpdateRowTrafo (the rank-only variant the paper
 * lists in Section 1); writes r to rank_dev and, if non-NULL, Ups and rho. */
gfe_status gfe_rank(const gfe_matrix *A, int64_t *rank_dev, int64_t *pivot_cols,
                    int64_t *pivot_rows, uint32_t flags, void *ws, size_t ws_bytes,
                    void *stream);

/*
 * gfe_batch_echelon -- count independent matrices (any sizes, any fields)
 * echelonised concurrently: small matrices (gfe_set_batch_small_max) by one
 * launch of a kernel that gives each its own thread block, the others by a
 * pool of host workers (gfe_set_batch_workers, default 8), each with its own
 * CUDA stream and its own slice of the workspace, taking them in order; the
 * work is ordered after what was queued on `stream` before the call and
 * `stream` waits for all of it.
 * outs[i] receives the result of As[i], identical to a separate gfe_echelon
 * call.  The paper's matrices are independent problems; the concurrency is
 * the GPU-side analogue of its many workers (Section 2.1).
 * gfe_query_batch_workspace: workers x the largest single workspace of the
 * matrices the workers take, plus m x ceil16(n) bytes (GF(2): m x
 * ceil128(n) / 8) for each small matrix and its job table.
 */
gfe_status gfe_query_batch_workspace(const gfe_matrix *As, int32_t count, uint32_t flags,
                                     size_t *ws_bytes);
gfe_status gfe_batch_echelon(const gfe_matrix *As, const gfe_result *outs, int32_t count,
                             uint32_t flags, void *ws, size_t ws_bytes, void *stream);
/*
 * Matrices of a batch with at most `side` rows and columns (side <= 2048,
 * the default) and work m n min(m,n) at most max_work (<= 0: the default
 * 4e9; the work of a GF(2) matrix counts a 16th, and that of a p <= 13 byte
 * matrix 1/2.5, for their faster kernels), over GF(2) (GFE_BITS64) or any odd prime
 * p <= 251 (GFE_U8), with no
 * dense E / T asked for, are echelonised together by ONE kernel launch per
 * kind (p <= 13, larger p, GF(2)), one thread block per matrix, with no host
 * round trip; the others go to the workers below.  side = 0 sends every
 * matrix to the workers.  GFE_EINVAL if side < 0.
 */
gfe_status gfe_set_batch_small_max(int32_t side, double max_work);
/* number of concurrent workers of gfe_batch_echelon (<= 0: default 8; at
 * most GFE_MAX_BATCH_WORKERS, larger values are clamped to it) */
#define GFE_MAX_BATCH_WORKERS 256
gfe_status gfe_set_batch_workers(int32_t workers);
/*
 * How gfe_batch_echelon's workers wait for the GPU (a leaf's result, the end
 * of a matrix): GFE_WAIT_SPIN polls (lowest latency, one host core per
 * worker), GFE_WAIT_BLOCK sleeps on a blocking-sync event (many workers on
 * few cores), GFE_WAIT_AUTO (the default) sleeps when there are more workers
 * than host threads.  GFE_EINVAL for any other value.
 */
#define GFE_WAIT_AUTO 0
#define GFE_WAIT_SPIN 1
#define GFE_WAIT_BLOCK 2
gfe_status gfe_set_wait_policy(int32_t policy);

/*
 * Serving form: requests arrive one matrix at a time and are echelonised
 * concurrently by `workers` host workers with their own CUDA streams.  The
 * server owns one device arena of hbm_cap_bytes (its HBM admission cap); a
 * request is admitted when a worker is free and its workspace
 * (gfe_query_workspace) fits in the arena, and any queued request that fits
 * may go first, so requests that arrive while others run join as slots and
 * memory free up and their work overlaps on the GPU.  The result is that of
 * gfe_echelon on the same matrix (the paper's computation, Section 3).
 *   gfe_submit: A and out as for gfe_echelon; both must stay valid and
 *     untouched until the request is done.  The request is ordered after the
 *     work queued on `stream` before the call.  A request whose workspace
 *     exceeds the cap fails with GFE_ENOMEM.
 *   gfe_poll: GFE_EBUSY while pending, else GFE_OK with the request's status.
 *   gfe_wait: blocks up to timeout_us (< 0: forever); GFE_ETIMEOUT if still
 *     pending.  When a request is done its outputs are complete on the device.
 *   gfe_server_latency: submit-to-done time of a finished request in
 *     microseconds (host clock); release != 0 forgets the ticket.
 *   gfe_server_destroy: finishes every queued request, then frees the arena.
 */
typedef struct gfe_server gfe_server;
gfe_status gfe_server_create(gfe_server **server, size_t hbm_cap_bytes, int32_t workers, int32_t device);
gfe_status gfe_submit(gfe_server *server, const gfe_matrix *A, const gfe_result *out, uint32_t flags,
                      void *stream, uint64_t *ticket);
gfe_status gfe_poll(gfe_server *server, uint64_t ticket, gfe_status *done_status);
gfe_status gfe_wait(gfe_server *server, uint64_t ticket, int64_t timeout_us, gfe_status *done_status);
gfe_status gfe_server_latency(gfe_server *server, uint64_t ticket, double *us, int32_t release);
gfe_status gfe_server_destroy(gfe_server *server);
/* Server requests of work m n min(m,n) at most max_work that the batched
 * form's one-launch kernels take are grouped: a worker runs every such
 * queued request with the same flags (up to 256) as one batched call.
 * Default 2e7 (about 270^3); <= 0 turns grouping off.  Applies to requests
 * admitted after the call. */
gfe_status gfe_set_server_group_work(double max_work);

/*
 * Solving and null spaces from the echelon result.  The transformation
 * matrix is what gives these (the paper's list of variants, Section 1):
 * with T = (M 0; K 1) P_rho and T A = E (Eq. (echelon), Section 3.1),
 *   left null space  {y : y A = 0} has the basis (K 1) P_rho, the rows r..m-1
 *     of T: row t holds K[t, s] at column rho_s and 1 at column rho_bar_t;
 *   right null space {x : A x = 0} has the basis whose vector j is 1 at the
 *     non-pivot column Ups_bar_j, 0 at the other non-pivot columns and
 *     R[l, j] at the pivot column Ups_l (from E_top x = 0, E_top = -RREF);
 *   A X = B: column b is consistent iff (T b)[r..] = K b[rho] + b[rho_bar]
 *     is zero, and then X[Ups_l] = -(M b[rho])[l] with every non-pivot
 *     variable 0 solves it.
 * A describes the matrix that was echelonised (p, m, n, fmt; its data is
 * not read) and res is gfe_echelon's result for it (device rank, pivots,
 * and K (left), R (right), or M and K (solve)).  Storage is A's: GFE_U8
 * residues, or GF(2) rows of 64-bit words (ld in bytes, a multiple of 8).
 *
 * gfe_nullspace: writes the basis, one vector per row, into N: (m - r) rows
 *   of m entries (GFE_LEFT) or (n - r) rows of n entries (GFE_RIGHT); N must
 *   hold m (n) rows when the rank is not known on the host.  Asynchronous
 *   on `stream` (the pivots stay on the device).  GFE_EINVAL for a bad side,
 *   a missing K (left) or R (right), or ldn too small.
 * gfe_solve: B is m x k, X is n x k (pitches ldb, ldx in bytes); X gets the
 *   solution above for every column (meaningful where consistent[j] = 1);
 *   consistent (device, k int32) gets 1 for columns in the column space of
 *   A, else 0.  ws: gfe_solve_workspace(A, k) bytes (its last 256 bytes hold
 *   the call's status word).  The call reads the rank on `stream` to size
 *   its two multiply-adds, and returns once the result is complete there.
 */
#define GFE_LEFT 0
#define GFE_RIGHT 1
gfe_status gfe_nullspace(const gfe_matrix *A, const gfe_result *res, int32_t side, void *N, int64_t ldn,
                         void *stream);
size_t gfe_solve_workspace(const gfe_matrix *A, int64_t k);
gfe_status gfe_solve(const gfe_matrix *A, const gfe_result *res, const void *B, int64_t ldb, int64_t k,
                     void *X, int64_t ldx, int32_t *consistent, void *ws, size_t ws_bytes, void *stream);

/*
 * gfe_mad -- the job MAD (Section 4.1): C := W + A B over GF(p), A m x k,
 * B k x n, W and C m x n, all GFE_U8 residues (device).  W may be NULL
 * (C := A B, the job MUL) and may equal C.  ws: gfe_mad_workspace() bytes;
 * its last 256 bytes hold the call's own status word, which the call zeroes
 * on `stream` before the product.  The call returns once the product is
 * complete on `stream`: it reads that word with a copy on `stream` (no
 * device-wide or legacy-stream synchronisation), and returns GFE_ETIMEOUT if
 * a bounded wait of the tensor-core kernel gave up.  Errors of one call are
 * never reported by another.  The block multiply-add is the dominant cost of
 * the method (Section 5, Lemma "closecosts").
 */
size_t gfe_mad_workspace(int32_t p, int64_t m, int64_t n, int64_t k);
gfe_status gfe_mad(int32_t p, int64_t m, int64_t n, int64_t k,
                   const uint8_t *W, int64_t ldw, const uint8_t *A, int64_t lda,
                   const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                   uint32_t flags, void *ws, size_t ws_bytes, void *stream);

/*
 * gfe_mad_gf2 -- the job MAD (Section 4.1) over GF(2) on bit-packed rows:
 * C := W + A B, A m x k, B k x n, W and C m x n, rows of 64-bit words
 * (GFE_BITS64 layout: bit c % 64 of word c / 64 is column c), pitches in
 * bytes (multiples of 8).  W may be NULL (C := A B) and may equal C.  Pad
 * bits of the inputs are ignored; those of C are written 0.  The kernel is
 * the Method of the Four Russians: tables of all 256 combinations of 8 rows
 * of B in shared memory, one table entry per row of A and 8 bits of k.
 * Asynchronous on `stream`; allocates nothing.  Products with few output
 * tiles split k over thread blocks that XOR into C atomically.
 *
 * gfe_gf2_peaks -- measures the two rates that bound that kernel on this
 * GPU: LOP3 instructions per second (one LOP3 computes (a AND b) XOR c on 32
 * bits, i.e. 32 GF(2) multiply-adds) and bytes per second of conflict-free
 * 128-bit shared-memory loads.  Synchronises `stream`.
 */
gfe_status gfe_mad_gf2(int64_t m, int64_t n, int64_t k, const uint64_t *W, int64_t ldw,
                       const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb,
                       uint64_t *C, int64_t ldc, void *stream);
gfe_status gfe_gf2_peaks(double *lop3_per_s, double *lds_bytes_per_s, void *stream);

/*
 * gfe_mad_noalloc -- the same multiply-add as gfe_mad, C := W + A B over
 * GF(p) on GFE_U8 residues, for callers that cannot allocate device memory:
 * a caller that owns a fixed device-memory budget and does not let libraries
 * grow it, or one on a latency-critical path, where cudaMalloc / cudaFree
 * may block or synchronise the device.  The paper has no counterpart; this
 * is an interface convenience of this library.
 * Needs no workspace: its scratch is a library-owned device array of
 * gfe_mad_noalloc_max_bytes() bytes (32 MiB).  A product whose scratch
 * (gfe_mad_workspace()) would exceed it is rejected with GFE_EINVAL; so is a
 * p that is not a prime <= 251, checked first, as in gfe_mad.
 * First call on a device: the CUDA runtime loads the library's device code
 * lazily, so the first call on each device (with that device current) loads
 * it, reserves the 32 MiB array, and looks up the array's device address;
 * that call can therefore fail with GFE_ECUDA when the device is full.  Make
 * it once as a warm-up, before any stream capture; from then on the device
 * holds the array until the process exits and no call allocates.
 * All calls on a device share the array and it keeps the last call's
 * contents (every element a call reads it first writes; the status word is
 * zeroed by each call).  Calls whose work overlaps on the GPU race on it and
 * must be ordered by the caller.  Like gfe_mad, the call returns once the
 * product is complete on `stream`.
 */
size_t gfe_mad_noalloc_max_bytes(void);
gfe_status gfe_mad_noalloc(int32_t p, int64_t m, int64_t n, int64_t k,
                           const uint8_t *W, int64_t ldw, const uint8_t *A, int64_t lda,
                           const uint8_t *B, int64_t ldb, uint8_t *C, int64_t ldc,
                           uint32_t flags, void *stream);

/*
 * Block partition policy of the planner (the "carefully chosen" block sizes
 * a_i, b_j of Section 3.1 and Section 5).  A block (or the whole input)
 * whose larger side exceeds `threshold` is split into square blocks of side
 * `block`; smaller ones into leaf blocks of at most 1024 rows x 64 columns
 * (256 columns for GF(2)), which the one-CTA ECH kernel echelonises.
 * threshold <= 0 and block <= 0 (the default): both equal gfe_auto_block of
 * the call's field and shape.  One of them <= 0: it takes the other's value.
 * GFE_EINVAL (policy unchanged) unless block <= threshold.  Blocks that are
 * multiples of 64 keep every operand aligned for the tensor-core path
 * (others fall back to the plain multiply-add where misaligned).  Process
 * wide.  Results never depend on it.
 */
gfe_status gfe_set_block_policy(int64_t threshold, int64_t block);

/* The block side the default policy uses for an m x n matrix over GF(p):
 * a table measured on GB300 (GF(2): 2048 below max(m, n) = 12288, 3072 up to
 * 65536, 6144 above; 3 <= p <= 13: 2048; p > 13: 1024).  The Python autotuner
 * (paper_1806_04211_gb300.gfe.autotune_block) times candidates on a seeded
 * matrix of the caller's shape and sets the winner with
 * gfe_set_block_policy. */
int64_t gfe_auto_block(int32_t p, int64_t m, int64_t n);

/* Rows of a leaf block in the planner's leaf grid: 1..1024, or 0 for the
 * default, which is the most the field's leaf kernels take (1024 for
 * p <= 13, 256 for larger p); larger values are capped at that.  Leaves of
 * at most 256 rows run the fp32 leaf kernel for every p > 2.  Process wide.
 * Results never depend on it.  GFE_EINVAL outside [0, 1024]. */
gfe_status gfe_set_leaf_rows(int64_t rows);
/* Tiles per thread block of the multiply-adds the planner runs beside its
 * critical path (the side streams): enough blocks are launched that none
 * takes more, so SMs come free for the critical path every few tiles.
 * 0 = one persistent block per SM.  Default 4.  Results never depend on it.
 * GFE_EINVAL outside [0, 1024]. */
gfe_status gfe_set_side_tiles(int32_t tiles);

/* Kernel profile of the calls made since the last reset (all streams).
 * While enabled every launch is counted; launches of the kinds selected by
 * the mask (bit k = kind k, -1 = all) are also timed with CUDA events
 * recorded on the stream they are launched on.  mask 0 disables. */
typedef struct {
    int64_t launches[8];     /* by kind: 0 MAD tensor, 1 MAD plain, 2 ECH leaf,   */
    double  ms[8];           /*   3 row extract/riffle (REX, RRF), 4 column        */
                             /*   extract/riffle (CEX, CRZ), 5 copy/zero/ADI,     */
                             /*   6 convert/assemble, 7 other                     */
    double  madds[8];        /* algorithmic multiply-adds done by the MAD kinds  */
    double  bytes[8];        /* algorithmic bytes of the tensor-core MAD: A, B,  */
                             /*   W (if any) read and C written once             */
    int64_t timed[8];        /* launches that were timed                         */
    int64_t host_syncs;      /* stream synchronisations made by the planner      */
    double  host_wait_ms;    /* host time spent blocked in them                  */
    double  host_ms;         /* host time inside the planner (all calls, summed  */
                             /*   over threads), waits included                  */
} gfe_profile;
gfe_status gfe_profile_enable(int32_t mask);
gfe_status gfe_profile_read(gfe_profile *out, int32_t reset);

/* Launch trace: while the profile is enabled and the trace holds fewer than
 * `capacity` records, every timed launch also leaves one record: its kind,
 * its shape (m x n x k for a multiply-add, rows x cols for the others,
 * k = 0), the CUDA stream it ran on and its start and duration.  The
 * tensor-core multiply-add times itself on the device (%globaltimer at its
 * first CTA's start and its last CTA's end, in a device buffer of `capacity`
 * slots that gfe_trace_enable allocates), so tracing it records no events;
 * the other kinds are timed with CUDA events.  Starts are relative to the
 * first traced launch of the same clock (field `clock`).  gfe_trace_enable(0)
 * stops tracing and drops the records and the buffer; gfe_trace_read waits
 * for the device, copies up to `cap` records to `out` (may be NULL with cap
 * 0), sets *count to the number held, and drops them all if `reset`. */
typedef struct {
    int32_t kind;            /* as gfe_profile's index                          */
    int32_t clock;           /* 0: CUDA events, 1: device %globaltimer          */
    int64_t m, n, k;
    uint64_t stream;         /* the cudaStream_t handle, as an integer          */
    double  start_ms;
    double  ms;
} gfe_trace_record;
gfe_status gfe_trace_enable(int64_t capacity);
gfe_status gfe_trace_read(gfe_trace_record *out, int64_t cap, int64_t *count, int32_t reset);

/*
 * Failure-detection self-test: a kernel waits, with the bounded wait every
 * pipeline wait of the library uses, on an mbarrier phase that nothing
 * completes; after limit_us microseconds it gives up, records the error and
 * returns normally.  Returns GFE_ETIMEOUT when the wait gave up as designed
 * (no fault, no hang, the context stays usable).  No counterpart in the
 * paper.
 */
gfe_status gfe_selftest_wait_timeout(int64_t limit_us, void *stream);

const char *gfe_status_str(gfe_status s);
const char *gfe_last_error(void);
const char *gfe_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GFE_H */
