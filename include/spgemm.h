/*
 * spgemm.h - C ABI of the GB300 (sm_103a) hash-based multi-phase SpGEMM.
 *
 * Computes C = A * B for sparse matrices in CSR form, following the three
 * phases of arXiv 2512.12036 Section III: row grouping by intermediate
 * products, the allocation (symbolic) phase that finds the structure of C,
 * and the accumulation (numeric) phase that produces sorted, canonical rows.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All matrix arrays are DEVICE pointers on the plan's device. Indices are
 *   int32, values fp32. Row r of a matrix occupies [row_ptr[r], row_ptr[r+1])
 *   of col_idx/vals; row_ptr[0] need not be 0, so a block of rows of a larger
 *   matrix can be passed as a view (row_ptr + r0, rows = r1 - r0) without
 *   copying. spgemm_csr.nnz is the length of the col_idx/vals arrays.
 * - Input rows may be unsorted and may repeat a column (repeats are summed).
 *   Stored zeros are structure: an entry of C exists wherever some stored
 *   a_ik meets some stored b_kj, whatever the values. Output rows are sorted
 *   by column with no repeats.
 * - The caller owns and allocates every device buffer, including the
 *   workspace; nothing here calls cudaMalloc after spgemm_plan_create.
 * - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *   enqueued on it; an entry point only blocks the host where it says so.
 * - Return value: SPGEMM_OK or one of the SPGEMM_ERR_* codes. Conditions the
 *   kernels find on the device (an index out of range, a row_ptr that is not
 *   monotone, an internal capacity guard) are recorded in a status word in
 *   the workspace and reported by the next entry point that synchronises,
 *   or by spgemm_status(). Kernels never fault or trap on bad input: they
 *   skip the offending access and record the condition.
 * - Value tolerance: every C value is within 1e-5 * sum_k |a_ik||b_kj| of
 *   the exact result. A plain fp32 sum of t products is only guaranteed
 *   within gamma_t = t*2^-24 of that scale, below 1e-5 for t <= 167
 *   (opts.fp32_max_terms). Entries that can gather more products (rows with
 *   more than fp32_max_terms A entries, on columns of B with more than
 *   fp32_max_terms entries) are summed in fp64, or as fp32 partial sums of
 *   at most 128 terms added together in fp64.
 */
#ifndef SPGEMM_H
#define SPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SPGEMM_OK = 0,
    SPGEMM_ERR_INVALID = 1,   /* null pointer, bad dimensions, bad row_ptr or index */
    SPGEMM_ERR_WORKSPACE = 2, /* workspace missing or smaller than spgemm_workspace_bytes */
    SPGEMM_ERR_OVERFLOW = 3,  /* result does not fit int32 row pointers: split A into row blocks */
    SPGEMM_ERR_BUDGET = 4,    /* a memory budget given by the caller is exceeded */
    SPGEMM_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
    SPGEMM_ERR_CUDA = 6,      /* a CUDA runtime call failed */
    SPGEMM_ERR_INTERNAL = 7,  /* an internal capacity guard tripped (a bug) */
    SPGEMM_ERR_UNSUPPORTED = 8 /* shape outside what the kernels handle */
};

/* CSR matrix view (device pointers). vals may be NULL where only structure is read. */
typedef struct {
    int32_t rows;
    int32_t cols;
    int64_t nnz;              /* length of col_idx / vals */
    const int32_t* row_ptr;   /* rows + 1 */
    const int32_t* col_idx;   /* nnz */
    const float* vals;        /* nnz */
} spgemm_csr;

/* Tunables. Defaults come from spgemm_opts_default(); the row-group
 * boundaries play the role of the paper's Table 1 (which fixes IP ranges
 * 0-31 / 32-511 / 512-8191 / >=8192 for an H200) and are re-chosen for the
 * GB300's 227 KB of shared memory per block. */
typedef struct {
    int32_t fp32_max_terms;   /* default 167: rows with more A entries accumulate in fp64 */
    int32_t esc_max;          /* default 32: IP and A-row length bound of the in-register tier */
    int32_t warp_max_ip;      /* default 1024: allocation phase, warp-per-row hash tier */
    int32_t block_max_ip;     /* default 16384: allocation phase, block-per-row hash tier */
    int32_t warp_max_nnz;     /* default 512: accumulation phase, warp-per-row hash tier */
    int32_t block_max_nnz;    /* default 8192: accumulation phase, block-per-row hash tier */
    int32_t panel_cols;       /* default 16384 (a power of two, 1024..16384): column panel of
                                 the dense heavy-row accumulator */
    int32_t row_cache_mb;     /* default 0: MiB of workspace for the allocation phase's
                                 row bitmaps. The allocation phase's bitmap tier keeps the
                                 column bitmap (B.cols bits) and the entry count of each
                                 column panel (4 bytes per panel) of every row that the
                                 accumulation phase will take in a dense tier, one slot per
                                 row while slots last; the accumulation phase then reads a
                                 row's columns from its slot instead of marking every product
                                 again. Rows without a slot are unaffected. B.cols must be at
                                 most 1,572,864 for the cache to be used. */
    int32_t dense_splits;     /* default 0 (automatic): work items per heavy row in the
                                 fp64-bound dense tier for rows with a cached bitmap. Each item
                                 takes one of that many consecutive column ranges of the row,
                                 so one row runs on up to that many SMs at once; items write
                                 disjoint, ordered slices of the row (no merge step). 0 picks
                                 one range per 128K intermediate products, at most 8 (1 to 8
                                 by the row's product count); k > 0 fixes k ranges for every
                                 row. */
    int32_t stage_b;          /* default 0: when 1, rows of the allocation phase's block hash
                                 tier with at most 8192 intermediate products first gather
                                 their B row-pointer pairs and copy all their B segments into
                                 shared memory (cp.async, double-buffered over rows), then
                                 insert from there: a software form of the paper's near-memory
                                 range-2 access (Section IV-D). Same results either way. */
    int32_t narrow_warps;     /* default 0 (= 8): warps per block (1..16) of the narrow tiers
                                 (B with at most 1024 columns: one warp per row with a dense
                                 per-warp accumulator over B's columns) */
    int32_t narrow_max_ip;    /* default 0 (= 32768): largest IP of a row in the narrow tiers */
    int32_t hash_load_pct;    /* default 0 (= 50): target load of the hash tiers' tables in
                                 percent (25..90); a row's table is the smallest power of two
                                 holding its keys at that load */
    int32_t reserved[3];
} spgemm_opts;

typedef struct spgemm_plan spgemm_plan;

/* Fill opts with the defaults above. */
int spgemm_opts_default(spgemm_opts* opts);

/* Create a plan on CUDA device `device` (queries SM count and occupancy once).
 * opts may be NULL for defaults. A plan holds no per-call state and may be
 * shared by concurrent calls that use distinct workspaces. */
int spgemm_plan_create(spgemm_plan** plan, const spgemm_opts* opts, int device);
int spgemm_plan_destroy(spgemm_plan* plan);

/* Bytes of workspace every phase below needs for these operand shapes
 * (depends on A.rows, A.nnz, B.rows, B.cols only, never on values). */
int spgemm_workspace_bytes(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                           size_t* bytes);

/* Zero the workspace's control block (status word, counters). Call once on
 * a newly allocated workspace before its first use; enqueued on `stream`. */
int spgemm_workspace_init(const spgemm_plan* plan, void* ws, size_t ws_bytes, void* stream);

/* Intermediate-product counting (Algorithm 1).
 * ip_row   [out, device, A.rows int64]: IP_i = sum over stored (i,k) of |row k of B|.
 * ip_total [out, host, nullable]: sum of ip_row; when non-NULL the call
 *          synchronises the stream and also reports device-side errors.
 * Requires A.cols == B.rows. Only the structure of A and B is read. */
int spgemm_count(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B, void* ws,
                 size_t ws_bytes, int64_t* ip_row, int64_t* ip_total, void* stream);

/* Row grouping (Section III-B): a stable partition of rows 0..n-1 by key
 * into ngroups = nthr + 1 groups, group g holding thr[g-1] <= key < thr[g].
 * map [out, device, n int32] lists the rows group by group, ascending row id
 * inside a group; offsets [out, device, ngroups+1 int32]. nthr <= 32.
 * key and thr are device int64 arrays. */
int spgemm_group(const spgemm_plan* plan, const int64_t* key, int32_t n, const int64_t* thr,
                 int32_t nthr, void* ws, size_t ws_bytes, int32_t* map, int32_t* offsets,
                 void* stream);

/* Allocation (symbolic) phase (Algorithms 2-4): the number of distinct
 * columns of every row of C.
 * ip_row    [in, device]: the output of spgemm_count for the same A and B.
 * row_nnz   [out, device, A.rows int32].
 * nnz_total [out, host, nullable]: int64 sum; non-NULL synchronises and
 *           reports device-side errors.
 * The workspace must stay untouched between this call and spgemm_numeric
 * for the same A and B (it carries the allocation phase's state). */
int spgemm_symbolic(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                    const int64_t* ip_row, void* ws, size_t ws_bytes, int32_t* row_nnz,
                    int64_t* nnz_total, void* stream);

/* Row pointers of C from the row counts (the rpt_C recurrence of
 * Algorithms 2-3, computed as an exclusive scan).
 * row_nnz [in, device, n], row_ptr [out, device, n+1] with row_ptr[0] = 0.
 * total [out, host, nullable]: non-NULL synchronises; the call then returns
 * SPGEMM_ERR_OVERFLOW when the sum exceeds INT32_MAX (row_ptr is then
 * unspecified: pass a block of rows at a time instead). */
int spgemm_row_ptr(const spgemm_plan* plan, const int32_t* row_nnz, int32_t n, void* ws,
                   size_t ws_bytes, int32_t* row_ptr, int64_t* total, void* stream);

/* Row pointers without a caller workspace (no counterpart in the paper; an
 * addition for callers that cannot allocate device memory: plugins whose
 * host framework owns every device allocation, fixed-budget or real-time
 * services that forbid allocation after start-up, code that runs where
 * cudaMalloc is not allowed or would synchronise the device).
 * Same result and arguments as spgemm_row_ptr, but the scan's scratch lives
 * in a fixed array compiled into the library (about 132 KB, resident on
 * every GPU that loads the library until the process exits); the call
 * allocates nothing. Limits and rules:
 *  - n <= 2^26 (67,108,864) rows, else SPGEMM_ERR_UNSUPPORTED before any work;
 *  - the calling thread's current device must be the plan's device;
 *  - the first call on each device looks up the scratch's device address
 *    (cudaGetSymbolAddress), and so does the first call after the device's
 *    context changes (cudaDeviceReset, a new primary context); make such a
 *    call before any stream capture;
 *  - within one process every call on a device shares the one scratch
 *    array, so calls that overlap on the GPU (different streams or host
 *    threads) race: order them on one stream or serialise them. Separate
 *    processes each get their own copy of the array.
 * total [out, host, nullable]: as for spgemm_row_ptr (non-NULL synchronises
 * and returns SPGEMM_ERR_OVERFLOW past INT32_MAX). */
int spgemm_row_ptr_static(const spgemm_plan* plan, const int32_t* row_nnz, int32_t n,
                          int32_t* row_ptr, int64_t* total, void* stream);

/* Accumulation (numeric) phase with sorting (Algorithm 5 and the
 * column-index sorting step): rows [row_begin, row_end) of C.
 * ip_row    [in, device, A.rows]: from spgemm_count.
 * row_ptr_C [in, device, row_end-row_begin+1]: row pointers of this block
 *           of rows (row_ptr_C[0] = 0, e.g. spgemm_row_ptr on row_nnz + row_begin).
 * col_C, val_C [out, device, row_ptr_C[last] entries].
 * Does not synchronise; errors found on the device surface via spgemm_status. */
int spgemm_numeric(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                   const int64_t* ip_row, int32_t row_begin, int32_t row_end,
                   const int32_t* row_ptr_C, void* ws, size_t ws_bytes, int32_t* col_C,
                   float* val_C, void* stream);

/* Backward of C = A*B with respect to the stored values (the gradient rule
 * of the pruned-GNN aggregation, Eq. 3, read per stored value):
 *   dA[j] = sum_{t in row k of B} dC(i, colB[t]) * valB[t]   for A entry j = (i,k)
 *           (an SDDMM of dC * B^T sampled at A's pattern),
 *   dB[t] = sum_{A entries j = (i,k)} valA[j] * dC(i, colB[t])   for B entry t in row k
 *           (A^T * dC sampled at B's pattern).
 * row_ptr_C [device, A.rows+1], col_C [device, nnz_C]: C's structure as
 *   spgemm produced it (rows sorted); it must contain every column a
 *   product of row i reaches (otherwise SPGEMM_ERR_INVALID on the status).
 * dC [device, nnz_C]: the gradient on C's stored values.
 * dA [out, device, A.nnz, nullable], dB [out, device, B.nnz, nullable]:
 *   fully overwritten (an entry that meets no product, e.g. an A entry
 *   whose row of B is empty, gets 0); sums are accumulated in fp64 and
 *   rounded once.
 * Workspace: spgemm_backward_workspace_bytes (includes B.nnz + A.nnz fp64
 * slots). Does not synchronise. C must fit int32 row pointers. */
int spgemm_backward_workspace_bytes(const spgemm_plan* plan, const spgemm_csr* A,
                                    const spgemm_csr* B, size_t* bytes);
int spgemm_backward(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                    const int32_t* row_ptr_C, const int32_t* col_C, int64_t nnz_C,
                    const float* dC, float* dA, float* dB, void* ws, size_t ws_bytes,
                    void* stream);

/* Dense fp32 GEMM for the pruned GNN layer's dense products (Section IV-C,
 * Eq. 1: the aggregated features times W_l; Eq. 3 and the weight gradient:
 * dY * W_l^T and C^T * dY):
 *   C[M x N] = op(A)[M x K] * op(B)[K x N]
 * All matrices row-major fp32 on the plan's device with leading dimensions
 * (elements): op(A) = A (M x K, lda >= K) or, with trans_a = 1, A^T of a
 * stored K x M matrix (lda >= M); op(B) = B (K x N, ldb >= N) or, with
 * trans_b = 1, B^T of a stored N x K matrix (ldb >= K); ldc >= N. C is
 * overwritten (K = 0 gives zeros). Products are fp32 fused multiply-adds;
 * a long reduction with few output tiles (K deep, e.g. C^T * dY over all
 * rows of a graph) is split over blocks along K when the caller passes a
 * workspace of spgemm_dense_gemm_workspace_bytes (256-byte aligned; 0 bytes
 * when no split is needed): each block's fp32 partial sum is added into an
 * fp64 accumulator there and rounded once. Without one, each output tile
 * runs the whole reduction in one block. Returns SPGEMM_ERR_INVALID for
 * bad sizes or pointers; does not synchronise. */
int spgemm_dense_gemm_workspace_bytes(const spgemm_plan* plan, int32_t M, int32_t N, int32_t K,
                                      size_t* bytes);
int spgemm_dense_gemm(const spgemm_plan* plan, int32_t M, int32_t N, int32_t K, const float* A,
                      int64_t lda, int32_t trans_a, const float* B, int64_t ldb, int32_t trans_b,
                      float* C, int64_t ldc, void* ws, size_t ws_bytes, void* stream);

/* Allocation callback for spgemm(): must return device buffers of nnz
 * entries (col and val) and 0, or nonzero to abort. */
typedef int (*spgemm_alloc_fn)(void* ctx, int64_t nnz, int32_t** col, float** val);

/* The whole product in one call: count, symbolic, row pointers, alloc,
 * numeric (the workspace is initialised first). ip_row and row_nnz are
 * device scratch of A.rows entries each,
 * row_ptr_C the device output of A.rows+1 entries. Synchronises twice (for
 * the nnz of C and for the final status). *nnz_C receives the nnz of C.
 * Returns SPGEMM_ERR_OVERFLOW (before allocating) when C needs more than
 * INT32_MAX entries. */
int spgemm(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B, void* ws,
           size_t ws_bytes, int64_t* ip_row, int32_t* row_nnz, int32_t* row_ptr_C,
           spgemm_alloc_fn alloc, void* alloc_ctx, int64_t* nnz_C, void* stream);

/* The whole product without host synchronisation or allocation, so that it
 * can be captured in a CUDA graph and replayed (e.g. thousands of small,
 * uneven products stacked as one block-diagonal A and one stacked B: the
 * result is the stacked per-problem products, since (blockdiag A_b) *
 * (stacked B_b) = stacked (A_b * B_b)). Same phases as spgemm().
 * ip_row [device, A.rows int64], row_nnz [device, A.rows int32]: scratch
 *   (left holding IP and nnz per row).
 * row_ptr_C [out, device, A.rows+1], col_C / val_C [out, device, capacity]:
 *   caller-sized output; capacity <= INT32_MAX.
 * nnz_C [out, DEVICE int64]: the number of entries of C.
 * When C needs more than `capacity` entries, nothing is written to
 * col_C/val_C, *nnz_C still holds the size, and the status word records
 * SPGEMM_ERR_BUDGET (read it with spgemm_status after the stream is done).
 * The workspace must be initialised (spgemm_workspace_init) before first use;
 * the status word is sticky until read. */
int spgemm_batched(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B, void* ws,
                   size_t ws_bytes, int64_t* ip_row, int32_t* row_nnz, int32_t* row_ptr_C,
                   int32_t* col_C, float* val_C, int64_t capacity, int64_t* nnz_C, void* stream);

/* One Markov-clustering step after the expansion (Algorithm 6), on the rows
 * of M^T (a column of M is a row of M^T, so with E = M^T * M^T = (M M)^T
 * every column operation of the algorithm is a row operation here):
 *   prune: drop entries with value < theta; top-k: keep the k largest of
 *   each row (ties: the smaller column; k < 0 keeps all); inflate: v^r;
 *   normalise: divide by the row sum.
 * order 0 prunes and cuts on the values, then inflates (the algorithm's
 * order); order 1 inflates first and decides on the fp32-rounded inflated
 * values. Decisions are made in fp32, weights and sums in fp64.
 * E: rows sorted by column (as spgemm produces them). Outputs (device):
 * row_ptr_out [E.rows+1], col_out / val_out [at least min(E.nnz, E.rows*k)
 * entries] in column order. nnz_out [host, nullable]: non-NULL synchronises.
 * Workspace: spgemm_workspace_bytes for a matrix of E.rows rows.
 * theta <= 0, k < 0, r = 1 is a plain row normalisation (the algorithm's
 * column-stochastic start on M^T). */
int spgemm_mcl_step(const spgemm_plan* plan, const spgemm_csr* E, float theta, int32_t k, float r,
                    int32_t order, void* ws, size_t ws_bytes, int32_t* row_ptr_out,
                    int32_t* col_out, float* val_out, int64_t* nnz_out, void* stream);

/* --- Pruned GNN layer (Section IV-C, Eqs. 1-3): X_l = A * TopK(X_{l-1}, k) * W_l.
 * The products with the dense W_l are plain dense GEMMs and are left to the
 * caller (a BLAS); these three calls supply the sparse steps around the
 * SpGEMM A * TopK(X) and its backward (spgemm_backward gives the gradient on
 * TopK's pattern, i.e. M_k (.) (A^T dC) of Eq. 3). */

/* TopK of Eq. 2 on each row of the dense row-major n x d matrix X (leading
 * dimension ldx >= d, device): keeps the min(k, d) largest values of the
 * row, the mask M_k and its values as CSR with row_ptr [n+1] (row i starts
 * at i*min(k,d)), col / val [n*min(k,d)] in ascending column order (device,
 * caller-allocated). Order: fp32 values by IEEE total order (a positive NaN
 * ranks above +inf, a negative one below -inf); equal values go to the
 * smaller column. Stored zeros count like any value. k = 0 gives empty rows.
 * Errors: SPGEMM_ERR_INVALID (null pointers, k < 0, ldx < d),
 * SPGEMM_ERR_OVERFLOW (n*min(k,d) beyond int32). Asynchronous. */
int spgemm_topk_dense(const spgemm_plan* plan, const float* X, int32_t n, int32_t d, int64_t ldx,
                      int32_t k, int32_t* row_ptr, int32_t* col, float* val, void* stream);

/* X[i, j] += v for every entry (i, j) of M, v = vals[q] (or M->vals[q] when
 * vals is NULL): M (.) applied to a gradient on M's pattern (Eq. 3) when X
 * starts at zero. X: dense row-major M->rows x ldx (ldx >= M->cols, device).
 * Repeated columns add up. ws: an initialised workspace (>= 1 KB, 256-byte
 * aligned; its status word records out-of-range columns, which are
 * skipped). Asynchronous. */
int spgemm_csr_scatter_dense(const spgemm_plan* plan, const spgemm_csr* M, const float* vals,
                             float* X, int64_t ldx, void* ws, size_t ws_bytes, void* stream);

/* out[q] = D[i, j] for every entry q = (i, j) of M: a dense matrix read at
 * M's pattern (the gradient of A * TopK(X), dY * W^T, is needed only where
 * that product has entries). D: dense row-major M->rows x ldd (ldd >=
 * M->cols, device); out [M->nnz] (device). ws as for the scatter; an
 * out-of-range column gives 0 and records SPGEMM_ERR_INVALID. Asynchronous. */
int spgemm_csr_gather_dense(const spgemm_plan* plan, const spgemm_csr* M, const float* D,
                            int64_t ldd, float* out, void* ws, size_t ws_bytes, void* stream);

/* --- Matrix-based bulk neighbourhood sampling (Section IV-C, mini-batch
 * training): per layer P = Q^l * A (spgemm), NORM, Q^{l-1} = SAMPLE(P, s)
 * and EXTRACT(A, Q^l, Q^{l-1}) = (Q^l * A) * S with S the selector of
 * Q^{l-1}'s vertices. */

/* SAMPLE: for each row of P draw s entries (1 <= s <= 32) by inverse
 * transform sampling with the caller's uniforms u [P->rows * s] in [0, 1)
 * (row-major, device): mode 0 uniform over the row's entries (entry
 * floor(u * len)); mode 1 proportional to the values (negative values count
 * as 0); mode 2 proportional to the squared values; modes 1-2 use fp64
 * cumulative weights and take the first entry whose prefix exceeds
 * u * total (a row of zero weight samples uniformly). A row with at most s
 * entries keeps them all. Repeated draws collapse: Q's row holds the
 * distinct drawn columns in ascending order, each with value 1 (at most s).
 * Outputs (device): row_ptr_Q [P->rows+1], col_Q / val_Q [P->rows * s].
 * nnz_Q [host, nullable]: non-NULL synchronises. Workspace:
 * spgemm_workspace_bytes for a matrix of P->rows rows. Errors:
 * SPGEMM_ERR_UNSUPPORTED for s outside 1..32. */
int spgemm_sample_rows(const spgemm_plan* plan, const spgemm_csr* P, int32_t s, const float* u,
                       int32_t mode, void* ws, size_t ws_bytes, int32_t* row_ptr_Q,
                       int32_t* col_Q, float* val_Q, int64_t* nnz_Q, void* stream);

/* The distinct columns of Q (the vertices Q^{l-1} selected), as
 *   S (Q->cols x m): S[v, r] = 1 for the r-th selected vertex v (ascending),
 *     row_ptr S_row_ptr [Q->cols+1] (also the rank of every vertex);
 *   F (m x Q->cols): its transpose, one row per selected vertex (the next
 *     layer's Q), row_ptr F_row_ptr [m+1];
 * S_col/S_val/F_col/F_val hold at least min(Q->cols, Q->nnz) entries
 * (device). m [host, nullable]: non-NULL synchronises. Workspace:
 * spgemm_workspace_bytes for a matrix of Q->cols rows. */
int spgemm_select_columns(const spgemm_plan* plan, const spgemm_csr* Q, void* ws, size_t ws_bytes,
                          int32_t* S_row_ptr, int32_t* S_col, float* S_val, int32_t* F_row_ptr,
                          int32_t* F_col, float* F_val, int64_t* m, void* stream);

/* Synchronise `stream`, read and clear the workspace's device status word;
 * *status receives the SPGEMM_ERR_* code it maps to (SPGEMM_OK if clean). */
int spgemm_status(const spgemm_plan* plan, void* ws, void* stream, int* status);

/* Launch accounting and per-kernel timing (diagnostics; not thread-safe
 * while enabled). Every kernel launch the library makes is counted in
 * spgemm_launch_total. With profiling on, each launch is bracketed by a
 * pair of CUDA events on its stream (up to 8192 launches between reads);
 * spgemm_profile_read synchronises on them and returns, per kernel id, the
 * summed device milliseconds and the number of timed launches, then resets
 * the timing slots. spgemm_kernel_name maps an id to a short name. */
int spgemm_profile_enable(spgemm_plan* plan, int on);
int spgemm_profile_read(spgemm_plan* plan, double* ms, int64_t* launches, int n);
int spgemm_kernel_count(void);
const char* spgemm_kernel_name(int kid);
int64_t spgemm_launch_total(const spgemm_plan* plan);

/* Short text for a status code. */
const char* spgemm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_H */
