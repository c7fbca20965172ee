/*
 * spgemm.h -- C ABI of the GB300 sparse matrix-matrix product library.
 *
 * The library computes C = A.B for sparse A (m x l) and B (l x n) in CSR,
 * row by row (Gustavson's algorithm, Alg. 1 of Azad et al., "Exploiting
 * Multiple Levels of Parallelism in Sparse Matrix-Matrix Multiplication",
 * written column-wise there; here on rows, the same method on the transposed
 * problem), in two phases on the GPU: a symbolic phase that counts the
 * nonzeros of every row of C, and a numeric phase that fills columns and
 * values.  A second entry family sums the partial products of k-slices of the
 * inner dimension (the multiway merge with duplicate reduction of Sec. 4.3,
 * the LocalMerge step of Alg. 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All matrix arrays are DEVICE pointers owned by the caller.  The library
 *   never frees caller memory and never keeps a pointer after the call that
 *   consumes it returns, except inside a plan (see spgemm_plan), which keeps
 *   the A/B descriptors and the plan workspace until spgemm_plan_destroy.
 * - Row pointers are int64 (nnz(C) can exceed 2^31).  Column indices are
 *   int32 or int64 (spgemm_csr.index_type); C uses the index type of A.
 * - Rows must have strictly ascending column indices (no duplicates) and
 *   0-based indices; C is produced the same way (the paper keeps columns
 *   sorted, Sec. 5.2).  The pattern is structural: products that sum to zero
 *   stay in C (explicit zeros are nonzeros, Sec. 5).
 * - Values: F64, F32 and I64 use the (+, x) semiring by default (I64 wraps
 *   around); BOOL is the (or, and) semiring and carries no value array; the
 *   (min, +) and (min, select2nd) semirings run on F64 and I64 values (see
 *   spgemm_semiring).  Every output entry reduces its products in ascending
 *   k, each product rounded before it is added (no fused multiply-add), so
 *   results are reproducible bit for bit from run to run and equal across
 *   the single, batched, device-sized and learned paths.
 * - Work is enqueued on the caller's CUDA stream (a cudaStream_t passed as
 *   void*; NULL = legacy default stream).  The calls that report a size to
 *   the host (spgemm_plan, spgemm_symbolic, spgemm_merge_symbolic) wait for
 *   that stream; the others return without waiting.
 * - Errors: every call returns a spgemm_status; on error the outputs are
 *   unspecified and spgemm_last_error() gives a message (thread-local).  No
 *   exception crosses the ABI.
 */
#ifndef SPGEMM_GB300_H
#define SPGEMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPGEMM_OK = 0,
    SPGEMM_ERR_INVALID_ARG = 1,    /* null pointer, negative size, dimension mismatch */
    SPGEMM_ERR_INVALID_CSR = 2,    /* checked mode: rowptr not monotone, column out of
                                      range, unsorted or duplicate columns */
    SPGEMM_ERR_INDEX_OVERFLOW = 3, /* a column index or nnz does not fit the index type */
    SPGEMM_ERR_OUT_OF_MEMORY = 4,  /* a caller workspace is smaller than required */
    SPGEMM_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    SPGEMM_ERR_CUDA = 6,           /* a CUDA runtime call failed (message has the code) */
    SPGEMM_ERR_NOT_SUPPORTED = 7,  /* a combination this build does not implement */
    SPGEMM_ERR_INTERNAL = 8        /* a device-side consistency check failed */
} spgemm_status;

typedef enum { SPGEMM_F64 = 0, SPGEMM_F32 = 1, SPGEMM_I64 = 2, SPGEMM_BOOL = 3 } spgemm_value_type;
typedef enum { SPGEMM_INDEX_I32 = 0, SPGEMM_INDEX_I64 = 1 } spgemm_index_type;
/* Semirings (Sec. 2 states the product over a semiring):
 *   PLUS_TIMES     (+, x) on the value type;
 *   OR_AND         (or, and): the pattern only;
 *   MIN_PLUS       (min, +): C(i,j) = min over k of A(i,k) + B(k,j);
 *   MIN_SELECT2ND  (min, select2nd): C(i,j) = min over k of B(k,j)
 *                  (the operations MIS-2 aggregation is built from, Alg. 3).
 * The min semirings take float64 or int64 values (NOT_SUPPORTED otherwise);
 * a min starts at +infinity (INT64_MAX) and keeps the running value unless a
 * term is strictly smaller (a NaN term is never the minimum; the first of
 * equal terms in ascending k is kept); int64 sums wrap around. */
typedef enum {
    SPGEMM_PLUS_TIMES = 0,
    SPGEMM_OR_AND = 1,
    SPGEMM_MIN_PLUS = 2,
    SPGEMM_MIN_SELECT2ND = 3
} spgemm_semiring;

/* A CSR matrix in device memory.
 *   rowptr  int64[nrows+1]; row i spans [rowptr[i], rowptr[i+1]) ...
 *   rowend  ... or, when non-NULL, [rowptr[i], rowend[i]) (int64[nrows]); this
 *           lets a k-slice of A be a view on A's own arrays (Alg. 2 splits
 *           the inner dimension into contiguous ranges, Sec. 4.1).
 *   col     int32 or int64 [nnz] per index_type
 *   val     double / float / int64 [nnz] per value_type; NULL for BOOL
 *   nnz     length of the col/val arrays (the largest row end) */
typedef struct {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    const int64_t* rowptr;
    const int64_t* rowend;
    const void* col;
    const void* val;
    int32_t index_type; /* spgemm_index_type */
    int32_t value_type; /* spgemm_value_type */
} spgemm_csr;

typedef struct {
    int32_t semiring;        /* spgemm_semiring; OR_AND ignores values and yields a pattern */
    int32_t checked;         /* nonzero: validate A and B on the device before planning */
    int32_t dense_chunk;     /* columns per dense-row chunk: 0 = library choice, 1024 or 2048 */
    int32_t dense_min_flops; /* rows with more products use dense accumulators:
                                0 = 1024, else 32..1024 (autotuned knob) */
    int32_t max_row_nnz;     /* device-sized plans: bound on the entries of a dense row of A
                                (cursor arena slot), 0 = 65536 */
    int32_t hash_shift;      /* hash-table sizing (autotuned knob): a hash row with f products
                                goes to the smallest bin whose bound is >= f << hash_shift, so
                                its table has at least 2^(1+hash_shift) f slots; 0..2 */
    int32_t seg_log2;        /* dense work-unit size (autotuned knob): a dense row with about
                                2^t products is cut into 2^clamp(t+1-seg_log2, 0, 4) column
                                segments, one warp each; 0 = chosen per plan from
                                the flops and the resident warps (16 for device-sized
                                plans), else 10..22 */
    int32_t merge_staged;    /* merge numeric pass (c <= 4 lists in 16-byte aligned arrays):
                                nonzero stages every list's entries in shared memory with
                                bulk asynchronous copies (cp.async.bulk, mbarrier waits bounded,
                                SPGEMM_ERR_TIMEOUT from spgemm_merge_check if one expires);
                                0 keeps register windows (measured faster on GB300) */
} spgemm_opts;

typedef struct spgemm_plan_s* spgemm_plan_t;

/* Row statistics gathered by spgemm_plan (flops as defined in Sec. 2: the
 * number of scalar multiplications, sum over rows of sum_{k in A(i,:)}
 * nnz(B(k,:))). */
typedef struct {
    int64_t m, l, n;
    int64_t flops;          /* total multiplications */
    int64_t max_row_flops;
    int64_t rows_empty;     /* rows with no products */
    int64_t rows_hash;      /* rows handled with per-warp hash tables */
    int64_t rows_dense;     /* rows handled with column-chunked dense accumulators */
    int64_t chunk_width;    /* columns per dense chunk */
    int64_t chunks_per_row; /* dense chunks per dense row */
    int64_t nnz_c;          /* set by spgemm_symbolic, -1 before */
} spgemm_info;

/* Number of kernels this library has launched in this process (all
 * devices, all threads); a diagnostic counter, never reset. */
int64_t spgemm_kernel_launches(void);

/* Library version string. */
const char* spgemm_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char* spgemm_last_error(void);

/* Bytes of device workspace spgemm_plan needs for an m-row A (pure function;
 * O(m)). */
size_t spgemm_plan_workspace_size(int64_t m);

/* spgemm_plan -- validate A and B, count flops per row and bin the rows by
 * their flops (the per-row flops of Sec. 2 decide which accumulator a row
 * gets).  Enqueues the row analysis on `stream`, waits for it, and returns a
 * plan that owns host state only.  `plan_ws` (>= spgemm_plan_workspace_size
 * bytes, 256-byte aligned, device memory) must stay alive and untouched until
 * spgemm_plan_destroy.  A and B arrays must stay alive and unchanged for the
 * life of the plan.  Errors: INVALID_ARG, INVALID_CSR (checked mode),
 * INDEX_OVERFLOW, OUT_OF_MEMORY (plan_ws too small), NOT_SUPPORTED, CUDA. */
spgemm_status spgemm_plan(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                          void* stream, void* plan_ws, size_t plan_ws_bytes,
                          spgemm_plan_t* plan);

/* ---- batches of products (many independent C_p = A_p . B_p in one set of
 *      launches) ----
 * A batch plan numbers the rows of all products consecutively (product p owns
 * rows [sum_{q<p} m_q, sum_{q<=p} m_q)); spgemm_symbolic / spgemm_numeric then
 * produce the concatenation: rowptrC has (sum m_p)+1 entries, product p's
 * entries are colC/valC[rowptrC[row_base_p] .. rowptrC[row_base_p + m_p]).
 * All products share one index type and one value type.  Not in the paper;
 * the paper's local multiply is one product per process (Alg. 2). */
size_t spgemm_batch_plan_workspace_size(int32_t count, const spgemm_csr* A);
spgemm_status spgemm_batch_plan(int32_t count, const spgemm_csr* A, const spgemm_csr* B,
                                const spgemm_opts* opts, void* stream, void* plan_ws,
                                size_t plan_ws_bytes, spgemm_plan_t* plan);

/* Per-product row pointers of a batch result: out[row_base_p + p + i] =
 * rowptrC[row_base_p + i] - rowptrC[row_base_p] for i = 0..m_p (each product's
 * rowptr array, m_p + 1 entries, stored one after the other).  No wait. */
spgemm_status spgemm_batch_rowptrs(spgemm_plan_t plan, const int64_t* rowptrC, int64_t* out);

/* ---- device-sized plans: the whole product enqueued with no host readback,
 *      so a sequence of products (e.g. the levels of an AMG hierarchy) can be
 *      captured in a CUDA graph and replayed ----
 * spgemm_plan_device records the batch and sizes every workspace by upper
 * bounds (B's nnz fields are read as capacities; A rows longer than
 * opts.max_row_nnz that need the dense path are reported by spgemm_check).
 * It does no device work besides uploading the descriptors and waits for
 * that upload.  spgemm_execute then enqueues row analysis, symbolic phase,
 * scan and numeric phase; C goes to colC/valC (capacity entries); nnz(C) is
 * rowptrC[sum m_p] on the device.  If C exceeds the capacity nothing beyond it
 * is written and spgemm_check reports OUT_OF_MEMORY. */
spgemm_status spgemm_plan_device(int32_t count, const spgemm_csr* A, const spgemm_csr* B,
                                 const spgemm_opts* opts, void* stream, void* plan_ws,
                                 size_t plan_ws_bytes, spgemm_plan_t* plan);
spgemm_status spgemm_execute(spgemm_plan_t plan, void* ws, size_t ws_bytes, int64_t* rowptrC,
                             int64_t capacity, void* colC, void* valC);

/* ---- persistent chains (not in the paper: batching and dependent chains of
 * products in one launch; the paper's nearest point is that R^T A and
 * (R^T A) R carry too little work for large concurrency, Sec. 5.4) ----
 * A chain is an ordered list of device-sized products (spgemm_plan_device).
 * spgemm_chain_launch runs all of them, every phase of every product, in ONE
 * persistent kernel launch: a resident grid that waits at a device-side
 * barrier after each phase (analysis, binning, symbolic, two scan stages,
 * numeric), so a product may read the output of an earlier product of the
 * chain (its A or B arrays may be that product's rowptrC/colC/valC, with nnz
 * fields read as capacities, as for spgemm_plan_device).  Results are the same
 * bit for bit as spgemm_execute on each plan in turn.  Each step gives its
 * plan, the plan's workspace (spgemm_workspace_size), and its outputs as for
 * spgemm_execute.  All steps use one index type and one value type (float64,
 * float32, int64 or Boolean; NOT_SUPPORTED otherwise).
 * Every barrier wait is bounded by opts.timeout_s (0: 10 s): a wait that
 * expires sets the chain's status, every block of the grid returns, and
 * spgemm_chain_check reports SPGEMM_ERR_TIMEOUT (outputs undefined).
 * opts.withhold_stage >= 0 makes no block signal the end of that stage (a
 * test of the timeout path); -1 otherwise.  Per-product errors (capacity,
 * rows too wide) are read with spgemm_check on each plan. */
typedef struct {
    spgemm_plan_t plan;     /* from spgemm_plan_device */
    void* ws;               /* the plan's workspace */
    size_t ws_bytes;
    int64_t* rowptrC;       /* int64[R + 1] */
    int64_t capacity;       /* entries of colC / valC */
    void* colC;
    void* valC;             /* NULL for Boolean products */
} spgemm_chain_step;

typedef struct {
    double timeout_s;       /* bound of every barrier wait; 0 = 10 s */
    int32_t withhold_stage; /* -1, or a stage whose completion is withheld (tests) */
    /* threads of a persistent block: 0 or 768 (24 warps of up to 80
     * registers; the dense numeric stage needs them), or 1024 (32 warps of up
     * to 64 registers: more rows in flight for chains of short rows, such as
     * the levels of a Galerkin hierarchy); INVALID_ARG otherwise */
    int32_t block_threads;
    /* NULL, or a device array of 2 + 6 * nsteps uint64 that every launch
     * fills with %globaltimer readings (ns) of block 0: [0] at its start,
     * [1 + s] when it passed the barrier after stage s (stage 0 clears the
     * counters; product p's stages are 1 + 6p .. 6 + 6p: analysis, binning,
     * symbolic, scan sums, scan apply, numeric).  Caller-owned, kept until
     * the chain is destroyed; entries of stages not reached are left as
     * they were. */
    uint64_t* stage_ns;
} spgemm_chain_opts;

typedef struct spgemm_chain_s* spgemm_chain_t;

/* Device bytes of a chain's workspace (step table and barrier state). */
size_t spgemm_chain_workspace_size(int32_t nsteps);
/* Checks the steps and uploads the step table into chain_ws (caller-owned,
 * 256-byte aligned, kept until the chain is destroyed); waits for the upload.
 * The library keeps only the host handle. */
spgemm_status spgemm_chain_create(int32_t nsteps, const spgemm_chain_step* steps,
                                  const spgemm_chain_opts* opts, void* chain_ws,
                                  size_t chain_ws_bytes, spgemm_chain_t* chain);
/* Enqueues the whole chain on `stream`: one memset of the barrier state and
 * one kernel launch; no host readback, so it can be captured in a CUDA
 * graph.  Does not wait. */
spgemm_status spgemm_chain_launch(spgemm_chain_t chain, void* stream);
/* Waits for `stream` and reads the chain's status: OK or TIMEOUT. */
spgemm_status spgemm_chain_check(spgemm_chain_t chain, void* stream);
/* Blocks of the last launch's grid (0 before the first launch). */
int32_t spgemm_chain_grid(spgemm_chain_t chain);
void spgemm_chain_destroy(spgemm_chain_t chain);

/* ---- learned sizing of C (not in the paper: an addition to the method) ----
 * A small MLP predicts nnz(C(i,:)) from row features: x = log2(1 + .) of
 * flops_i, |A(i,:)|, max_k |B(k,:)|, n, flops_i / |A(i,:)|, min(flops_i, n);
 * layers F -> 32 -> 32 -> 1 with ReLU, float32.  Parameters are one device
 * float array of spgemm_sizer_param_count(F) entries: W1 (32 x F, row-major),
 * b1 (32), W2 (32 x 32, row-major), b2 (32), w3 (32), b3 (1).  The target the
 * network is trained on is log2(1 + nnz(C(i,:))) from the exact symbolic
 * phase. */
int32_t spgemm_sizer_param_count(int32_t features);
/* y[s] = MLP(X[s*F .. s*F+F)) for N samples (device arrays).  No wait. */
spgemm_status spgemm_sizer_forward(const float* X, int64_t N, int32_t F, const float* params,
                                   float* y, void* stream);
/* Gradient of 0.5 * mean_s (MLP(X_s) - T_s)^2 over all N samples into grad
 * (param_count floats) and the loss into *loss (device).  No wait. */
spgemm_status spgemm_sizer_grad(const float* X, const float* T, int64_t N, int32_t F,
                                const float* params, float* grad, float* loss, void* stream);
/* `steps` Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) on mini-batches of
 * `batch` consecutive entries of `order` (a permutation of 0..N-1, device
 * int64), updating params, adam_m, adam_v (zero-initialised by the caller);
 * grad is scratch (param_count floats); loss_trace[t] receives the batch loss
 * of step t (device).  No wait. */
spgemm_status spgemm_sizer_train(const float* X, const float* T, const int64_t* order, int64_t N,
                                 int32_t F, float* params, float* adam_m, float* adam_v,
                                 float* grad, int32_t steps, int32_t batch, float lr,
                                 float* loss_trace, void* stream);
/* Row features (F = 6, device float [rows x 6]) of a plan's rows, the
 * predictor's input, for building training sets.  No wait. */
spgemm_status spgemm_row_features(spgemm_plan_t plan, float* X);
/* Training targets T[i] = log2(1 + rowptrC[i+1] - rowptrC[i]) (device float
 * [m]) from the row pointers of the exact symbolic phase.  No wait. */
spgemm_status spgemm_sizer_targets(const int64_t* rowptrC, int64_t m, float* T, void* stream);
/* Trained predictor to a host byte record, so that it can be reused by
 * another process: magic "SGSIZER", format version 1, F, hidden width 32,
 * feature set 1 (the six features above, in that order), target 1
 * (log2(1 + nnz)), parameter count, the float32 parameters (device array,
 * copied on `stream`; the call waits for it), then a 64-bit FNV-1a hash of the
 * preceding bytes; little-endian.  *bytes_out = record size; with buf NULL
 * only the size is returned.  INVALID_ARG if buf_bytes is too small. */
spgemm_status spgemm_sizer_save(const float* params, int32_t F, void* stream, void* buf,
                                size_t buf_bytes, size_t* bytes_out);
/* Reads a record written by spgemm_sizer_save into params (device array of
 * spgemm_sizer_param_count(F) floats; waits for the copy).  INVALID_ARG for
 * a wrong magic, F, network shape, feature set, target, a truncated record or
 * a hash mismatch; NOT_SUPPORTED for another format version.  params is left
 * untouched on any error. */
spgemm_status spgemm_sizer_load(const void* buf, size_t buf_bytes, int32_t F, float* params,
                                void* stream);

/* Device allocation callback: returns `bytes` (>= 256-byte aligned) of
 * device memory owned by the caller, or NULL. */
typedef void* (*spgemm_alloc_fn)(size_t bytes, void* ctx);

typedef struct {
    int64_t nrows, ncols;
    int64_t nnz;           /* entries of col/val */
    int64_t* rowptr;       /* row i starts at rowptr[i] ... */
    int64_t* rowend;       /* ... and ends at rowend[i] (slots), or NULL: plain CSR */
    void* col;
    void* val;
    int64_t slot_total;    /* sum of the predicted slots */
    int64_t overflow_rows; /* rows that did not fit their slot (re-run exactly) */
    int64_t total_flops;
} spgemm_learned_result;

/* spgemm_learned_multiply -- C = A.B with the symbolic phase replaced by
 * the predictor (params, plus `margin` in log2 units of safety): every row is
 * multiplied straight into a predicted slot (a dense row's column segments
 * each fill a share of it in proportion to their chunks, then are packed
 * together); rows that overflow are listed and multiplied again by the exact
 * two-phase path.  Row contents equal spgemm_symbolic + spgemm_numeric bit
 * for bit.  C is returned as slots (row i spans [rowptr[i], rowend[i]); gaps
 * allowed; rowptr need not be monotone: re-run rows are placed in spare space
 * after the slots) unless the re-run rows do not fit that space, in which
 * case C is a plain compacted CSR (rowend NULL).  All device memory comes
 * from `alloc`; the call waits for the stream (it reads sizes back three to
 * five times).  Single product; A may be a view (rowend). */
spgemm_status spgemm_learned_multiply(const spgemm_csr* A, const spgemm_csr* B,
                                      const spgemm_opts* opts, const float* params, float margin,
                                      void* stream, spgemm_alloc_fn alloc, void* ctx,
                                      spgemm_learned_result* out);

/* Statistics of a plan (host call, no device work). */
spgemm_status spgemm_plan_info(spgemm_plan_t plan, spgemm_info* info);

/* Device workspace (bytes) that spgemm_symbolic / spgemm_numeric need for
 * this plan (dense-chunk counts and per-entry cursors).  Host call. */
spgemm_status spgemm_workspace_size(spgemm_plan_t plan, size_t* bytes);

/* spgemm_symbolic -- count the nonzeros of every row of C (the size of the
 * union of the column sets of the rows of B selected by A(i,:)), write the
 * row pointers rowptrC (int64[m+1], device) and nnz(C) to *nnz_c (host).
 * Waits for the stream.  `ws` is the workspace of spgemm_workspace_size; it
 * must be passed unchanged to spgemm_numeric. */
spgemm_status spgemm_symbolic(spgemm_plan_t plan, void* ws, size_t ws_bytes, int64_t* rowptrC,
                              int64_t* nnz_c);

/* spgemm_numeric -- fill colC (index type of A, [nnz_c]) and valC (value
 * type of A, [nnz_c]; NULL for OR_AND/BOOL) given the rowptrC of
 * spgemm_symbolic.  C(i,j) = sum over k ascending of A(i,k)*B(k,j) (Alg. 1).
 * Does not wait for the stream. */
spgemm_status spgemm_numeric(spgemm_plan_t plan, void* ws, size_t ws_bytes,
                             const int64_t* rowptrC, void* colC, void* valC);

/* Reads the plan's device error word (waits for the stream).  Returns
 * OUT_OF_MEMORY if C exceeded the capacity of spgemm_execute, NOT_SUPPORTED
 * if a dense row exceeded max_row_nnz, INTERNAL if another device-side check
 * failed since the plan was made. */
spgemm_status spgemm_check(spgemm_plan_t plan);

/* Release a plan (host memory only; the caller frees plan_ws). */
void spgemm_plan_destroy(spgemm_plan_t plan);

/* ---- transpose ----
 * spgemm_transpose -- A^T (n x m) in CSR with ascending columns: rowptrT
 * int64[n+1], colT (index type of A) and valT (value type of A; NULL for
 * BOOL) of nnz(A) entries, all device, caller-owned.  `ws` is device memory of
 * spgemm_transpose_workspace_size(A) bytes, 256-byte aligned.  Does not wait.
 * The paper transposes the B blocks locally while redistributing them
 * (Alg. 2, the all-to-all of B); here it provides R^T for R^T A R. */
size_t spgemm_transpose_workspace_size(const spgemm_csr* A);
spgemm_status spgemm_transpose(const spgemm_csr* A, void* stream, void* ws, size_t ws_bytes,
                               int64_t* rowptrT, void* colT, void* valT);

/* ---- Markov-clustering epilogue (MCL expansion = squaring, Sec. 5.3) ----
 * On M^T in CSR (float64; rowend views allowed): keep entries >= threshold,
 * divide each row by the sum of its kept entries (rows that lose every entry
 * stay empty).  Count pass writes rowptrP (int64[m+1]) and nnz to the host
 * (waits); fill pass writes colP (index type of C) / valP (float64).  `ws` is
 * spgemm_mcl_workspace_size(m) bytes, 256-byte aligned, kept between the two
 * calls. */
size_t spgemm_mcl_workspace_size(int64_t m);

/* ---- masked product (the structural mask MIS-2 applies to its semiring
 *      products, Alg. 3) ----
 * Keeps the entries (i, j) of C that are in the pattern of M (complement =
 * 0) or not in it (complement != 0).  C and M: same shape and index type,
 * rows sorted ascending; either may be a view (rowend).  The mask is applied
 * to the finished product (the product's own work is not reduced).  Count
 * pass: row pointers of the result into rowptrP (int64[m+1], device) and its
 * nnz to *nnz_host (waits); `ws` is spgemm_mask_workspace_size(m) bytes,
 * 256-byte aligned.  Fill pass: colP (index type of C), valP (value type of
 * C; NULL for BOOL); no wait.  Errors: INVALID_ARG, CUDA. */
size_t spgemm_mask_workspace_size(int64_t m);

/* ---- MIS-2 aggregation: the restriction operator of the paper's AMG
 *      experiments (Sec. 5.4, Alg. 3) ----
 * A: square CSR (the graph; its pattern only is read, diagonal allowed; rows
 * sorted; at most 2^31-1 vertices).  Computes a distance-2 maximal
 * independent set with Alg. 3's rounds of (min, select2nd) products: a
 * candidate joins when its key is the smallest within distance 2, where
 * key(seed, t, v) = ((splitmix64(seed ^ (t * 0xD1B54A32D192ED03) + v) >> 33)
 * << 31) | v in round t (SplitMix64 as published); the new members and every
 * candidate within distance 2 of them leave the candidates.  Aggregates:
 * members in increasing vertex order own themselves and their neighbours;
 * every other vertex joins the smallest-numbered aggregate among its
 * neighbours.  Writes R (n x naggs, one 1.0 per row): rowptrR int64[n+1],
 * colR (index type of A) [n], valR double[n]; *naggs_host, *rounds_host.
 * Waits for the stream once per round.  `ws` is
 * spgemm_mis2_workspace_size(n) bytes, 256-byte aligned.  Errors:
 * INVALID_ARG, NOT_SUPPORTED, INTERNAL (no progress / unaggregated vertex,
 * which the construction rules out), CUDA. */
size_t spgemm_mis2_workspace_size(int64_t n);

/* ---- doubly compressed rows (the row-wise form of DCSC, Sec. 3: only rows
 *      with entries are represented, with their ids) ----
 * spgemm_dcsr_view lists the nonempty rows of A (a CSR or a view, e.g. a
 * k-slice): rowids[t], rowptr_v[t], rowend_v[t] for t < *nzr_host (device
 * arrays of at least A->nrows entries; ids ascending).  {nrows = nzr, rowptr =
 * rowptr_v, rowend = rowend_v, col/val of A} is a view of those rows, and the
 * product of that view has the same column and value arrays as the product
 * of A; spgemm_dcsr_expand turns its row pointers (rowptr_c, nzr+1 entries)
 * back into the m+1 row pointers of the full product (rowptr_full).  `ws` is
 * spgemm_dcsr_workspace_size(m) bytes, 256-byte aligned.  The view call
 * waits for the stream (it reads nzr back); expand does not. */
size_t spgemm_dcsr_workspace_size(int64_t m);
spgemm_status spgemm_dcsr_view(const spgemm_csr* A, void* stream, void* ws, size_t ws_bytes,
                               int64_t* rowids, int64_t* rowptr_v, int64_t* rowend_v,
                               int64_t* nzr_host);
spgemm_status spgemm_dcsr_expand(int64_t m, int64_t nzr, const int64_t* rowids,
                                 const int64_t* rowptr_c, void* stream, int64_t* rowptr_full);
spgemm_status spgemm_mis2_restriction(const spgemm_csr* A, uint64_t seed, void* stream, void* ws,
                                      size_t ws_bytes, int64_t* rowptrR, void* colR,
                                      double* valR, int64_t* naggs_host, int32_t* rounds_host);
spgemm_status spgemm_mask_count(const spgemm_csr* C, const spgemm_csr* M, int32_t complement,
                                void* stream, void* ws, size_t ws_bytes, int64_t* rowptrP,
                                int64_t* nnz_host);
spgemm_status spgemm_mask_fill(const spgemm_csr* C, const spgemm_csr* M, int32_t complement,
                               void* stream, const int64_t* rowptrP, void* colP, void* valP);
spgemm_status spgemm_mcl_prune_count(const spgemm_csr* C, double threshold, void* stream,
                                     void* ws, size_t ws_bytes, int64_t* rowptrP,
                                     int64_t* nnz_host);
spgemm_status spgemm_mcl_prune_fill(const spgemm_csr* C, double threshold, void* stream, void* ws,
                                    size_t ws_bytes, const int64_t* rowptrP, void* colP,
                                    double* valP);

/* ---- k-slices and their merge (Alg. 2 split of the inner dimension;
 *      multiway merge with duplicate reduction, Sec. 4.3) ---- */

/* spgemm_kslice_bounds -- for A (m x l, CSR, no rowend), write the c+1
 * boundary arrays bounds[s*m + i] (int64, device, (c+1)*m entries) so that
 * slice s of row i is [bounds[s*m+i], bounds[(s+1)*m+i]): the entries of
 * A(i,:) with column in K_s = [floor(s*l/c), floor((s+1)*l/c)).  Slice s of A
 * is then the view {rowptr = bounds + s*m, rowend = bounds + (s+1)*m} on A's
 * arrays, and C_s = A_s . B.  Does not wait. */
spgemm_status spgemm_kslice_bounds(const spgemm_csr* A, int32_t c, void* stream,
                                   int64_t* bounds);

/* Workspace for the merge of c partials with m rows. */
size_t spgemm_merge_workspace_size(int32_t c, int64_t m, int64_t n);

/* spgemm_merge_symbolic -- parts[0..c-1]: c partial products of equal shape
 * (sorted rows).  Writes rowptrC (int64[m+1]) of C = sum_s parts[s] and
 * nnz(C) (host).  Waits for the stream.  Performance only: with c <= 4 and
 * int32 column arrays whose addresses are multiples of 16 bytes, the count
 * reads four columns per lane per load; each part's nnz must then be the
 * length of its col array (as stated for spgemm_csr). */
spgemm_status spgemm_merge_symbolic(int32_t c, const spgemm_csr* parts, const spgemm_opts* opts,
                                    void* stream, void* ws, size_t ws_bytes, int64_t* rowptrC,
                                    int64_t* nnz_c);

/* spgemm_merge_numeric -- fill colC/valC of C = sum_s parts[s]; equal
 * (i,j) entries are added in ascending s.  Does not wait. */
spgemm_status spgemm_merge_numeric(int32_t c, const spgemm_csr* parts, const spgemm_opts* opts,
                                   void* stream, void* ws, size_t ws_bytes,
                                   const int64_t* rowptrC, void* colC, void* valC);

/* spgemm_merge_symbolic_static -- the paper has no counterpart: this is an
 * interface variant.  Same result as spgemm_merge_symbolic (rowptrC of
 * C = sum_s parts[s] and nnz(C) on the host; waits for the stream) for callers
 * that may not allocate device memory and have no workspace to pass: code
 * that runs under a fixed device-memory budget reserved at start-up, or a
 * plug-in interface that hands over only inputs and outputs.  It allocates
 * nothing: its scratch (error word and scan partial sums, about 33 KB) is one
 * file-scope device array that every GPU loading the library keeps until the
 * process exits.
 * Limits: at most 2^24 rows (INVALID_ARG beyond).  All calls on a device
 * share the array, which keeps the last call's contents (the error word is
 * cleared at the start of each call); calls that overlap on the GPU race on
 * it.  Arguments are checked as by spgemm_merge_symbolic.  The first call on
 * a device looks up the array's device address (with that device current),
 * and a call after the device's context changed (a device reset) looks it up
 * again; make that first call before any stream capture. */
spgemm_status spgemm_merge_symbolic_static(int32_t c, const spgemm_csr* parts,
                                           const spgemm_opts* opts, void* stream,
                                           int64_t* rowptrC, int64_t* nnz_c);

/* Reads the device error word the merge calls record in `ws` (waits for the
 * stream); SPGEMM_ERR_INTERNAL if a row's emitted count disagreed with
 * rowptrC. */
spgemm_status spgemm_merge_check(void* stream, void* ws);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_GB300_H */
