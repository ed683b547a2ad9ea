/*
 * spmv.h -- C ABI of the GB300 cache-size-aware SpMV library.
 *
 * The library computes the repeated sparse matrix-vector product y <- A x of
 * Akbudak, Kayaaslan and Aykanat ("Analyzing and enhancing OSKI for sparse
 * matrix-vector multiplication") on sm_103a, in three forms of A:
 *
 *   - the K-way singly-bordered form A_SB = P_r A P_c (Sec. 3.1, eqs. 1-3),
 *   - the K-way doubly-bordered form A_DB (Sec. 3.2, eq. 5),
 *   - a nonzero-disjoint split A = A^1 + ... + A^K evaluated as the sequence
 *     y <- y + A^k x (Sec. 4),
 *
 * plus the plain natural-order CSR product (Sec. 2.1) as the baseline.  The
 * reorderings and splits come from the host-side recursive hypergraph
 * bisection of Sec. 3.1 (column-net model), Sec. 3.2 (enhanced
 * row-column-net model) and Sec. 4.1 (row-column-net model), or from the
 * caller.
 *
 * Conventions for every call:
 *   - Indices are int32 and 0-based.  Permutations map NEW -> OLD:
 *     row_perm[i'] is the original row placed at position i'.
 *   - spmv_exec works in the permuted space (x_hat = x P_c, y_hat = P_r y,
 *     Sec. 3): an iterative solver stays there; spmv_permute_x and
 *     spmv_unpermute_y move vectors in and out.
 *   - Host pointers are read during the call only; nothing is retained.
 *     Device pointers are plain CUDA device addresses on the current device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it; the call returns before the
 *     work completes unless stated otherwise.
 *   - No exception crosses the ABI.  Every call returns spmv_status; on
 *     failure spmv_last_error() gives a thread-local message naming the
 *     offending index.
 *   - A plan is not thread-safe: calls on one plan must not overlap (two
 *     spmv_exec of one plan on different streams race on its scratch).
 */
#ifndef SPMV_H
#define SPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spmv_status {
    SPMV_OK = 0,
    SPMV_E_INVALID = 1,      /* malformed argument (bad CSR, size, dtype, NULL) */
    SPMV_E_STRUCTURE = 2,    /* perm not a bijection, or a nonzero outside the
                                blocks and borders of the declared form */
    SPMV_E_NOMEM = 3,        /* device or host allocation failed */
    SPMV_E_CUDA = 4,         /* a CUDA runtime call or launch failed */
    SPMV_E_TIMEOUT = 5,      /* a bounded device wait gave up */
    SPMV_E_UNSUPPORTED = 6,  /* valid request outside what the library builds */
    SPMV_E_INTERNAL = 7      /* broken internal invariant (a bug) */
} spmv_status;

/* value / vector precisions (not in the paper, which uses FP64, Sec. 5.2):
 * F64: values, x, y and accumulation in FP64.
 * F32: values, x, y and accumulation in FP32.
 * BF16: values in BF16, x, y and accumulation in FP32.
 * Values are rounded to nearest-even from the FP64 master values. */
enum { SPMV_F64 = 0, SPMV_F32 = 1, SPMV_BF16 = 2 };

/* forms of A (Sec. 2.1, 3.1, 3.2, 4) */
enum { SPMV_NATURAL = 0, SPMV_SB = 1, SPMV_DB = 2, SPMV_SPLIT = 3 };

/* plan flags */
enum {
    SPMV_FLAG_NO_STAGING = 1,    /* never stage x in shared memory (ablation;
                                    overrides SPMV_FLAG_STAGE) */
    SPMV_FLAG_TILED_NATURAL = 2, /* natural form through the tiled kernel
                                    instead of the plain vector-per-row kernel */
    SPMV_FLAG_SM_AFFINE = 4,     /* persistent CTAs that first work the tiles
                                    queued for their own SM (a part's tiles on
                                    one SM, sharing its L1) (ablation) */
    SPMV_FLAG_PERSISTENT = 8,    /* persistent CTAs, one per resident slot,
                                    claiming tiles in order (ablation); the
                                    default is one CTA per tile, with tiles
                                    sized so that they fill about one wave of
                                    resident CTAs */
    SPMV_FLAG_STAGE = 16,        /* stage x in 256-thread CTAs too; by default
                                    only 512- and 1024-thread CTAs stage, whose
                                    windows are large enough to pay */
    SPMV_FLAG_TEST_WAIT_EXPIRES = 32, /* tests of failure detection only: the
                                    first wait of every staged tile on its
                                    staging copy gives up at once, so every
                                    staged tile is skipped and spmv_plan_check
                                    reports SPMV_E_TIMEOUT (the copy is still
                                    awaited, with the normal bound, before the
                                    CTA exits) */
    SPMV_FLAG_COL_DELTA = 64     /* tiled forms: the chunks of tiles that stage
                                    nothing store their column indices as
                                    16-bit increments along each row from a
                                    32-bit base column per chunk (the colDiff
                                    array of ICSR, Sec. 2.1, kept per lane: 2
                                    bytes per nonzero instead of 4).  A chunk
                                    with an increment above 65535 keeps 32-bit
                                    indices.  Rows too long for one lane (the
                                    warp rows and the chunk tiles) always do */
};

/* CSR matrix in host memory, caller-owned (Sec. 2.1: nonzero = vals,
 * colIndex = colidx, rowStart = rowptr).  rowptr has m+1 entries with
 * rowptr[0] = 0 and rowptr[m] = nnz < 2^31; column indices are sorted and
 * unique inside each row.  Values are the FP64 master copy. */
typedef struct spmv_csr {
    int32_t m, n;
    int64_t nnz;
    const int32_t *rowptr;
    const int32_t *colidx;
    const double *vals;
} spmv_csr;

/* Row and column permutations (new -> old).  NULL = identity. */
typedef struct spmv_perm {
    const int32_t *row_perm;   /* m entries */
    const int32_t *col_perm;   /* n entries */
} spmv_perm;

/* The form of P_r A P_c.
 *   SB / DB (eqs. 1, 5): row_part_ptr and col_part_ptr have K+2 entries.
 *     In the permuted space R_k = rows [row_part_ptr[k], row_part_ptr[k+1])
 *     for k < K and R_B = [row_part_ptr[K], row_part_ptr[K+1]) (empty for SB);
 *     C_k and C_B likewise from col_part_ptr.  Every nonzero of R_k must lie
 *     in C_k or C_B; R_B is unrestricted.
 *   SPLIT (Sec. 4): nz_part[p] in [0, K) is the part of the p-th nonzero of the
 *     ORIGINAL CSR.  row_part_ptr / col_part_ptr (K+2 entries, may be NULL)
 *     give each part's home rows / columns in the permuted space (as produced
 *     by spmv_form_from_labels: rows and columns grouped by first-touching
 *     part); they only guide the staging of x.
 *   NATURAL: the struct may be NULL. */
typedef struct spmv_splits {
    int32_t form;
    int32_t K;
    const int32_t *row_part_ptr;
    const int32_t *col_part_ptr;
    const int32_t *nz_part;
} spmv_splits;

/* Plan options.  Zero-initialise and set what you need. */
typedef struct spmv_opts {
    int32_t dtype;        /* SPMV_F64 / SPMV_F32 / SPMV_BF16 */
    int32_t nrhs;         /* right-hand sides r: X is n x r, Y is m x r, row
                             major; r in {1, 2, 4, 8} (0 = 1) */
    int32_t tile_cols;    /* max x entries staged per tile (0 = default) */
    int32_t tile_nnz;     /* target nonzeros per tile (0 = default) */
    int32_t long_row;     /* rows longer than this are reduced in chunks by
                             several CTAs (0 = default) */
    int32_t lanes;        /* threads cooperating on one row: 2, 4, 8, 16 or 32
                             (0 = chosen from the mean row length) */
    int32_t flags;        /* SPMV_FLAG_* */
    int32_t warp_rows;    /* tiled forms: rows longer than this are reduced
                             by a whole warp, shorter ones go into the chunks
                             of 32 rows (0 = 64) */
    int32_t cta_threads;  /* tiled forms: 256 = several CTAs per SM, tiles
                             for one wave of them, x through L1/L2 (0 = this);
                             512 = two CTAs per SM, tiles for two waves, each
                             staging up to 96 KB of x in shared memory;
                             1024 = one wide CTA per SM, tiles for four waves,
                             each staging up to 200 KB (for parts with large
                             column windows) */
    /* optional device allocator for plan-owned memory (NULL = cudaMalloc) */
    void *(*alloc)(size_t bytes, void *ctx);
    void (*release)(void *ptr, void *ctx);
    void *alloc_ctx;
} spmv_opts;

typedef struct spmv_plan spmv_plan;

/* What a plan holds and moves, for measurement and tests. */
typedef struct spmv_plan_info {
    int32_t m, n;
    int64_t nnz;
    int32_t form, K, dtype, nrhs;
    int32_t lanes;              /* threads per row in the row kernels */
    int32_t tile_cols;          /* staging capacity per tile (x entries) */
    int32_t n_tiles, n_staged_tiles, n_global_tiles, n_chunk_tiles;
    int32_t launches_per_exec;  /* kernel launches one spmv_exec makes */
    int32_t smem_bytes;         /* dynamic shared memory per CTA */
    int64_t staged_entries;     /* x entries staged per exec, summed over tiles */
    int64_t list_entries;       /* of which gathered through an index list */
    int64_t partial_slots;      /* partial sums written per exec (split rows
                                   shared by parts, chunks of long rows) */
    int64_t fixup_rows;         /* rows finished by the fix-up kernel */
    int64_t device_bytes;       /* plan-owned device memory */
    int64_t compulsory_bytes;   /* nnz*(value+4) + (m+1)*4 + n*r*xb + m*r*yb */
    int64_t moved_bytes;        /* bytes one exec reads/writes if every array
                                   element it touches is moved once */
    int32_t cta_threads;        /* tiled kernel CTA size (0: plain CSR kernel) */
    int64_t delta_nnz;          /* nonzeros stored as 16-bit column increments
                                   (SPMV_FLAG_COL_DELTA) */
} spmv_plan_info;

/* Build a plan: validate A, the permutation and the form (eqs. 1, 2, 5 or
 * Sec. 4), apply P_r A P_c, split per part, tile each part so its x working
 * set fits one CTA's shared memory, convert values to opts->dtype, and upload
 * everything to the current device.  Synchronous.  The plan owns its device
 * memory (through opts->alloc when given).
 * Errors: SPMV_E_INVALID (bad CSR or options), SPMV_E_STRUCTURE (bad perm,
 * nonzero outside C_k and C_B, bad part pointers), SPMV_E_NOMEM, SPMV_E_CUDA. */
spmv_status spmv_plan_create(const spmv_csr *A, const spmv_perm *perm,
                             const spmv_splits *splits, const spmv_opts *opts,
                             spmv_plan **out);

/* Batched plan (not in the paper): `count` independent matrices A[b], each
 * with its own perms[b] (NULL array or NULL members = identity) and, for the
 * split form, splits[b] (all with the same K; splits NULL = natural form),
 * in one plan whose spmv_exec is one launch over all of them.  The plan is
 * the block-diagonal matrix diag(A[0], ..., A[count-1]); x_hat is the
 * concatenation of the matrices' x_hat (n[b]*r entries each, in order) and
 * y_hat that of their y_hat.  For the split form, part k of the batch is the
 * union of the matrices' parts k: it is itself a nonzero-disjoint split
 * (Sec. 4) of the block-diagonal matrix.  SB / DB are not batched (each
 * matrix's border would have to share one border): SPMV_E_UNSUPPORTED.
 * Other errors as spmv_plan_create, with the matrix index in the message. */
spmv_status spmv_plan_create_batched(int32_t count, const spmv_csr *A, const spmv_perm *perms,
                                     const spmv_splits *splits, const spmv_opts *opts,
                                     spmv_plan **out);

/* y_hat <- A_hat x_hat (Sec. 3), or y_hat <- 0; y_hat <- y_hat + A^k x_hat for
 * k = 1..K (Sec. 4), on `stream`.  x_hat: n*r device elements, y_hat: m*r
 * device elements (double for F64, float for F32/BF16), row major, no
 * aliasing; x_hat 16-byte aligned (SPMV_E_INVALID otherwise: tiles copy
 * their x segments with bulk copies that need it, and with r > 1 the r
 * entries of a column are read as 16-byte words).  y_hat is overwritten.
 * Asynchronous. */
spmv_status spmv_exec(spmv_plan *plan, const void *x_hat, void *y_hat, void *stream);

/* Synchronise `stream` and report whether any earlier spmv_exec of the plan
 * hit a bounded device wait that gave up (the bulk copy of a tile's x
 * segment into shared memory not completing): SPMV_E_TIMEOUT, after which
 * the plan's results are not to be trusted and the plan should be destroyed;
 * SPMV_OK otherwise.  spmv_exec_host checks on its own. */
spmv_status spmv_plan_check(spmv_plan *plan, void *stream);

/* spmv_exec with HOST x_hat / y_hat: copies x_hat in, runs, copies y_hat out
 * and synchronises the stream before returning.  Device staging buffers are
 * allocated on the first call and kept by the plan.  Pinned host memory makes
 * the copies asynchronous DMA. */
spmv_status spmv_exec_host(spmv_plan *plan, const void *x_hat_host, void *y_hat_host,
                           void *stream);

/* x_hat[j'] = x[col_perm[j']] and y[row_perm[i']] = y_hat[i'] (Sec. 3), on
 * device memory, r values per entry.  Identity plans copy. */
spmv_status spmv_permute_x(const spmv_plan *plan, const void *x, void *x_hat, void *stream);
spmv_status spmv_unpermute_y(const spmv_plan *plan, const void *y_hat, void *y, void *stream);

spmv_status spmv_plan_get_info(const spmv_plan *plan, spmv_plan_info *info);

/* Release the plan and its device memory (synchronises the device first).
 * NULL is accepted. */
spmv_status spmv_plan_destroy(spmv_plan *plan);

/* Mixed-precision conjugate gradients with iterative refinement (not in the
 * paper, which computes in FP64, Sec. 5.2): solves A x = b for a symmetric
 * positive definite A from two plans of it built with the same permutations
 * and form -- `low` (any dtype) for the inner products and `f64` (SPMV_F64)
 * for the residual.  Each outer step computes r = b - A x in FP64 with the
 * f64 plan and stops once ||r||_2 <= tol ||b||_2; otherwise it runs plain CG
 * on A d = r / ||r|| with the low plan's products (FP32 vectors and
 * accumulation for F32 / BF16 values, FP64 for F64) until the inner residual
 * falls by inner_tol, and updates x <- x + ||r|| d in FP64.  The solver works
 * in the plans' column space (x_hat = x P_c), moving each product from row
 * to column space when the permutations differ.  Inner iterations run as a
 * CUDA graph of 8 captured iterations, replayed until the inner test holds.
 * b, x: n device doubles in the ORIGINAL order; x holds the initial guess on
 * entry and the solution on return.  Synchronous (work on an internal stream
 * ordered after `stream`); workspace comes from the low plan's allocator and
 * is released before returning.
 * Errors: SPMV_E_INVALID (plans of different shapes / permutations, f64 plan
 * not SPMV_F64, CG breakdown on a matrix that is not SPD), SPMV_E_UNSUPPORTED
 * (nrhs != 1), SPMV_E_NOMEM, SPMV_E_CUDA.  Not reaching tol within max_outer
 * steps is not an error: info->converged is 0. */
typedef struct spmv_cg_opts {
    double tol;           /* relative FP64 residual to reach (0 = 1e-10) */
    double inner_tol;     /* inner relative reduction (0 = 1e-4; 1e-12 for F64) */
    int32_t max_outer;    /* refinement steps (0 = 50) */
    int32_t max_inner;    /* inner iterations per step (0 = 2000) */
} spmv_cg_opts;

typedef struct spmv_cg_info {
    int32_t outer;        /* refinement steps taken */
    int32_t inner_total;  /* inner CG iterations, all steps */
    double rel_residual;  /* ||b - A x||_2 / ||b||_2 in FP64 at return */
    int32_t converged;    /* rel_residual <= tol */
} spmv_cg_info;

spmv_status spmv_cg_ir(spmv_plan *low, spmv_plan *f64, const double *b, double *x,
                       const spmv_cg_opts *opts, spmv_cg_info *info, void *stream);

/* ---- Learned form selector (not in the paper, which chooses its methods
 * by experiment, Sec. 5).  A multilayer perceptron maps SPMV_SEL_FEATURES
 * features of a matrix to scores of (form, K, tile shape) classes; it is
 * trained on the GPU by the kernels below from autotuner timings. */
enum { SPMV_SEL_FEATURES = 16 };

/* Features of a host CSR matrix (validated as for spmv_plan_create), into
 * out[SPMV_SEL_FEATURES]: log2 of m, n, nnz; row-degree mean, coefficient of
 * variation, log2 max, max/mean; column-degree coefficient of variation,
 * log2 max, max/mean; mean |j - i n/m| / n; share of nonzeros within n/64 of
 * the diagonal; share of touched columns used by more than one of 16
 * contiguous row blocks; share of empty rows; share of nonzeros in rows
 * longer than 64; log2 of the CSR bytes relative to 128 MB.  Host only. */
spmv_status spmv_features(const spmv_csr *A, float *out);

/* The network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3,
 * FP32, W row major [out][in]; `params` is ONE device array holding W1
 * (nh x nin), b1, W2 (nh x nh), b2, W3 (nc x nh), b3 back to back
 * (spmv_mlp_param_count(nin, nh, nc) floats).  Caller-owned. */
typedef struct spmv_mlp {
    int32_t nin, nh, nc;
    float *params;
} spmv_mlp;

int64_t spmv_mlp_param_count(int32_t nin, int32_t nh, int32_t nc);
/* Device workspace bytes spmv_mlp_forward / spmv_mlp_grad need for `batch`. */
size_t spmv_mlp_work_bytes(int32_t nh, int32_t nc, int32_t batch);

/* logits (batch x nc) = net(X), X batch x nin; device pointers; async. */
spmv_status spmv_mlp_forward(const spmv_mlp *net, const float *X, int32_t batch,
                             float *logits, void *work, void *stream);

/* Predicted class (largest score, the lower class on ties) and its softmax
 * probability for each of `batch` feature rows: cls[batch] (int32) and
 * conf[batch] (float), device arrays; work as spmv_mlp_forward.  Async. */
spmv_status spmv_mlp_predict(const spmv_mlp *net, const float *X, int32_t batch,
                             int32_t *cls, float *conf, void *work, void *stream);

/* Fold a feature standardisation x' = (x - mu) / sd into the first layer, so
 * that the network reads unscaled features: W1[o][i] /= sd[i], then
 * b1[o] -= sum_i W1[o][i] mu[i].  mu, sd: nin device floats.  Async. */
spmv_status spmv_mlp_fold_scaling(const spmv_mlp *net, const float *mu, const float *sd,
                                  void *stream);

/* Mean softmax cross-entropy over the batch of labels[b] in [0, nc) (a
 * label outside that range makes *loss NaN and contributes no gradient):
 * *loss (one device float) and its gradient with
 * respect to every parameter into grads (same layout as params).  Fixed-order
 * sums: deterministic.  Async. */
spmv_status spmv_mlp_grad(const spmv_mlp *net, const float *X, const int32_t *labels,
                          int32_t batch, float *grads, float *loss, void *work, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected for step
 * `step` >= 1) on the parameters with moment buffers m, v (device, zeroed
 * before step 1).  Async. */
spmv_status spmv_mlp_adam(const spmv_mlp *net, const float *grads, float *m, float *v,
                          int32_t step, float lr, void *stream);

/* Autotuner (not in the paper; the shapes the paper leaves to OSKI are picked
 * by measurement here): build one plan per candidate option set for the same
 * A / perm / splits (all of them live at once), make one warm call of each,
 * then `reps` rounds of one timed call per candidate in turn on `stream`
 * (zero input vectors, allocated from the first candidate's allocator and
 * released before returning), keep the candidate with the smallest median
 * call and destroy the others.  *best receives the index of the kept
 * candidate, *best_ms its median time per call.  Synchronous.  Errors as
 * spmv_plan_create, plus SPMV_E_CUDA. */
spmv_status spmv_plan_autotune(const spmv_csr *A, const spmv_perm *perm,
                               const spmv_splits *splits, const spmv_opts *candidates,
                               int32_t n_candidates, int32_t reps, void *stream,
                               spmv_plan **out, int32_t *best, float *best_ms);

/* Derive a form from labels, on the host.
 *   SPMV_SB: labels[m] in [0, K): rows ordered by (label, index); C_k = the
 *     columns whose only part is k (lambda = 1, eq. 3), ordered by index;
 *     C_B = columns with lambda >= 2 by index, then untouched columns.
 *   SPMV_DB: labels[m] in [0, K]; label K puts the row in R_B (eq. 5);
 *     lambda' counts non-border rows only.
 *   SPMV_SPLIT: labels[nnz] in [0, K) per nonzero of the original CSR; rows
 *     and columns ordered by the first part (smallest k) touching them,
 *     untouched ones last, ties by index.
 * Outputs (caller-allocated): row_perm[m], col_perm[n], row_part_ptr[K+2],
 * col_part_ptr[K+2] in the layout of spmv_splits. */
spmv_status spmv_form_from_labels(const spmv_csr *A, int32_t form, int32_t K,
                                  const int32_t *labels, int32_t *row_perm,
                                  int32_t *col_perm, int32_t *row_part_ptr,
                                  int32_t *col_part_ptr);

/* Hypergraph models for spmv_partition */
enum {
    SPMV_PART_CN = 0,     /* column-net model, connectivity metric -> SB
                             (sHP_CN, Sec. 3.1) */
    SPMV_PART_ERCN = 1,   /* enhanced row-column-net model: column nets cost 1
                             with the connectivity metric (cut-net splitting),
                             row nets cost nnz(r_i) with the cut-net metric
                             (cut-net removal) -> DB (sHP_eRCN, Sec. 3.2) */
    SPMV_PART_RCN = 2,    /* row-column-net model, connectivity metric on
                             both net types -> split (mHP_RCN, Sec. 4.1) */
    SPMV_PART_RANDOM = 3, /* uniform random row labels -> SB (a baseline) */
    SPMV_PART_RN = 4      /* row-net model (sHP_RN, Sec. 5.1, a baseline):
                             columns are vertices, rows are nets (the
                             column-net model of A^T); labels[n] are column
                             parts, the form is SPMV_NATURAL with the nested
                             separated block-diagonal order of spmv_reorder
                             (SPMV_ORDER_SBD); cost = cost_rows = the sum
                             over rows of their connectivity */
};

/* Stop rule of the recursive bisection (Sec. 5.1) */
enum {
    SPMV_FIT_CSR = 0,     /* part's CSR storage + x + y subvectors < part_bytes
                             (FP64 values, int32 indices; the paper's rule) */
    SPMV_FIT_X = 1        /* part's x subvector (8 bytes per column it touches;
                             plus its y subvector for RCN) < part_bytes: the
                             shared-memory adaptation */
};

typedef struct spmv_partition_opts {
    int32_t method;       /* SPMV_PART_* */
    int32_t K;            /* > 0: bisect to depth log2(K) (K a power of two) */
    int64_t part_bytes;   /* K == 0: bisect until every part fits */
    int32_t fit_rule;     /* SPMV_FIT_* */
    int32_t threads;      /* host threads (0 = hardware concurrency) */
    double imbalance;     /* allowed imbalance per bisection (0 = 0.10) */
    uint64_t seed;
} spmv_partition_opts;

/* Output of spmv_partition; arrays are allocated by the library and released
 * by spmv_partition_free. */
typedef struct spmv_partition_out {
    int32_t form;         /* SPMV_SB, SPMV_DB or SPMV_SPLIT */
    int32_t K;            /* number of parts */
    int32_t n_labels;     /* m (SB, DB) or nnz (SPLIT) */
    int32_t *labels;      /* row labels (DB: K = row border) or nonzero labels */
    int32_t *row_perm, *col_perm, *row_part_ptr, *col_part_ptr;
    int64_t cost;         /* the partitioner's own accounting of the bound:
                             eq. 4 for CN, eq. 6 for eRCN, eq. 7 for RCN */
    int64_t cost_cols;    /* column share of cost (lambda sums over columns) */
    int64_t cost_rows;    /* row share (RCN: sum lambda(r_i); eRCN: nnz(R_B)) */
    double seconds;       /* wall time */
} spmv_partition_out;

/* Recursive hypergraph bisection of A under a model (Sec. 3.1, 3.2, 4.1,
 * 5.1), host-only.  Deterministic for a given seed and thread count.
 * Returns labels and the derived form (as spmv_form_from_labels).
 * Errors: SPMV_E_INVALID (bad CSR, K not a power of two, no stop rule),
 * SPMV_E_NOMEM. */
spmv_status spmv_partition(const spmv_csr *A, const spmv_partition_opts *opts,
                           spmv_partition_out *out);
void spmv_partition_free(spmv_partition_out *out);

/* Row and column orders of the paper's comparison methods (Sec. 5.1) and
 * the nested border order of the SB / DB forms, host only, into
 * caller-allocated row_perm[m] and col_perm[n] (new -> old), for a plan of
 * form SPMV_NATURAL (through the tiled kernel: SPMV_FLAG_TILED_NATURAL).  The bipartite graph of A has a vertex per
 * row and per column and an edge per nonzero; ties go to the lower vertex
 * (rows before columns, then by index).
 *   SPMV_ORDER_BFS (sBFS): breadth-first search from row 0, neighbours in
 *     increasing order; when the queue runs dry, from the lowest unvisited
 *     vertex.  Rows and columns in visiting order.
 *   SPMV_ORDER_RCM (sRCM): reverse Cuthill-McKee: per connected component
 *     (in order of its lowest vertex), a pseudo-peripheral start by the
 *     George-Liu procedure from the component's vertex of least degree,
 *     unvisited neighbours enqueued by increasing degree; the whole visiting
 *     sequence reversed.
 *   SPMV_ORDER_SBD (the order of sHP_RN): col_labels[n] in [0, K), K a power
 *     of two, are the leaves of a recursive bisection of the columns (left
 *     subtree first); columns by (label, index); a row whose columns all lie
 *     in leaf k goes to block k, a row whose labels span a..b (a < b) to the
 *     separator of the bisection that split a from b, placed between that
 *     bisection's two halves; empty rows last; ties by index.  labels are
 *     the n column labels.
 *   SPMV_ORDER_NESTED (the SB / DB forms with a nested border, Sec. 3.1 and
 *     3.2): labels[m] in [0, K], K a power of two, are the row parts of an SB
 *     (CN) or DB (eRCN, label K = the row border R_B) partition, the leaves
 *     of its recursive bisection (left subtree first).  Rows by (label,
 *     index), R_B last.  A column whose rows outside R_B all lie in part k
 *     goes to C_k; a coupling column whose rows span parts a..b (a < b) goes
 *     to the border of the bisection that split a from b, placed between
 *     that bisection's two halves (the cut columns of a bisection sit
 *     between the column slices of its halves instead of in one C_B at the
 *     end); columns no part touches last; ties by index.
 * Errors: SPMV_E_INVALID (bad CSR, K, labels or method). */
enum { SPMV_ORDER_BFS = 0, SPMV_ORDER_RCM = 1, SPMV_ORDER_SBD = 2, SPMV_ORDER_NESTED = 3 };
spmv_status spmv_reorder(const spmv_csr *A, int32_t method, int32_t K, const int32_t *labels,
                         int32_t *row_perm, int32_t *col_perm);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *spmv_last_error(void);

/* y = A x for a CSR matrix that is already in device memory, allocating
 * nothing.  The paper has no counterpart: this entry point serves callers that
 * cannot allocate device memory when they need the product (code running
 * inside a memory pool it does not own, a plugin given only its buffers, a
 * step that must leave the allocator untouched).  It needs no plan.
 *
 * rowptr_dev[m+1], colidx_dev[nnz] (int32), vals_dev[nnz], x_dev[n] and
 * y_dev[m] (double) are caller-owned device arrays on the current device; the
 * CSR has the layout of spmv_csr (sorted columns not required).  y is
 * overwritten.  Rows are reduced in chunks of 4096 nonzeros; the partial sums
 * of rows that cross a chunk boundary go to a fixed scratch array compiled
 * into the library (2 * SPMV_NOALLOC_MAX_NNZ / 4096 doubles = 4 MiB, held on
 * every device that loads the library until the process exits).
 *   - nnz > SPMV_NOALLOC_MAX_NNZ is rejected with SPMV_E_UNSUPPORTED.
 *   - The first call on a device sets the entry point up with that device
 *     current: it looks up the scratch array's device address
 *     (cudaGetSymbolAddress) and loads this entry point's kernels.  CUDA
 *     loads modules lazily by default, so this first call is the one that
 *     places the scratch array and the kernels' code in device memory, and
 *     it can fail with SPMV_E_CUDA when the device is out of memory.  Make it
 *     at set-up time, before the code that cannot allocate and before any
 *     stream capture: a call with m = 0 (every pointer may then be NULL)
 *     does the set-up and nothing else.  Later calls on that device allocate
 *     nothing.
 *   - Every call shares the one scratch array and overwrites what it uses:
 *     calls whose kernels overlap on the GPU (different streams, threads)
 *     race and must be serialised by the caller.
 * Asynchronous on `stream`.  Errors: SPMV_E_INVALID (negative size, NULL),
 * SPMV_E_UNSUPPORTED, SPMV_E_CUDA. */
#define SPMV_NOALLOC_MAX_NNZ 1073741824LL
spmv_status spmv_csr_exec_noalloc(int32_t m, int32_t n, int64_t nnz,
                                  const int32_t *rowptr_dev, const int32_t *colidx_dev,
                                  const double *vals_dev, const double *x_dev,
                                  double *y_dev, void *stream);

/* Diagnostics: build the host image of the plan spmv_plan_create would build
 * for A, perm, splits and opts on a device with n_sm SMs (0 = 152, GB300),
 * and evaluate the product by walking that image the way the kernels do
 * (Sec. 3: y_hat = A_hat x_hat; Sec. 4: the sum over k of A^k x_hat, through
 * the partial slots and the fix-ups), on the host in FP64.  No device call.
 * x (n x r) and y (m x r, overwritten) are host arrays in the ORIGINAL
 * order, row major, r = opts->nrhs; values are used in FP64 whatever
 * opts->dtype says (the image's layout is the one of that dtype).  Every
 * index of the image is checked against its array, and every row of y and
 * every partial slot must be written exactly once: a violation returns
 * SPMV_E_INTERNAL with the offending indices in spmv_last_error().
 * stats (may be NULL) receives SPMV_EMULATE_STATS counts: tiles, chunk
 * tiles, staged tiles, partial slots, fix-ups, warp rows, stored chunk
 * elements (with padding), 1 if the plain CSR kernel is used, nonzeros whose
 * x is gathered (not staged), FMA lanes the tiles issue, element slots that
 * load x from both global and shared memory, x entries staged, tiles that
 * stage a second run, nonzeros stored as 16-bit column increments
 * (SPMV_FLAG_COL_DELTA).  Errors: those of spmv_plan_create's validation,
 * SPMV_E_INTERNAL, SPMV_E_NOMEM. */
#define SPMV_EMULATE_STATS 14
spmv_status spmv_plan_emulate(const spmv_csr *A, const spmv_perm *perm,
                              const spmv_splits *splits, const spmv_opts *opts,
                              int32_t n_sm, const double *x, double *y, int64_t *stats);

#ifdef __cplusplus
}
#endif

#endif /* SPMV_H */
