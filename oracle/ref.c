/*
 * CPU oracle for cache-size-aware SpMxV (Akbudak, Kayaaslan, Aykanat,
 * "Analyzing and enhancing OSKI for sparse matrix-vector multiplication").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded, FP64.  Nothing in the
 * product library links, includes or calls this file; it shares no code,
 * header, table or helper with the CUDA path.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark load it.
 *
 * Every function cites the passage of the paper it restates:
 *   ref_spmv            y = A x by the CSR definition (Sec. 2.1, Sec. 1),
 *                       compensated (Neumaier) FP64 sums, plus (|A||x|)_i.
 *   ref_spmv_plain      the same product as the paper's plain CSR loop
 *                       (Sec. 2.1: one FP64 running sum per row), the timed
 *                       CPU baseline; with OpenMP (when the build has it) the
 *                       rows are shared among host threads.
 *   ref_permute_csr     A_hat = P_r A P_c (Sec. 3, first paragraph).
 *   ref_form_rows       SB form (eqs. 1-3) / DB form (eq. 5) from row labels;
 *                       coupling columns grouped by the part holding most of
 *                       their nonzeros (Sec. 3, similar patterns nearby).
 *   ref_form_split      row/column order of a split (Sec. 4) by first-touching part.
 *   ref_split_parts     the A^k matrices of a split in GCSR (Sec. 4, Sec. 5.2).
 *   ref_lambda_rows     lambda(c_j) over row parts (eq. 3; lambda' for DB).
 *   ref_lambda_split    lambda(r_i), lambda(c_j) over a split (Sec. 4.1).
 *   ref_check_structure every nonzero of R_k lies in C_k or C_B (eqs. 1, 2, 5).
 *   ref_is_perm         bijection check.
 *   ref_cachesim_*      fully associative LRU cache replaying the CSR SpMxV
 *                       access order (Sec. 2.2, Sec. 3 fully-associative
 *                       assumption), counting misses per array.
 *   ref_cg              conjugate gradients in FP64 (iterative solvers, Sec. 1).
 *   ref_mlp_loss_grad   the selector extension's multilayer perceptron (not in
 *                       the paper): forward pass, softmax cross-entropy, and
 *                       the gradients by the chain rule, in FP64.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- SpMV --- */

/* y_i = sum_p val[p] * x[col[p]] for each right-hand side c (X is n x r, row
 * major).  Neumaier's compensated summation keeps the oracle's own error far
 * below the FP64 tolerance of the path under test.  absax_i = sum |val||x|. */
void ref_spmv(int32_t m, const int64_t *rowptr, const int32_t *col,
              const double *val, const double *x, int32_t r, double *y,
              double *absax)
{
    for (int32_t i = 0; i < m; ++i) {
        for (int32_t c = 0; c < r; ++c) {
            double s = 0.0, comp = 0.0, a = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                double t = val[p] * x[(int64_t)col[p] * r + c];
                double u = s + t;
                if (fabs(s) >= fabs(t))
                    comp += (s - u) + t;
                else
                    comp += (t - u) + s;
                s = u;
                a += fabs(t);
            }
            y[(int64_t)i * r + c] = s + comp;
            if (absax) absax[(int64_t)i * r + c] = a;
        }
    }
}

/* ------------------------------------------------------- permutations --- */

/* The plain CSR SpMxV of Sec. 2.1: for each row, one FP64 running sum over
 * its nonzeros in storage order, written to y.  No compensation: this is the
 * loop whose speed the CPU baseline reports, not a checker.  threads > 1
 * shares the rows among that many OpenMP threads (static schedule) when the
 * oracle was built with OpenMP; the sums are the same either way. */
void ref_spmv_plain(int32_t m, const int64_t *rowptr, const int32_t *col,
                    const double *val, const double *x, double *y, int32_t threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (int32_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[col[p]];
        y[i] = s;
    }
    (void)threads;
}

/* Host threads ref_spmv_plain can use: OpenMP's maximum, 1 without OpenMP. */
int32_t ref_plain_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

int32_t ref_is_perm(int32_t n, const int32_t *perm)
{
    char *seen = (char *)calloc((size_t)n + 1, 1);
    int32_t ok = 1;
    for (int32_t i = 0; i < n && ok; ++i) {
        if (perm[i] < 0 || perm[i] >= n || seen[perm[i]]) ok = 0;
        else seen[perm[i]] = 1;
    }
    free(seen);
    return ok;
}

static int cmp_int(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int cmp_pair(const void *a, const void *b)
{
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

/* A_hat = P_r A P_c with perms mapping new -> old: row i' of A_hat is row
 * row_perm[i'] of A, and column j of A becomes column colinv[j].  Columns are
 * re-sorted inside each row.  Output arrays are caller-allocated. */
void ref_permute_csr(int32_t m, int32_t n, const int64_t *rowptr,
                     const int32_t *col, const double *val,
                     const int32_t *row_perm, const int32_t *col_perm,
                     int64_t *out_rowptr, int32_t *out_col, double *out_val)
{
    int32_t *colinv = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t j = 0; j < n; ++j) colinv[col_perm[j]] = j;
    out_rowptr[0] = 0;
    for (int32_t i = 0; i < m; ++i) {
        int32_t old = row_perm[i];
        out_rowptr[i + 1] = out_rowptr[i] + (rowptr[old + 1] - rowptr[old]);
    }
    int32_t *buf = NULL;
    size_t cap = 0;
    for (int32_t i = 0; i < m; ++i) {
        int32_t old = row_perm[i];
        int64_t len = rowptr[old + 1] - rowptr[old];
        if ((size_t)len > cap) {
            cap = (size_t)len;
            buf = (int32_t *)realloc(buf, sizeof(int32_t) * 2 * cap);
        }
        for (int64_t t = 0; t < len; ++t) {
            buf[2 * t] = colinv[col[rowptr[old] + t]];
            buf[2 * t + 1] = (int32_t)t;
        }
        qsort(buf, (size_t)len, 2 * sizeof(int32_t), cmp_pair);
        for (int64_t t = 0; t < len; ++t) {
            out_col[out_rowptr[i] + t] = buf[2 * t];
            out_val[out_rowptr[i] + t] = val[rowptr[old] + buf[2 * t + 1]];
        }
    }
    free(buf);
    free(colinv);
}

/* ---------------------------------------------------- connectivities --- */

/* lambda(c_j) = number of distinct row parts R_k (label in [0, K)) that hold a
 * nonzero of column j (eq. 3).  Rows with label outside [0, K) -- the row
 * border R_B of the DB form -- are ignored, which gives lambda'(c_j) of
 * eq. 5.  single[j] receives the only part when lambda = 1, else -1. */
void ref_lambda_rows(int32_t m, int32_t n, const int64_t *rowptr,
                     const int32_t *col, int32_t K, const int32_t *labels,
                     int32_t *lambda, int32_t *single)
{
    /* gather the labels of each column's rows (a transpose), then count the
     * distinct ones per column */
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t i = 0; i < m; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) cnt[col[p] + 1]++;
    for (int32_t j = 0; j < n; ++j) cnt[j + 1] += cnt[j];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    memcpy(pos, cnt, sizeof(int64_t) * ((size_t)n + 1));
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt[n] + 1));
    for (int32_t i = 0; i < m; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            lab[pos[col[p]]++] = labels[i];
    for (int32_t j = 0; j < n; ++j) {
        /* sort the column's row labels, then count distinct labels in [0,K) */
        int64_t len = cnt[j + 1] - cnt[j];
        qsort(lab + cnt[j], (size_t)len, sizeof(int32_t), cmp_int);
        int32_t l = 0, s = -1;
        for (int64_t a = cnt[j]; a < cnt[j + 1]; ++a) {
            int32_t la = lab[a];
            if (la < 0 || la >= K) continue;
            if (a > cnt[j] && lab[a - 1] == la) continue;
            ++l;
            s = la;
        }
        lambda[j] = l;
        single[j] = (l == 1) ? s : -1;
    }
    free(lab);
    free(pos);
    free(cnt);
}

/* lambda(r_i) and lambda(c_j) over a split Pi = {A^1..A^K} given the part of
 * every nonzero (Sec. 4.1). */
void ref_lambda_split(int32_t m, int32_t n, const int64_t *rowptr,
                      const int32_t *col, int32_t K, const int32_t *nz_part,
                      int32_t *lambda_r, int32_t *lambda_c)
{
    char *hit = (char *)calloc((size_t)K * ((size_t)n > (size_t)m ? (size_t)n : (size_t)m) + 1, 1);
    /* rows */
    for (int32_t i = 0; i < m; ++i) {
        int32_t l = 0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            size_t key = (size_t)i * K + nz_part[p];
            if (!hit[key]) { hit[key] = 1; ++l; }
        }
        lambda_r[i] = l;
    }
    memset(hit, 0, (size_t)K * ((size_t)n > (size_t)m ? (size_t)n : (size_t)m) + 1);
    for (int32_t j = 0; j < n; ++j) lambda_c[j] = 0;
    for (int32_t i = 0; i < m; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            size_t key = (size_t)col[p] * K + nz_part[p];
            if (!hit[key]) { hit[key] = 1; lambda_c[col[p]]++; }
        }
    free(hit);
}

/* ------------------------------------------------------- form rules --- */

/* SB form of eq. (1) (border = 0) or DB form of eq. (5) (border = 1) from row
 * labels ell(i) in [0, K), and label K for the row border R_B (DB only).
 *   rows:    ordered by (ell(i), i); R_B rows last, by i.
 *   columns: C_k = columns with lambda = 1 in part k, ordered by (k, j);
 *            C_B = columns with lambda >= 2 ordered by j, then columns with
 *            lambda = 0 (untouched, or touched only by R_B rows) ordered by j.
 * lambda is counted over the non-border rows (lambda' of eq. 5 for DB).
 * Perms map new -> old.  row_part_ptr/col_part_ptr have K+2 entries:
 * R_k = [p[k], p[k+1]), R_B = [p[K], p[K+1]); likewise C_k and C_B.
 * Returns 0, or -1 on a label outside the allowed range. */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* For each column, the part (label < K) holding most of its nonzeros, the
 * lower part on ties; K for a column no non-border row touches.  The order
 * of the coupling columns inside the border is not fixed by eqs. (1)-(2) or
 * (5); Sec. 3 asks that columns with similar sparsity patterns be placed near
 * each other, so the border groups its columns by this part.  Plain: the
 * labels of each column's rows are collected, sorted and counted. */
int32_t *ref_majority_part(int32_t m, int32_t n, const int64_t *rowptr,
                           const int32_t *col, int32_t K, const int32_t *labels)
{
    int64_t *cstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t i = 0; i < m; ++i)
        if (labels[i] < K)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) cstart[col[p] + 1]++;
    for (int32_t j = 0; j < n; ++j) cstart[j + 1] += cstart[j];
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cstart[n] + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    for (int32_t j = 0; j < n; ++j) fill[j] = cstart[j];
    for (int32_t i = 0; i < m; ++i)
        if (labels[i] < K)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) lab[fill[col[p]]++] = labels[i];
    int32_t *maj = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t j = 0; j < n; ++j) {
        int64_t a = cstart[j], b = cstart[j + 1];
        qsort(lab + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
        int32_t best = K;
        int64_t best_cnt = 0;
        for (int64_t p = a; p < b;) {
            int64_t q = p;
            while (q < b && lab[q] == lab[p]) ++q;
            if (q - p > best_cnt) {     /* strictly more: ties keep the lower part */
                best_cnt = q - p;
                best = lab[p];
            }
            p = q;
        }
        maj[j] = best;
    }
    free(cstart);
    free(lab);
    free(fill);
    return maj;
}

int32_t ref_form_rows(int32_t m, int32_t n, const int64_t *rowptr,
                      const int32_t *col, int32_t K, const int32_t *labels,
                      int32_t border, int32_t *row_perm, int32_t *col_perm,
                      int32_t *row_part_ptr, int32_t *col_part_ptr)
{
    int32_t maxlab = border ? K : K - 1;
    for (int32_t i = 0; i < m; ++i)
        if (labels[i] < 0 || labels[i] > maxlab) return -1;
    /* rows: stable counting sort by label */
    int32_t t = 0;
    for (int32_t k = 0; k <= K; ++k) {
        row_part_ptr[k] = t;
        for (int32_t i = 0; i < m; ++i)
            if (labels[i] == k) row_perm[t++] = i;
    }
    row_part_ptr[K + 1] = m;
    /* columns */
    int32_t *lam = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *one = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    ref_lambda_rows(m, n, rowptr, col, K, labels, lam, one);
    t = 0;
    for (int32_t k = 0; k < K; ++k) {
        col_part_ptr[k] = t;
        for (int32_t j = 0; j < n; ++j)
            if (lam[j] == 1 && one[j] == k) col_perm[t++] = j;
    }
    col_part_ptr[K] = t;
    /* coupling columns (lambda >= 2) by the part holding most of their
     * nonzeros, then by index; untouched columns last, by index */
    int32_t *maj = ref_majority_part(m, n, rowptr, col, K, labels);
    for (int32_t k = 0; k < K; ++k)
        for (int32_t j = 0; j < n; ++j)
            if (lam[j] >= 2 && maj[j] == k) col_perm[t++] = j;
    for (int32_t j = 0; j < n; ++j)
        if (lam[j] == 0) col_perm[t++] = j;
    col_part_ptr[K + 1] = n;
    free(maj);
    free(lam);
    free(one);
    return 0;
}

/* Order of rows and columns for a split Pi (Sec. 4): each row (column) goes to
 * the first part, in the sequence k = 0..K-1, that touches it, i.e. the
 * smallest part index among its nonzeros; ties by original index; rows
 * (columns) no part touches go last, by index.  row_part_ptr[k] is the start
 * of the rows first touched by part k, [K] the start of the untouched rows,
 * [K+1] = m; likewise for columns.  Returns -1 on a bad label. */
int32_t ref_form_split(int32_t m, int32_t n, const int64_t *rowptr,
                       const int32_t *col, int32_t K, const int32_t *nz_part,
                       int32_t *row_perm, int32_t *col_perm,
                       int32_t *row_part_ptr, int32_t *col_part_ptr)
{
    int32_t *rfirst = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
    int32_t *cfirst = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t j = 0; j < n; ++j) cfirst[j] = K;
    for (int32_t i = 0; i < m; ++i) {
        rfirst[i] = K;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t k = nz_part[p];
            if (k < 0 || k >= K) { free(rfirst); free(cfirst); return -1; }
            if (k < rfirst[i]) rfirst[i] = k;
            if (k < cfirst[col[p]]) cfirst[col[p]] = k;
        }
    }
    int32_t t = 0;
    for (int32_t k = 0; k <= K; ++k) {
        row_part_ptr[k] = t;
        for (int32_t i = 0; i < m; ++i)
            if (rfirst[i] == k) row_perm[t++] = i;
    }
    row_part_ptr[K + 1] = m;
    t = 0;
    for (int32_t k = 0; k <= K; ++k) {
        col_part_ptr[k] = t;
        for (int32_t j = 0; j < n; ++j)
            if (cfirst[j] == k) col_perm[t++] = j;
    }
    col_part_ptr[K + 1] = n;
    free(rfirst);
    free(cfirst);
    return 0;
}

/* The A^k of a split in GCSR (Sec. 4; GCSR of Sec. 5.2): for each part, its
 * non-empty rows in increasing row order and, per row, its nonzeros in CSR
 * order.  Outputs (caller-allocated):
 *   part_row_ptr[K+1]   rows of part k are part_rows[part_row_ptr[k]..]
 *   part_rows[total]    row index of each GCSR row (total = sum_i lambda(r_i))
 *   gcsr_ptr[total+1]   nonzeros of GCSR row t are nz_pos[gcsr_ptr[t]..]
 *   nz_pos[nnz]         original CSR position of each nonzero
 * Returns the number of GCSR rows. */
int64_t ref_split_parts(int32_t m, const int64_t *rowptr, int32_t K,
                        const int32_t *nz_part, int64_t *part_row_ptr,
                        int32_t *part_rows, int64_t *gcsr_ptr, int64_t *nz_pos)
{
    int64_t nnz = rowptr[m];
    /* stable bucket of the nonzero positions by part: inside a part, positions
     * stay increasing, so rows come in increasing order and each row keeps
     * its CSR order */
    int64_t *start = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    int32_t *row_of = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nnz + 1));
    for (int32_t i = 0; i < m; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            row_of[p] = i;
            start[nz_part[p] + 1]++;
        }
    for (int32_t k = 0; k < K; ++k) start[k + 1] += start[k];
    for (int64_t p = 0; p < nnz; ++p) nz_pos[start[nz_part[p]]++] = p;
    int64_t rows = 0, q = 0;
    gcsr_ptr[0] = 0;
    for (int32_t k = 0; k < K; ++k) {
        part_row_ptr[k] = rows;
        int64_t end = start[k];              /* after the fill, start[k] = end of part k */
        while (q < end) {
            int32_t i = row_of[nz_pos[q]];
            while (q < end && row_of[nz_pos[q]] == i) ++q;
            part_rows[rows] = i;
            gcsr_ptr[++rows] = q;
        }
    }
    part_row_ptr[K] = rows;
    free(start);
    free(row_of);
    return rows;
}

/* ------------------------------------------------------- validators --- */

/* Structure rule of eqs. (1), (2), (5): with A_hat = P_r A P_c, every nonzero
 * of a row in R_k (k < K) lies in a column of C_k or C_B; rows of R_B are
 * unrestricted.  Returns the number of violating nonzeros; the first one's
 * (row, col) in the permuted space goes to first_bad[0..1]. */
int64_t ref_check_structure(int32_t m, int32_t n, const int64_t *rowptr,
                            const int32_t *col, const int32_t *row_perm,
                            const int32_t *col_perm, int32_t K,
                            const int32_t *row_part_ptr,
                            const int32_t *col_part_ptr, int32_t *first_bad)
{
    int32_t *colinv = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t j = 0; j < n; ++j) colinv[col_perm[j]] = j;
    int64_t bad = 0;
    first_bad[0] = first_bad[1] = -1;
    if (row_part_ptr[K + 1] != m) return -1;
    for (int32_t k = 0; k < K; ++k)
        for (int32_t ii = row_part_ptr[k]; ii < row_part_ptr[k + 1]; ++ii) {
            int32_t i = row_perm[ii];
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int32_t jj = colinv[col[p]];
                int in_ck = jj >= col_part_ptr[k] && jj < col_part_ptr[k + 1];
                int in_cb = jj >= col_part_ptr[K] && jj < col_part_ptr[K + 1];
                if (!in_ck && !in_cb) {
                    if (bad == 0) { first_bad[0] = ii; first_bad[1] = jj; }
                    ++bad;
                }
            }
        }
    free(colinv);
    return bad;
}

/* ------------------------------------------------ LRU cache simulator --- */
/* Fully associative LRU cache (the assumption stated before Theorem 1) with
 * `lines` lines of `line_bytes` bytes.  Each array lives in its own address
 * range.  Misses are counted per array id. */

enum { A_ROWPTR = 0, A_COL = 1, A_VAL = 2, A_X = 3, A_Y = 4, A_ROWLIST = 5, A_N = 6 };

typedef struct {
    int64_t cap, size, head, tail;
    int64_t *key, *prev, *next;      /* node arrays, size cap */
    int64_t *hkey, *hval;            /* open addressing: key -> node */
    int64_t hmask;
    int64_t misses[A_N];
    int64_t line_bytes;
} lru_t;

static uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void lru_init(lru_t *c, int64_t lines, int64_t line_bytes)
{
    memset(c, 0, sizeof(*c));
    c->cap = lines;
    c->line_bytes = line_bytes;
    c->head = c->tail = -1;
    c->key = (int64_t *)malloc(sizeof(int64_t) * (size_t)lines);
    c->prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)lines);
    c->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)lines);
    int64_t hs = 1;
    while (hs < 4 * lines) hs <<= 1;
    c->hmask = hs - 1;
    c->hkey = (int64_t *)malloc(sizeof(int64_t) * (size_t)hs);
    c->hval = (int64_t *)malloc(sizeof(int64_t) * (size_t)hs);
    for (int64_t i = 0; i < hs; ++i) c->hkey[i] = -1;
}

static void lru_free(lru_t *c)
{
    free(c->key); free(c->prev); free(c->next); free(c->hkey); free(c->hval);
}

static int64_t h_find(lru_t *c, int64_t key)
{
    int64_t h = (int64_t)(mix64((uint64_t)key) & (uint64_t)c->hmask);
    while (c->hkey[h] != -1) {
        if (c->hkey[h] == key) return h;
        h = (h + 1) & c->hmask;
    }
    return -(h + 1);
}

static void h_erase(lru_t *c, int64_t slot)
{
    /* backward-shift deletion for linear probing */
    int64_t i = slot;
    for (;;) {
        c->hkey[i] = -1;
        int64_t j = i;
        for (;;) {
            j = (j + 1) & c->hmask;
            if (c->hkey[j] == -1) return;
            int64_t home = (int64_t)(mix64((uint64_t)c->hkey[j]) & (uint64_t)c->hmask);
            int move = (i <= j) ? (home <= i || home > j) : (home <= i && home > j);
            if (move) {
                c->hkey[i] = c->hkey[j];
                c->hval[i] = c->hval[j];
                i = j;
                break;
            }
        }
    }
}

static void unlink_node(lru_t *c, int64_t v)
{
    if (c->prev[v] >= 0) c->next[c->prev[v]] = c->next[v]; else c->head = c->next[v];
    if (c->next[v] >= 0) c->prev[c->next[v]] = c->prev[v]; else c->tail = c->prev[v];
}

static void push_front(lru_t *c, int64_t v)
{
    c->prev[v] = -1;
    c->next[v] = c->head;
    if (c->head >= 0) c->prev[c->head] = v;
    c->head = v;
    if (c->tail < 0) c->tail = v;
}

/* access element `idx` of array `arr` whose elements are `esize` bytes */
static void lru_access(lru_t *c, int arr, int64_t idx, int64_t esize)
{
    int64_t addr = ((int64_t)arr << 44) + idx * esize;
    int64_t line = addr / c->line_bytes;
    int64_t s = h_find(c, line);
    if (s >= 0) {
        int64_t v = c->hval[s];
        unlink_node(c, v);
        push_front(c, v);
        return;
    }
    c->misses[arr]++;
    int64_t v;
    if (c->size < c->cap) {
        v = c->size++;
    } else {
        v = c->tail;
        unlink_node(c, v);
        h_erase(c, h_find(c, c->key[v]));
    }
    c->key[v] = line;
    push_front(c, v);
    s = h_find(c, line);
    s = -s - 1;
    c->hkey[s] = line;
    c->hval[s] = v;
}

/* Single SpMxV y = A x in CSR order (Sec. 2.1, 2.2): per row i, rowStart[i]
 * and rowStart[i+1], then per nonzero colIndex[p], nonzero[p] and x[col], then
 * the write of y[i].  Index arrays are 4-byte elements, values 8-byte.
 * misses[6] receives the per-array counts (rowptr, col, val, x, y, rowlist). */
void ref_cachesim_csr(int32_t m, const int64_t *rowptr, const int32_t *col,
                      int64_t cache_bytes, int64_t line_bytes, int64_t *misses)
{
    lru_t c;
    lru_init(&c, cache_bytes / line_bytes, line_bytes);
    for (int32_t i = 0; i < m; ++i) {
        lru_access(&c, A_ROWPTR, i, 4);
        lru_access(&c, A_ROWPTR, i + 1, 4);
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            lru_access(&c, A_COL, p, 4);
            lru_access(&c, A_VAL, p, 8);
            lru_access(&c, A_X, col[p], 8);
        }
        lru_access(&c, A_Y, i, 8);
    }
    for (int a = 0; a < A_N; ++a) misses[a] = c.misses[a];
    lru_free(&c);
}

/* Multiple SpMxV y <- y + A^k x, k = 1..K (Sec. 4) over GCSR parts laid out
 * one after another: GCSR row t (global over parts) has row index
 * part_rows[t] (read from the row list) and nonzeros gcsr_ptr[t]..; its y
 * entry is read-modified-written once.  gcsr_col[q] is the column of the q-th
 * stored nonzero. */
void ref_cachesim_gcsr(int64_t total_rows, const int32_t *part_rows,
                       const int64_t *gcsr_ptr, const int32_t *gcsr_col,
                       int64_t cache_bytes, int64_t line_bytes, int64_t *misses)
{
    lru_t c;
    lru_init(&c, cache_bytes / line_bytes, line_bytes);
    for (int64_t t = 0; t < total_rows; ++t) {
        lru_access(&c, A_ROWLIST, t, 4);
        lru_access(&c, A_ROWPTR, t, 4);
        lru_access(&c, A_ROWPTR, t + 1, 4);
        for (int64_t q = gcsr_ptr[t]; q < gcsr_ptr[t + 1]; ++q) {
            lru_access(&c, A_COL, q, 4);
            lru_access(&c, A_VAL, q, 8);
            lru_access(&c, A_X, gcsr_col[q], 8);
        }
        lru_access(&c, A_Y, part_rows[t], 8);
    }
    for (int a = 0; a < A_N; ++a) misses[a] = c.misses[a];
    lru_free(&c);
}

/* Generic trace replay (tests): element accesses (arr[t], idx[t]) with 8-byte
 * elements. */
void ref_cachesim_trace(int64_t len, const int32_t *arr, const int64_t *idx,
                        int64_t cache_bytes, int64_t line_bytes, int64_t *misses)
{
    lru_t c;
    lru_init(&c, cache_bytes / line_bytes, line_bytes);
    for (int64_t t = 0; t < len; ++t) lru_access(&c, arr[t], idx[t], 8);
    for (int a = 0; a < A_N; ++a) misses[a] = c.misses[a];
    lru_free(&c);
}

/* ---------------------------------------------------------------- CG --- */

static double dot(int32_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Plain FP64 conjugate gradients for SPD A from x (in/out); stops when
 * ||b - A x|| <= tol * ||b|| or after maxit iterations.  Returns the
 * iteration count; *relres receives the final true relative residual. */
int32_t ref_cg(int32_t n, const int64_t *rowptr, const int32_t *col,
               const double *val, const double *b, double *x, double tol,
               int32_t maxit, double *relres)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    ref_spmv(n, rowptr, col, val, x, 1, q, NULL);
    for (int32_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) bn = 1.0;
    double rr = dot(n, r, r);
    int32_t it = 0;
    while (it < maxit && sqrt(rr) > tol * bn) {
        ref_spmv(n, rowptr, col, val, p, 1, q, NULL);
        double alpha = rr / dot(n, p, q);
        for (int32_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rr2 = dot(n, r, r);
        double beta = rr2 / rr;
        rr = rr2;
        for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        ++it;
    }
    ref_spmv(n, rowptr, col, val, x, 1, q, NULL);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    *relres = sqrt(dot(n, r, r)) / bn;
    free(r); free(p); free(q);
    return it;
}


/* ------------------------------------------------------------------ MLP --- */

/* Selector network (an extension; the paper has no learned component):
 *   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3,
 *   loss = mean over the batch of -log softmax(z)[label].
 * W1 is nh x nin, W2 nh x nh, W3 nc x nh, row major ([out][in]).  Returns the
 * loss; writes the logits (batch x nc) if `logits` is not NULL and the
 * gradients of the loss if gW1 is not NULL.  Plain loops, FP64. */
double ref_mlp_loss_grad(int32_t batch, int32_t nin, int32_t nh, int32_t nc,
                         const double *X, const int32_t *labels,
                         const double *W1, const double *b1, const double *W2,
                         const double *b2, const double *W3, const double *b3,
                         double *gW1, double *gb1, double *gW2, double *gb2,
                         double *gW3, double *gb3, double *logits)
{
    double *h1 = (double *)calloc((size_t)batch * nh, sizeof(double));
    double *h2 = (double *)calloc((size_t)batch * nh, sizeof(double));
    double *z = (double *)calloc((size_t)batch * nc, sizeof(double));
    double *dz = (double *)calloc((size_t)batch * nc, sizeof(double));
    double *d2 = (double *)calloc((size_t)batch * nh, sizeof(double));
    double *d1 = (double *)calloc((size_t)batch * nh, sizeof(double));
    double loss = 0.0;
    for (int32_t b = 0; b < batch; ++b) {
        const double *x = X + (size_t)b * nin;
        for (int32_t o = 0; o < nh; ++o) {
            double a = b1[o];
            for (int32_t i = 0; i < nin; ++i) a += W1[(size_t)o * nin + i] * x[i];
            h1[(size_t)b * nh + o] = a > 0.0 ? a : 0.0;
        }
        for (int32_t o = 0; o < nh; ++o) {
            double a = b2[o];
            for (int32_t i = 0; i < nh; ++i) a += W2[(size_t)o * nh + i] * h1[(size_t)b * nh + i];
            h2[(size_t)b * nh + o] = a > 0.0 ? a : 0.0;
        }
        double zmax = -INFINITY;
        for (int32_t o = 0; o < nc; ++o) {
            double a = b3[o];
            for (int32_t i = 0; i < nh; ++i) a += W3[(size_t)o * nh + i] * h2[(size_t)b * nh + i];
            z[(size_t)b * nc + o] = a;
            if (a > zmax) zmax = a;
        }
        double se = 0.0;
        for (int32_t o = 0; o < nc; ++o) se += exp(z[(size_t)b * nc + o] - zmax);
        const double lse = zmax + log(se);
        loss += lse - z[(size_t)b * nc + labels[b]];
        /* d loss / d z = (softmax - onehot) / batch */
        for (int32_t o = 0; o < nc; ++o) {
            const double p = exp(z[(size_t)b * nc + o] - lse);
            dz[(size_t)b * nc + o] = (p - (o == labels[b] ? 1.0 : 0.0)) / batch;
        }
    }
    loss /= batch;
    if (logits) memcpy(logits, z, (size_t)batch * nc * sizeof(double));
    if (gW1) {
        memset(gW3, 0, (size_t)nc * nh * sizeof(double));
        memset(gb3, 0, (size_t)nc * sizeof(double));
        memset(gW2, 0, (size_t)nh * nh * sizeof(double));
        memset(gb2, 0, (size_t)nh * sizeof(double));
        memset(gW1, 0, (size_t)nh * nin * sizeof(double));
        memset(gb1, 0, (size_t)nh * sizeof(double));
        for (int32_t b = 0; b < batch; ++b) {
            for (int32_t o = 0; o < nc; ++o) {
                const double g = dz[(size_t)b * nc + o];
                gb3[o] += g;
                for (int32_t i = 0; i < nh; ++i) gW3[(size_t)o * nh + i] += g * h2[(size_t)b * nh + i];
            }
            for (int32_t i = 0; i < nh; ++i) {
                double a = 0.0;
                for (int32_t o = 0; o < nc; ++o) a += dz[(size_t)b * nc + o] * W3[(size_t)o * nh + i];
                d2[(size_t)b * nh + i] = h2[(size_t)b * nh + i] > 0.0 ? a : 0.0;
            }
            for (int32_t o = 0; o < nh; ++o) {
                const double g = d2[(size_t)b * nh + o];
                gb2[o] += g;
                for (int32_t i = 0; i < nh; ++i) gW2[(size_t)o * nh + i] += g * h1[(size_t)b * nh + i];
            }
            for (int32_t i = 0; i < nh; ++i) {
                double a = 0.0;
                for (int32_t o = 0; o < nh; ++o) a += d2[(size_t)b * nh + o] * W2[(size_t)o * nh + i];
                d1[(size_t)b * nh + i] = h1[(size_t)b * nh + i] > 0.0 ? a : 0.0;
            }
            for (int32_t o = 0; o < nh; ++o) {
                const double g = d1[(size_t)b * nh + o];
                gb1[o] += g;
                for (int32_t i = 0; i < nin; ++i)
                    gW1[(size_t)o * nin + i] += g * X[(size_t)b * nin + i];
            }
        }
    }
    free(h1);
    free(h2);
    free(z);
    free(dz);
    free(d2);
    free(d1);
    return loss;
}

