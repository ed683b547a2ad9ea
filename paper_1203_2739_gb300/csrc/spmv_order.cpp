// The comparison reorderings of the paper's experiments (Sec. 5.1), host
// side: sBFS and sRCM order the rows and columns by a breadth-first search
// (plain, or Cuthill-McKee reversed) of the bipartite graph of A, whose
// vertices are the m rows and the n columns and whose edges are the
// nonzeros; sHP_RN orders the columns by the parts of a row-net hypergraph
// partition and the rows into the nested separated block-diagonal form
// (rows inside one part with it, rows cut at a bisection between its two
// halves).  The same nesting, applied to the column border of the SB / DB
// forms a row-side bisection gives, is the nested border order: each
// bisection's cut columns between its two halves.
//
// Vertex ids: rows 0 .. m-1, columns m .. m+n-1.  Ties are broken by the
// lower id throughout, so every order is deterministic.
#include <algorithm>
#include <numeric>
#include <vector>

#include "spmv_internal.h"

namespace spmv {
namespace {

// the bipartite graph: adjacency lists of rows (their columns, increasing)
// and of columns (their rows, increasing)
struct Bipartite {
    int32_t m, n;
    const int32_t *rp, *ci;                // rows -> columns (the CSR)
    std::vector<int64_t> cp;               // columns -> rows
    std::vector<int32_t> ri;
    explicit Bipartite(const spmv_csr *A) : m(A->m), n(A->n), rp(A->rowptr), ci(A->colidx)
    {
        cp.assign((size_t)n + 1, 0);
        for (int64_t p = 0; p < A->nnz; ++p) cp[(size_t)ci[p] + 1]++;
        for (int32_t j = 0; j < n; ++j) cp[(size_t)j + 1] += cp[(size_t)j];
        ri.resize((size_t)A->nnz);
        std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
        for (int32_t i = 0; i < m; ++i)
            for (int32_t p = rp[i]; p < rp[i + 1]; ++p) ri[(size_t)fill[ci[p]]++] = i;
    }
    int64_t degree(int64_t v) const
    {
        return v < m ? (int64_t)rp[v + 1] - rp[v] : cp[(size_t)(v - m) + 1] - cp[(size_t)(v - m)];
    }
    // neighbours of v, increasing id
    template <class F>
    void each(int64_t v, F f) const
    {
        if (v < m) {
            for (int32_t p = rp[v]; p < rp[v + 1]; ++p) f((int64_t)m + ci[p]);
        } else {
            const int64_t j = v - m;
            for (int64_t p = cp[(size_t)j]; p < cp[(size_t)j + 1]; ++p) f((int64_t)ri[(size_t)p]);
        }
    }
};

// split a vertex sequence into the row and column orders
void to_perms(const Bipartite &G, const std::vector<int64_t> &seq, int32_t *row_perm,
              int32_t *col_perm)
{
    int32_t r = 0, c = 0;
    for (int64_t v : seq) {
        if (v < G.m) row_perm[r++] = (int32_t)v;
        else col_perm[c++] = (int32_t)(v - G.m);
    }
}

// sBFS: breadth-first search from row 0, neighbours in increasing id; when
// the queue runs dry, from the lowest unvisited row, then the lowest
// unvisited column.
void order_bfs(const Bipartite &G, std::vector<int64_t> &seq)
{
    const int64_t N = (int64_t)G.m + G.n;
    std::vector<char> seen((size_t)N, 0);
    seq.clear();
    seq.reserve((size_t)N);
    for (int64_t s = 0; s < N; ++s) {
        if (seen[(size_t)s]) continue;
        seen[(size_t)s] = 1;
        size_t head = seq.size();
        seq.push_back(s);
        while (head < seq.size()) {
            const int64_t v = seq[head++];
            G.each(v, [&](int64_t u) {
                if (!seen[(size_t)u]) {
                    seen[(size_t)u] = 1;
                    seq.push_back(u);
                }
            });
        }
    }
}

// breadth-first level structure of the component of s, restricted to
// vertices not in `done`; returns the last level's vertices and the depth
int32_t levels(const Bipartite &G, int64_t s, const std::vector<char> &done,
               std::vector<int32_t> &lev, std::vector<int64_t> &touched,
               std::vector<int64_t> &last)
{
    touched.clear();
    touched.push_back(s);
    lev[(size_t)s] = 0;
    int32_t depth = 0;
    for (size_t h = 0; h < touched.size(); ++h) {
        const int64_t v = touched[h];
        G.each(v, [&](int64_t u) {
            if (!done[(size_t)u] && lev[(size_t)u] < 0) {
                lev[(size_t)u] = lev[(size_t)v] + 1;
                depth = std::max(depth, lev[(size_t)u]);
                touched.push_back(u);
            }
        });
    }
    last.clear();
    for (int64_t v : touched)
        if (lev[(size_t)v] == depth) last.push_back(v);
    for (int64_t v : touched) lev[(size_t)v] = -1;
    return depth;
}

// sRCM: per connected component (taken in order of their lowest vertex),
// a pseudo-peripheral start vertex by the George-Liu procedure from the
// component's vertex of least degree; Cuthill-McKee order (each dequeued
// vertex enqueues its unvisited neighbours by increasing degree); the
// whole sequence reversed.
void order_rcm(const Bipartite &G, std::vector<int64_t> &seq)
{
    const int64_t N = (int64_t)G.m + G.n;
    std::vector<char> done((size_t)N, 0);
    std::vector<int32_t> lev((size_t)N, -1);
    std::vector<int64_t> touched, last, nb;
    seq.clear();
    seq.reserve((size_t)N);
    auto less = [&](int64_t a, int64_t b) {
        const int64_t da = G.degree(a), db = G.degree(b);
        return da != db ? da < db : a < b;
    };
    for (int64_t s0 = 0; s0 < N; ++s0) {
        if (done[(size_t)s0]) continue;
        // the component and its least-degree vertex
        levels(G, s0, done, lev, touched, last);
        int64_t v = *std::min_element(touched.begin(), touched.end(), less);
        int32_t ecc = levels(G, v, done, lev, touched, last);
        for (;;) {
            const int64_t u = *std::min_element(last.begin(), last.end(), less);
            const int32_t e2 = levels(G, u, done, lev, touched, last);
            if (e2 <= ecc) break;
            v = u;
            ecc = e2;
            levels(G, v, done, lev, touched, last);
        }
        // Cuthill-McKee from v
        size_t head = seq.size();
        done[(size_t)v] = 1;
        seq.push_back(v);
        while (head < seq.size()) {
            const int64_t w = seq[head++];
            nb.clear();
            G.each(w, [&](int64_t u) {
                if (!done[(size_t)u]) {
                    done[(size_t)u] = 1;
                    nb.push_back(u);
                }
            });
            std::sort(nb.begin(), nb.end(), less);
            for (int64_t u : nb) seq.push_back(u);
        }
    }
    std::reverse(seq.begin(), seq.end());
}

}  // namespace

// Nested separated block-diagonal order from column labels in [0, K), K a
// power of two (the leaves of a recursive bisection, left subtree first):
// columns by (label, index); a row whose columns all carry label k goes to
// block k, a row whose labels span a..b (a < b) to the separator of the
// bisection that split a from b, between its two halves; empty rows last.
spmv_status order_sbd(const spmv_csr *A, int32_t K, const int32_t *labels, int32_t *row_perm,
                      int32_t *col_perm)
{
    const int32_t m = A->m, n = A->n;
    if (K < 1 || (K & (K - 1))) {
        set_error("K=%d must be a power of two", K);
        return SPMV_E_INVALID;
    }
    for (int32_t j = 0; j < n; ++j)
        if (labels[j] < 0 || labels[j] >= K) {
            set_error("column label %d of column %d outside [0, %d)", labels[j], j, K);
            return SPMV_E_INVALID;
        }
    std::iota(col_perm, col_perm + n, 0);
    std::stable_sort(col_perm, col_perm + n,
                     [&](int32_t a, int32_t b) { return labels[a] < labels[b]; });
    // key: leaf k -> 2k; the separator whose right half starts at leaf s
    // -> 2s - 1; empty rows -> 2K
    std::vector<int64_t> key((size_t)m);
    for (int32_t i = 0; i < m; ++i) {
        if (A->rowptr[i] == A->rowptr[i + 1]) {
            key[(size_t)i] = 2 * (int64_t)K;
            continue;
        }
        int32_t a = K, b = -1;
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
            a = std::min(a, labels[A->colidx[p]]);
            b = std::max(b, labels[A->colidx[p]]);
        }
        if (a == b) {
            key[(size_t)i] = 2 * (int64_t)a;
        } else {
            int32_t hb = 31 - __builtin_clz((unsigned)(a ^ b));   // highest differing bit
            const int64_t s = ((int64_t)b >> hb) << hb;
            key[(size_t)i] = 2 * s - 1;
        }
    }
    std::iota(row_perm, row_perm + m, 0);
    std::stable_sort(row_perm, row_perm + m,
                     [&](int32_t a, int32_t b) { return key[(size_t)a] < key[(size_t)b]; });
    return SPMV_OK;
}

// Nested bisection order of the SB / DB forms: labels[m] are row parts in
// [0, K] (K = the DB row border), the leaves of a bisection tree.  Rows by
// (part, index), border last.  A column's key comes from the parts of its
// rows outside the row border: one part k -> 2k; parts a < b -> 2s - 1, s the
// first leaf of the right half of the bisection that parted a from b (the
// bits of a and b above their highest differing bit, that bit set); no part
// -> 2K.
spmv_status order_nested(const spmv_csr *A, int32_t K, const int32_t *labels, int32_t *row_perm,
                         int32_t *col_perm)
{
    const int32_t m = A->m, n = A->n;
    if (K < 1 || (K & (K - 1))) {
        set_error("K=%d must be a power of two", K);
        return SPMV_E_INVALID;
    }
    for (int32_t i = 0; i < m; ++i)
        if (labels[i] < 0 || labels[i] > K) {
            set_error("row label %d of row %d outside [0, %d]", labels[i], i, K);
            return SPMV_E_INVALID;
        }
    std::iota(row_perm, row_perm + m, 0);
    std::stable_sort(row_perm, row_perm + m,
                     [&](int32_t a, int32_t b) { return labels[a] < labels[b]; });
    std::vector<int32_t> lo((size_t)n, K), hi((size_t)n, -1);
    for (int32_t i = 0; i < m; ++i) {
        const int32_t l = labels[i];
        if (l == K) continue;
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
            const int32_t c = A->colidx[p];
            lo[(size_t)c] = std::min(lo[(size_t)c], l);
            hi[(size_t)c] = std::max(hi[(size_t)c], l);
        }
    }
    std::vector<int64_t> key((size_t)n);
    for (int32_t j = 0; j < n; ++j) {
        const int32_t a = lo[(size_t)j], b = hi[(size_t)j];
        if (b < 0) {
            key[(size_t)j] = 2 * (int64_t)K;
        } else if (a == b) {
            key[(size_t)j] = 2 * (int64_t)a;
        } else {
            const int32_t hb = 31 - __builtin_clz((unsigned)(a ^ b));
            const int64_t s = ((int64_t)b >> hb) << hb;
            key[(size_t)j] = 2 * s - 1;
        }
    }
    std::iota(col_perm, col_perm + n, 0);
    std::stable_sort(col_perm, col_perm + n,
                     [&](int32_t a, int32_t b) { return key[(size_t)a] < key[(size_t)b]; });
    return SPMV_OK;
}

spmv_status reorder(const spmv_csr *A, int32_t method, int32_t K, const int32_t *labels,
                    int32_t *row_perm, int32_t *col_perm)
{
    spmv_status st = validate_csr(A);
    if (st != SPMV_OK) return st;
    if (!row_perm || !col_perm || (method == SPMV_ORDER_SBD && !labels && A->n > 0) ||
        (method == SPMV_ORDER_NESTED && !labels && A->m > 0)) {
        set_error("NULL argument");
        return SPMV_E_INVALID;
    }
    if (method == SPMV_ORDER_SBD) return order_sbd(A, K, labels, row_perm, col_perm);
    if (method == SPMV_ORDER_NESTED) return order_nested(A, K, labels, row_perm, col_perm);
    if (method != SPMV_ORDER_BFS && method != SPMV_ORDER_RCM) {
        set_error("unknown ordering %d", method);
        return SPMV_E_INVALID;
    }
    Bipartite G(A);
    std::vector<int64_t> seq;
    if (method == SPMV_ORDER_BFS) order_bfs(G, seq);
    else order_rcm(G, seq);
    to_perms(G, seq, row_perm, col_perm);
    return SPMV_OK;
}

}  // namespace spmv

extern "C" spmv_status spmv_reorder(const spmv_csr *A, int32_t method, int32_t K,
                                    const int32_t *labels, int32_t *row_perm, int32_t *col_perm)
{
    spmv::clear_error();
    try {
        return spmv::reorder(A, method, K, labels, row_perm, col_perm);
    } catch (const std::bad_alloc &) {
        spmv::set_error("out of host memory");
        return SPMV_E_NOMEM;
    } catch (...) {
        spmv::set_error("internal error");
        return SPMV_E_INTERNAL;
    }
}
