// Host side of a plan: validation, the permuted matrix P_r A P_c (Sec. 3),
// the parts of the SB / DB forms (eqs. 1, 5) and of a split (Sec. 4), and the
// tiling of every part into CTA-sized pieces whose x working set fits in
// shared memory -- the GPU counterpart of the paper's "fits into the cache"
// (Sec. 3, Sec. 5.1).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <thread>

#include "spmv_internal.h"

namespace spmv {

// ---------------------------------------------------------------- errors --
static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[768];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

void clear_error() { g_err.clear(); }

int hardware_threads()
{
    unsigned h = std::thread::hardware_concurrency();
    return h == 0 ? 1 : (int)std::min(h, 64u);
}

template <class F>
static void parallel_for(int64_t n, int threads, F f)
{
    if (threads <= 1 || n < (1 << 16)) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> ts;
    int64_t chunk = (n + threads - 1) / threads;
    for (int t = 0; t < threads; ++t) {
        int64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) break;
        ts.emplace_back(f, b, e);
    }
    for (auto &t : ts) t.join();
}

// ------------------------------------------------------------ validation --
spmv_status validate_csr(const spmv_csr *A)
{
    if (!A) {
        set_error("matrix is NULL");
        return SPMV_E_INVALID;
    }
    if (A->m < 0 || A->n < 0 || A->nnz < 0) {
        set_error("negative size m=%d n=%d nnz=%lld", A->m, A->n, (long long)A->nnz);
        return SPMV_E_INVALID;
    }
    if (A->nnz >= (int64_t)INT32_MAX) {
        set_error("nnz=%lld does not fit int32 row starts", (long long)A->nnz);
        return SPMV_E_UNSUPPORTED;
    }
    if (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->vals))) {
        set_error("NULL CSR array");
        return SPMV_E_INVALID;
    }
    if (A->rowptr[0] != 0 || A->rowptr[A->m] != A->nnz) {
        set_error("rowptr[0]=%d rowptr[m]=%d, expected 0 and nnz=%lld", A->rowptr[0],
                  A->rowptr[A->m], (long long)A->nnz);
        return SPMV_E_INVALID;
    }
    for (int32_t i = 0; i < A->m; ++i) {
        int32_t a = A->rowptr[i], b = A->rowptr[i + 1];
        if (b < a) {
            set_error("rowptr decreases at row %d", i);
            return SPMV_E_INVALID;
        }
        for (int32_t p = a; p < b; ++p) {
            int32_t c = A->colidx[p];
            if (c < 0 || c >= A->n) {
                set_error("column %d out of range at (row %d, nonzero %d)", c, i, p);
                return SPMV_E_INVALID;
            }
            if (p > a && c <= A->colidx[p - 1]) {
                set_error("columns not sorted/unique in row %d at column %d", i, c);
                return SPMV_E_INVALID;
            }
        }
    }
    return SPMV_OK;
}

static spmv_status check_perm(const int32_t *p, int32_t n, const char *what)
{
    std::vector<char> seen((size_t)n, 0);
    for (int32_t i = 0; i < n; ++i) {
        if (p[i] < 0 || p[i] >= n || seen[p[i]]) {
            set_error("%s is not a bijection: entry %d = %d", what, i, p[i]);
            return SPMV_E_STRUCTURE;
        }
        seen[p[i]] = 1;
    }
    return SPMV_OK;
}

static spmv_status check_part_ptr(const int32_t *p, int32_t K, int32_t total, const char *what)
{
    if (!p) {
        set_error("%s is NULL", what);
        return SPMV_E_INVALID;
    }
    if (p[0] != 0 || p[K + 1] != total) {
        set_error("%s must start at 0 and end at %d", what, total);
        return SPMV_E_STRUCTURE;
    }
    for (int32_t k = 0; k <= K; ++k)
        if (p[k + 1] < p[k]) {
            set_error("%s decreases at part %d", what, k);
            return SPMV_E_STRUCTURE;
        }
    return SPMV_OK;
}

// ------------------------------------------------------------------ bf16 --
uint16_t bf16_rne(double v)
{
    uint16_t sign = std::signbit(v) ? 0x8000 : 0;
    if (std::isnan(v)) return (uint16_t)(sign | 0x7FC0);
    double a = std::fabs(v);
    if (a == 0.0) return sign;
    if (std::isinf(a)) return (uint16_t)(sign | 0x7F80);
    int e;
    std::frexp(a, &e);                       // a = f * 2^e, f in [0.5, 1)
    int qe = std::max(e - 8, -133);          // 8 significant bits; subnormal quantum 2^-133
    double r = std::nearbyint(std::ldexp(a, -qe));   // ties to even
    double res = std::ldexp(r, qe);
    const double maxbf = std::ldexp(255.0, 120);     // (2 - 2^-7) * 2^127
    if (res > maxbf) return (uint16_t)(sign | 0x7F80);
    float f = (float)res;                    // exact
    uint32_t bits;
    std::memcpy(&bits, &f, 4);
    return (uint16_t)(sign | (bits >> 16));
}

// ------------------------------------------------------- P_r A P_c (Sec. 3) --
struct Permuted {
    std::vector<int32_t> rp;   // m+1
    std::vector<int32_t> col;  // new column index
    std::vector<int32_t> src;  // original CSR position of each nonzero
};

static void build_permuted(const spmv_csr *A, const int32_t *rperm, const int32_t *cperm,
                           Permuted *P)
{
    const int32_t m = A->m, n = A->n;
    const int64_t nnz = A->nnz;
    P->rp.assign((size_t)m + 1, 0);
    P->col.resize((size_t)nnz);
    P->src.resize((size_t)nnz);
    for (int32_t i = 0; i < m; ++i) {
        int32_t o = rperm ? rperm[i] : i;
        P->rp[i + 1] = P->rp[i] + (A->rowptr[o + 1] - A->rowptr[o]);
    }
    std::vector<int32_t> colinv;
    if (cperm) {
        colinv.resize((size_t)n);
        for (int32_t j = 0; j < n; ++j) colinv[cperm[j]] = j;
    }
    const int threads = hardware_threads();
    parallel_for(m, threads, [&](int64_t b, int64_t e) {
        std::vector<std::pair<int32_t, int32_t>> buf;
        for (int64_t i = b; i < e; ++i) {
            int32_t o = rperm ? rperm[i] : (int32_t)i;
            int32_t a = A->rowptr[o], z = A->rowptr[o + 1];
            int32_t q = P->rp[i];
            if (!cperm) {
                for (int32_t p = a; p < z; ++p, ++q) {
                    P->col[q] = A->colidx[p];
                    P->src[q] = p;
                }
                continue;
            }
            buf.clear();
            for (int32_t p = a; p < z; ++p) buf.emplace_back(colinv[A->colidx[p]], p);
            std::sort(buf.begin(), buf.end());
            for (auto &pr : buf) {
                P->col[q] = pr.first;
                P->src[q] = pr.second;
                ++q;
            }
        }
    });
}

// ------------------------------------------------------------------ tiler --
namespace {

struct TileCfg {
    int32_t W;          // staging capacity (x entries)
    int32_t tnnz;       // nonzero budget per tile
    int32_t long_t;     // rows longer than this become chunks
    int32_t chunk;      // nonzeros per chunk
    int32_t max_rows;   // rows per tile
    bool stage;         // staging allowed
    double min_reuse;   // stage only if nnz >= min_reuse * gathered list entries
};

struct Tiler {
    const TileCfg cfg;
    const std::vector<int32_t> &prp;   // plan row starts
    const std::vector<int32_t> &col;   // plan-order global columns
    HostPlan &P;
    std::vector<int32_t> mark, mark2, loc;
    int32_t stamp = 0;
    std::vector<int32_t> distinct;

    Tiler(const TileCfg &c, const std::vector<int32_t> &rp, const std::vector<int32_t> &cl,
          HostPlan &plan, int32_t n)
        : cfg(c), prp(rp), col(cl), P(plan), mark((size_t)n, -1), mark2((size_t)n, -1),
          loc((size_t)n, 0) {}

    // Close a tile over plan rows [r0, r1) whose distinct columns carry mark
    // == stamp.  Decide staged vs global, pick the contiguous run, fill local
    // indices.  y0 as in Tile.
    void emit(int32_t r0, int32_t r1, int32_t y0, int32_t h0, int32_t h1, bool force_global)
    {
        if (r1 <= r0) return;
        const int32_t p0 = prp[r0], p1 = prp[r1];
        const int32_t tile_nnz = p1 - p0;
        Tile t{};
        t.r0 = r0;
        t.r1 = r1;
        t.y0 = y0;
        bool staged = cfg.stage && !force_global && tile_nnz > 0;
        if (staged) {
            distinct.clear();
            for (int32_t q = p0; q < p1; ++q) {
                int32_t c = col[q];
                if (mark2[c] != stamp) {
                    mark2[c] = stamp;
                    distinct.push_back(c);
                }
            }
            std::sort(distinct.begin(), distinct.end());
            // contiguous run inside the home column range, if dense enough
            int32_t lo = -1, hi = -1, in_home = 0;
            for (int32_t c : distinct)
                if (c >= h0 && c < h1) {
                    if (lo < 0) lo = c;
                    hi = c;
                    ++in_home;
                }
            int32_t runlen = 0, run0 = 0;
            if (in_home > 0) {
                int32_t span = hi - lo + 1;
                int32_t others = (int32_t)distinct.size() - in_home;
                if (span <= 2 * in_home && span + others <= cfg.W) {
                    run0 = lo;
                    runlen = span;
                }
            }
            int32_t listlen = 0;
            for (int32_t c : distinct)
                if (!(runlen > 0 && c >= run0 && c < run0 + runlen)) ++listlen;
            if (runlen + listlen > cfg.W ||
                (double)tile_nnz < cfg.min_reuse * (double)listlen)
                staged = false;
            if (staged) {
                t.kind = TILE_STAGED;
                t.run0 = run0;
                t.runlen = runlen;
                t.list0 = (int32_t)P.xlist.size();
                t.listlen = listlen;
                int32_t pos = runlen;
                for (int32_t c : distinct) {
                    if (runlen > 0 && c >= run0 && c < run0 + runlen) {
                        loc[c] = c - run0;
                    } else {
                        loc[c] = pos++;
                        P.xlist.push_back(c);
                    }
                }
                for (int32_t q = p0; q < p1; ++q) P.col16[q] = (uint16_t)loc[col[q]];
                P.staged_entries += runlen + listlen;
                P.list_entries += listlen;
                P.n_staged_tiles++;
            }
        }
        if (!staged) {
            t.kind = TILE_GLOBAL;
            P.n_global_tiles++;
        }
        P.tiles.push_back(t);
    }

    // Tile plan rows [rb, re).  chunked[r] marks rows handled as chunks.
    // identity: plan row r writes y[r] (SB/DB); else via dst.
    void tile_rows(int32_t rb, int32_t re, int32_t h0, int32_t h1, bool identity,
                   const std::vector<char> &chunked, bool force_global)
    {
        int32_t cur0 = -1, cur_rows = 0, cur_nnz = 0, cur_d = 0;
        auto close = [&](int32_t end) {
            if (cur0 >= 0) emit(cur0, end, identity ? cur0 : -1, h0, h1, force_global);
            cur0 = -1;
            cur_rows = cur_nnz = cur_d = 0;
            ++stamp;
        };
        for (int32_t r = rb; r < re; ++r) {
            if (chunked[r]) {
                close(r);
                continue;
            }
            const int32_t a = prp[r], b = prp[r + 1], len = b - a;
            int32_t newd = 0;
            if (cur0 >= 0)
                for (int32_t q = a; q < b; ++q) newd += (mark[col[q]] != stamp);
            if (cur0 >= 0 && (cur_d + newd > cfg.W || cur_nnz + len > cfg.tnnz ||
                              cur_rows >= cfg.max_rows)) {
                close(r);
            }
            if (cur0 < 0) {
                cur0 = r;
                newd = len;
            }
            for (int32_t q = a; q < b; ++q) mark[col[q]] = stamp;
            cur_d += newd;
            cur_nnz += len;
            cur_rows++;
        }
        close(re);
    }
};

int32_t pow2_lanes(double mean)
{
    double want = mean / 2.0;
    int32_t l = 2;
    while (l < 32 && l < want) l *= 2;
    return l;
}

}  // namespace

// --------------------------------------------------------------- the plan --
spmv_status build_host_plan(const spmv_csr *A, const spmv_perm *perm,
                            const spmv_splits *splits, const spmv_opts *opts,
                            HostPlan *P)
{
    spmv_status st = validate_csr(A);
    if (st != SPMV_OK) return st;
    spmv_opts o{};
    if (opts) o = *opts;
    if (o.nrhs == 0) o.nrhs = 1;
    if (o.dtype < SPMV_F64 || o.dtype > SPMV_BF16) {
        set_error("unknown dtype %d", o.dtype);
        return SPMV_E_INVALID;
    }
    if (o.nrhs != 1 && o.nrhs != 2 && o.nrhs != 4 && o.nrhs != 8) {
        set_error("nrhs=%d: supported right-hand-side counts are 1, 2, 4, 8", o.nrhs);
        return SPMV_E_UNSUPPORTED;
    }
    if (o.lanes != 0 && o.lanes != 2 && o.lanes != 4 && o.lanes != 8 && o.lanes != 16 &&
        o.lanes != 32) {
        set_error("lanes=%d: must be 0, 2, 4, 8, 16 or 32", o.lanes);
        return SPMV_E_INVALID;
    }
    const int32_t form = splits ? splits->form : SPMV_NATURAL;
    if (form < SPMV_NATURAL || form > SPMV_SPLIT) {
        set_error("unknown form %d", form);
        return SPMV_E_INVALID;
    }
    const int32_t m = A->m, n = A->n;
    const int64_t nnz = A->nnz;
    const int xb = (o.dtype == SPMV_F64) ? 8 : 4;
    int32_t W = o.tile_cols > 0 ? o.tile_cols : (48 * 1024) / (xb * o.nrhs);
    if ((int64_t)W * xb * o.nrhs > 227 * 1024 || W > 65535) {
        set_error("tile_cols=%d does not fit shared memory (x entries of %d bytes, r=%d)", W,
                  xb, o.nrhs);
        return SPMV_E_UNSUPPORTED;
    }
    P->m = m;
    P->n = n;
    P->nnz = nnz;
    P->form = form;
    P->dtype = o.dtype;
    P->nrhs = o.nrhs;
    P->flags = o.flags;
    P->tile_cols = W;

    // permutation
    const int32_t *rperm = perm ? perm->row_perm : nullptr;
    const int32_t *cperm = perm ? perm->col_perm : nullptr;
    if (rperm && (st = check_perm(rperm, m, "row_perm")) != SPMV_OK) return st;
    if (cperm && (st = check_perm(cperm, n, "col_perm")) != SPMV_OK) return st;
    if (rperm) P->row_perm.assign(rperm, rperm + m);
    if (cperm) P->col_perm.assign(cperm, cperm + n);

    Permuted Ah;
    build_permuted(A, rperm, cperm, &Ah);

    const double mean_len = m > 0 ? (double)nnz / (double)m : 1.0;

    // ---------------------------------------- natural form, plain kernel --
    if (form == SPMV_NATURAL && !(o.flags & SPMV_FLAG_TILED_NATURAL)) {
        P->use_k1 = true;
        P->K = 1;
        P->lanes = o.lanes ? o.lanes : pow2_lanes(mean_len);
        P->long_thresh = o.long_row > 0 ? o.long_row : std::max(1024, 64 * P->lanes);
        P->rowptr.swap(Ah.rp);
        P->col32.swap(Ah.col);
        P->val.resize((size_t)nnz);
        for (int64_t q = 0; q < nnz; ++q) P->val[q] = A->vals[Ah.src[q]];
        for (int32_t i = 0; i < m; ++i)
            if (P->rowptr[i + 1] - P->rowptr[i] > P->long_thresh) P->long_rows.push_back(i);
        return SPMV_OK;
    }

    // --------------------------------------------------------- tiled forms --
    P->use_k1 = false;
    int32_t K = 1;
    std::vector<int32_t> rp_part, cp_part;   // K+2 each (home ranges)
    // plan rows: their starts (prp), y row (prow), part boundaries (pr_part)
    std::vector<int32_t> prp, prow, pr_part;
    std::vector<int32_t> pcol;               // plan-order global columns
    std::vector<int32_t> psrc;               // plan-order original positions

    if (form == SPMV_SB || form == SPMV_DB) {
        K = splits->K;
        if (K < 1) {
            set_error("K=%d must be >= 1", K);
            return SPMV_E_INVALID;
        }
        if ((st = check_part_ptr(splits->row_part_ptr, K, m, "row_part_ptr")) != SPMV_OK)
            return st;
        if ((st = check_part_ptr(splits->col_part_ptr, K, n, "col_part_ptr")) != SPMV_OK)
            return st;
        rp_part.assign(splits->row_part_ptr, splits->row_part_ptr + K + 2);
        cp_part.assign(splits->col_part_ptr, splits->col_part_ptr + K + 2);
        if (form == SPMV_SB && rp_part[K] != m) {
            set_error("SB form has a non-empty row border (row_part_ptr[K]=%d < m=%d)",
                      rp_part[K], m);
            return SPMV_E_STRUCTURE;
        }
        // structure rule of eqs. (1), (2), (5)
        const int32_t cb0 = cp_part[K], cb1 = cp_part[K + 1];
        for (int32_t k = 0; k < K; ++k)
            for (int32_t i = rp_part[k]; i < rp_part[k + 1]; ++i)
                for (int32_t q = Ah.rp[i]; q < Ah.rp[i + 1]; ++q) {
                    int32_t c = Ah.col[q];
                    bool ok = (c >= cp_part[k] && c < cp_part[k + 1]) || (c >= cb0 && c < cb1);
                    if (!ok) {
                        set_error("nonzero (%d, %d) of row slice R_%d lies outside C_%d and "
                                  "the column border", i, c, k, k);
                        return SPMV_E_STRUCTURE;
                    }
                }
        prp.swap(Ah.rp);
        pcol.swap(Ah.col);
        psrc.swap(Ah.src);
        prow.resize((size_t)m);
        std::iota(prow.begin(), prow.end(), 0);
        pr_part = rp_part;
    } else if (form == SPMV_SPLIT) {
        K = splits->K;
        if (K < 1) {
            set_error("K=%d must be >= 1", K);
            return SPMV_E_INVALID;
        }
        if (!splits->nz_part && nnz > 0) {
            set_error("split form needs nz_part");
            return SPMV_E_INVALID;
        }
        for (int64_t p = 0; p < nnz; ++p)
            if (splits->nz_part[p] < 0 || splits->nz_part[p] >= K) {
                set_error("nz_part[%lld]=%d outside [0, %d)", (long long)p, splits->nz_part[p], K);
                return SPMV_E_INVALID;
            }
        if (splits->col_part_ptr) {
            if ((st = check_part_ptr(splits->col_part_ptr, K, n, "col_part_ptr")) != SPMV_OK)
                return st;
            cp_part.assign(splits->col_part_ptr, splits->col_part_ptr + K + 2);
        }
        // bucket nonzeros by part, stable: rows increase inside each part and
        // each row keeps its CSR order (GCSR of each A^k, Sec. 4, 5.2)
        std::vector<int64_t> cnt((size_t)K + 1, 0);
        for (int64_t q = 0; q < nnz; ++q) cnt[splits->nz_part[Ah.src[q]] + 1]++;
        for (int32_t k = 0; k < K; ++k) cnt[k + 1] += cnt[k];
        std::vector<int32_t> order((size_t)nnz);
        std::vector<int32_t> row_of((size_t)nnz);
        {
            std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
            for (int32_t i = 0; i < m; ++i)
                for (int32_t q = Ah.rp[i]; q < Ah.rp[i + 1]; ++q) {
                    int32_t k = splits->nz_part[Ah.src[q]];
                    int64_t d = pos[k]++;
                    order[d] = q;
                    row_of[d] = i;
                }
        }
        pcol.resize((size_t)nnz);
        psrc.resize((size_t)nnz);
        for (int64_t d = 0; d < nnz; ++d) {
            pcol[d] = Ah.col[order[d]];
            psrc[d] = Ah.src[order[d]];
        }
        prp.clear();
        prow.clear();
        pr_part.assign((size_t)K + 2, 0);
        int64_t d = 0;
        for (int32_t k = 0; k < K; ++k) {
            pr_part[k] = (int32_t)prow.size();
            while (d < cnt[k + 1]) {
                int32_t i = row_of[d];
                prp.push_back((int32_t)d);
                prow.push_back(i);
                while (d < cnt[k + 1] && row_of[d] == i) ++d;
            }
        }
        pr_part[K] = pr_part[K + 1] = (int32_t)prow.size();
        prp.push_back((int32_t)nnz);
    } else {
        // natural form through the tiled kernel: one part, no home range
        K = 1;
        prp.swap(Ah.rp);
        pcol.swap(Ah.col);
        psrc.swap(Ah.src);
        prow.resize((size_t)m);
        std::iota(prow.begin(), prow.end(), 0);
        pr_part = {0, m, m};
    }
    P->K = K;
    const int32_t R = (int32_t)prow.size();

    // tile configuration
    TileCfg cfg;
    cfg.W = W;
    cfg.tnnz = o.tile_nnz > 0 ? o.tile_nnz : 8192;
    cfg.long_t = std::min(o.long_row > 0 ? o.long_row : 2048, W);
    cfg.chunk = std::max(cfg.long_t, 1024);
    cfg.max_rows = 4096;
    cfg.stage = !(o.flags & SPMV_FLAG_NO_STAGING);
    cfg.min_reuse = 1.25;
    {
        // mean length of the rows the row kernels see
        int64_t s = 0, c = 0;
        for (int32_t r = 0; r < R; ++r) {
            int32_t len = prp[r + 1] - prp[r];
            if (len <= cfg.long_t) {
                s += len;
                ++c;
            }
        }
        P->lanes = o.lanes ? o.lanes : pow2_lanes(c ? (double)s / (double)c : 1.0);
    }
    P->long_thresh = cfg.long_t;

    // pieces per plan row, slots and fix-ups (split rows shared by several
    // parts and chunked long rows are summed in part / chunk order)
    std::vector<char> chunked((size_t)R, 0), has_chunk((size_t)m, 0);
    std::vector<int32_t> pieces((size_t)R, 1), tot((size_t)m, 0);
    for (int32_t r = 0; r < R; ++r) {
        int32_t len = prp[r + 1] - prp[r];
        if (len > cfg.long_t) {
            chunked[r] = 1;
            has_chunk[prow[r]] = 1;
            pieces[r] = (len + cfg.chunk - 1) / cfg.chunk;
        }
        tot[prow[r]] += pieces[r];
    }
    std::vector<int32_t> base((size_t)m, -1);
    int64_t slots = 0;
    for (int32_t i = 0; i < m; ++i)
        if (tot[i] != 1 || has_chunk[i]) {
            base[i] = (int32_t)slots;
            P->fixups.push_back(Fixup{i, (int32_t)slots, tot[i], 0});
            slots += tot[i];
        }
    if (slots >= INT32_MAX) {
        set_error("too many partial sums");
        return SPMV_E_UNSUPPORTED;
    }
    P->partial_slots = slots;
    const bool identity = (form == SPMV_SB || form == SPMV_DB || form == SPMV_NATURAL);
    std::vector<int32_t> run((size_t)m, 0);
    if (!identity) P->dst.assign((size_t)R, 0);
    std::vector<Tile> chunk_tiles;
    for (int32_t r = 0; r < R; ++r) {
        int32_t i = prow[r];
        int32_t slot = base[i] >= 0 ? base[i] + run[i] : -1;
        run[i] += pieces[r];
        if (!identity) P->dst[r] = (slot >= 0) ? -(slot + 1) : i;
        if (chunked[r]) {
            for (int32_t c = 0; c < pieces[r]; ++c) {
                Tile t{};
                t.kind = TILE_CHUNK;
                t.r0 = prp[r] + c * cfg.chunk;
                t.r1 = std::min(prp[r + 1], t.r0 + cfg.chunk);
                t.y0 = slot + c;
                chunk_tiles.push_back(t);
            }
        }
    }
    // chunk tiles first so the longest work starts early
    P->tiles = chunk_tiles;
    P->n_chunk_tiles = (int32_t)chunk_tiles.size();
    P->col16.assign((size_t)nnz, 0);

    Tiler tiler(cfg, prp, pcol, *P, n);
    for (int32_t k = 0; k < K; ++k) {
        int32_t h0 = 0, h1 = n;
        if (!cp_part.empty()) {
            h0 = cp_part[k];
            h1 = cp_part[k + 1];
        }
        tiler.tile_rows(pr_part[k], pr_part[k + 1], h0, h1, identity, chunked, false);
    }
    // DB row border R_B: x entries gathered through L2, as the paper charges
    // every border nonzero a miss (eq. 6)
    if (pr_part[K + 1] > pr_part[K])
        tiler.tile_rows(pr_part[K], pr_part[K + 1], 0, 0, identity, chunked, true);

    P->rowptr.swap(prp);
    P->col32.swap(pcol);
    P->val.resize((size_t)nnz);
    for (int64_t q = 0; q < nnz; ++q) P->val[q] = A->vals[psrc[q]];

    // coverage: every y row is written exactly once (by a tile row or a fix-up)
    {
        std::vector<int32_t> cover((size_t)m, 0);
        for (const Tile &t : P->tiles) {
            if (t.kind == TILE_CHUNK) continue;
            for (int32_t r = t.r0; r < t.r1; ++r) {
                if (t.y0 >= 0) cover[t.y0 + (r - t.r0)]++;
                else if (P->dst[r] >= 0) cover[P->dst[r]]++;
            }
        }
        for (const Fixup &f : P->fixups) cover[f.row]++;
        for (int32_t i = 0; i < m; ++i)
            if (cover[i] != 1) {
                set_error("internal: y row %d written %d times", i, cover[i]);
                return SPMV_E_INTERNAL;
            }
    }
    return SPMV_OK;
}

// ------------------------------------------------------ form from labels --
spmv_status form_from_labels(const spmv_csr *A, int32_t form, int32_t K,
                             const int32_t *labels, int32_t *row_perm, int32_t *col_perm,
                             int32_t *row_part_ptr, int32_t *col_part_ptr)
{
    spmv_status st = validate_csr(A);
    if (st != SPMV_OK) return st;
    if (K < 1) {
        set_error("K=%d must be >= 1", K);
        return SPMV_E_INVALID;
    }
    if (!labels || !row_perm || !col_perm || !row_part_ptr || !col_part_ptr) {
        set_error("NULL argument");
        return SPMV_E_INVALID;
    }
    const int32_t m = A->m, n = A->n;
    if (form == SPMV_SB || form == SPMV_DB) {
        const int32_t maxlab = (form == SPMV_DB) ? K : K - 1;
        std::vector<int32_t> cnt((size_t)K + 2, 0);
        for (int32_t i = 0; i < m; ++i) {
            if (labels[i] < 0 || labels[i] > maxlab) {
                set_error("row label %d of row %d outside [0, %d]", labels[i], i, maxlab);
                return SPMV_E_INVALID;
            }
            cnt[labels[i] + 1]++;
        }
        for (int32_t k = 0; k <= K; ++k) cnt[k + 1] += cnt[k];
        for (int32_t k = 0; k <= K + 1; ++k) row_part_ptr[k] = cnt[k];
        row_part_ptr[K + 1] = m;
        {
            std::vector<int32_t> pos(cnt.begin(), cnt.end() - 1);
            for (int32_t i = 0; i < m; ++i) row_perm[pos[labels[i]]++] = i;
        }
        // connectivity of each column over non-border rows (eq. 3 / eq. 5):
        // track the part seen first and whether a second one appeared
        std::vector<int32_t> first((size_t)n, -1);
        std::vector<char> multi((size_t)n, 0);
        for (int32_t i = 0; i < m; ++i) {
            int32_t l = labels[i];
            if (l >= K) continue;
            for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
                int32_t c = A->colidx[p];
                if (first[c] < 0) first[c] = l;
                else if (first[c] != l) multi[c] = 1;
            }
        }
        std::vector<int32_t> ccnt((size_t)K + 3, 0);   // C_0..C_{K-1}, multi, none
        auto cls = [&](int32_t c) { return first[c] < 0 ? K + 1 : (multi[c] ? K : first[c]); };
        for (int32_t c = 0; c < n; ++c) ccnt[cls(c) + 1]++;
        for (int32_t k = 0; k <= K + 1; ++k) ccnt[k + 1] += ccnt[k];
        for (int32_t k = 0; k <= K; ++k) col_part_ptr[k] = ccnt[k];
        col_part_ptr[K + 1] = n;
        std::vector<int32_t> pos(ccnt.begin(), ccnt.end() - 1);
        for (int32_t c = 0; c < n; ++c) col_perm[pos[cls(c)]++] = c;
        return SPMV_OK;
    }
    if (form == SPMV_SPLIT) {
        // rows / columns grouped by the first part (smallest k) touching them
        std::vector<int32_t> rf((size_t)m, K), cf((size_t)n, K);
        for (int32_t i = 0; i < m; ++i)
            for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
                int32_t k = labels[p];
                if (k < 0 || k >= K) {
                    set_error("nonzero label %d at position %d outside [0, %d)", k, p, K);
                    return SPMV_E_INVALID;
                }
                rf[i] = std::min(rf[i], k);
                cf[A->colidx[p]] = std::min(cf[A->colidx[p]], k);
            }
        auto group = [K](const std::vector<int32_t> &f, int32_t cnt_total, int32_t *perm,
                         int32_t *ptr) {
            std::vector<int32_t> c((size_t)K + 2, 0);
            for (int32_t v : f) c[v + 1]++;
            for (int32_t k = 0; k <= K; ++k) c[k + 1] += c[k];
            for (int32_t k = 0; k <= K; ++k) ptr[k] = c[k];
            ptr[K + 1] = cnt_total;
            std::vector<int32_t> pos(c.begin(), c.end() - 1);
            for (int32_t i = 0; i < (int32_t)f.size(); ++i) perm[pos[f[i]]++] = i;
        };
        group(rf, m, row_perm, row_part_ptr);
        group(cf, n, col_perm, col_part_ptr);
        return SPMV_OK;
    }
    set_error("form %d has no labels", form);
    return SPMV_E_INVALID;
}

}  // namespace spmv

extern "C" const char *spmv_last_error(void) { return spmv::g_err.c_str(); }

extern "C" spmv_status spmv_form_from_labels(const spmv_csr *A, int32_t form, int32_t K,
                                             const int32_t *labels, int32_t *row_perm,
                                             int32_t *col_perm, int32_t *row_part_ptr,
                                             int32_t *col_part_ptr)
{
    spmv::clear_error();
    try {
        return spmv::form_from_labels(A, form, K, labels, row_perm, col_perm, row_part_ptr,
                                      col_part_ptr);
    } catch (const std::bad_alloc &) {
        spmv::set_error("out of host memory");
        return SPMV_E_NOMEM;
    } catch (...) {
        spmv::set_error("internal error");
        return SPMV_E_INTERNAL;
    }
}
