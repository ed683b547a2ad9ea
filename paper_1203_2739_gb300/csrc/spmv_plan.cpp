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
    int32_t align;      // staged runs start and end on multiples of this (16 bytes)
    int32_t n;          // columns (a run may end at n unaligned)
    int32_t tnnz;       // nonzero budget of a tile
    int32_t long_t;     // rows longer than this become chunks
    int32_t chunk;      // nonzeros per chunk of a long row
    int32_t max_rows;   // rows per tile
    int32_t vrow_len;   // rows longer than this are reduced by a whole warp
    int32_t entry_bytes;  // bytes of one x entry (r values)
    int32_t list_min;   // uses in the tile that put a column outside the run on the list
    bool stage;         // staging allowed
    bool delta;         // chunks of unstaged tiles store column increments
};

// Cuts the plan rows of the parts into tiles of consecutive rows with a
// fixed nonzero budget, and gives each tile the part of the paper's "cache"
// a CTA owns: shared memory for W x entries (Theorem 1 asks that every part
// fit the cache; here the tile stages what fits and gathers the rest).  Two
// staging sets are weighed: (a) the span of home columns the tile uses --
// the C_k of its parts, a contiguous range of x_hat copied in bulk -- plus
// the border columns it uses often (list_min times or more), or (b) the
// columns it uses often, most used first, up to W.  A gathered x entry costs
// one L2 request per use; a staged one costs a 128-byte line per 128 bytes of
// run (one request per list entry) and nothing per use.  The tile takes the
// set that saves more requests, if it saves at least what it costs.  Rows
// are sorted by length into chunks of 32 stored column-major.
struct Tiler {
    const TileCfg cfg;
    const std::vector<int32_t> &prp;   // plan row starts
    const std::vector<int32_t> &col;   // plan-order global columns
    const std::vector<double> &pval;   // plan-order values
    const std::vector<int32_t> &pdst;  // plan row -> slot_dst encoding
    HostPlan &P;
    std::vector<int32_t> mark, cnt, loc;
    int32_t stamp = 0;
    std::vector<int32_t> used;
    std::vector<int32_t> order;

    Tiler(const TileCfg &c, const std::vector<int32_t> &rp, const std::vector<int32_t> &cl,
          const std::vector<double> &pv, const std::vector<int32_t> &pd, HostPlan &plan,
          int32_t n)
        : cfg(c), prp(rp), col(cl), pval(pv), pdst(pd), P(plan), mark((size_t)n, -1),
          cnt((size_t)n, 0), loc((size_t)n, 0) {}

    // the aligned run covering columns [lo, hi]
    void aligned_run(int32_t lo, int32_t hi, int32_t *run0, int32_t *runlen) const
    {
        const int32_t a = cfg.align;
        const int32_t b = lo - lo % a;
        int64_t e = (int64_t)hi + 1;
        e = std::min<int64_t>(cfg.n, (e + a - 1) / a * a);
        *run0 = b;
        *runlen = (int32_t)(e - b);
    }

    // The contiguous range of x_hat of at most `span` columns that maximises
    // (uses covered) - lam * (columns spanned), over the tile's columns cs
    // (ascending), skipping columns in [skip0, skip1): a staged entry costs
    // lam of a gathered use (its bytes copied in bulk against the 32-byte
    // sector a gather fetches).  Returns the uses covered (0 if no range
    // scores above 0) and the first / last column.
    int64_t best_window(const std::vector<int32_t> &cs, int32_t span, double lam,
                        int32_t skip0, int32_t skip1, int32_t *lo, int32_t *hi) const
    {
        *lo = 0;
        *hi = -1;
        if (span <= 0 || cs.empty()) return 0;
        // score(i..j) = P[j+1] - P[i] - lam (c_j - c_i + 1); for each j the
        // best i within the span maximises lam c_i - P[i] (a monotone deque)
        const size_t n = cs.size();
        std::vector<double> P(n + 1, 0.0);
        for (size_t j = 0; j < n; ++j) P[j + 1] = P[j] + cnt[cs[j]];
        std::vector<size_t> dq(n);
        size_t qh = 0, qt = 0;
        double best = 0.0;
        int64_t best_uses = 0;
        auto key = [&](size_t i) { return lam * cs[i] - P[i]; };
        for (size_t j = 0; j < n; ++j) {
            const int32_t c = cs[j];
            if (c >= skip0 && c < skip1) {
                qh = qt = 0;            // a range may not straddle the skipped one
                continue;
            }
            while (qt > qh && key(dq[qt - 1]) <= key(j)) --qt;
            dq[qt++] = j;
            while ((int64_t)c - cs[dq[qh]] + 1 > span) ++qh;
            const size_t i = dq[qh];
            const double sc = P[j + 1] - P[i] - lam * ((double)c - cs[i] + 1);
            if (sc > best) {
                best = sc;
                *lo = cs[i];
                *hi = c;
                best_uses = (int64_t)(P[j + 1] - P[i]);
            }
        }
        return best_uses;
    }

    // A staging set: up to two runs and a list, the uses it covers (x
    // gathers it saves) and its cost in gathers: a run entry costs its bytes
    // over a 32-byte sector (what a gather of it would fetch), a list entry a
    // gather.
    struct Stage {
        int32_t run0 = 0, runlen = 0, run2_0 = 0, run2len = 0, run2_at = 0;
        std::vector<int32_t> list;
        int64_t saved = 0;
        double cost = 0.0;
        double gain() const { return (double)saved - cost; }
        int32_t entries() const { return run2_at + run2len + (int32_t)list.size(); }
    };

    double lam() const { return std::min(1.0, cfg.entry_bytes / 32.0); }

    bool in_runs(const Stage &g, int32_t c) const
    {
        return (c >= g.run0 && c < g.run0 + g.runlen) ||
               (c >= g.run2_0 && c < g.run2_0 + g.run2len);
    }

    // Complete a set whose runs are chosen: uses covered by the runs, then
    // the most used of the other columns (list_min uses or more) on the list
    // while capacity lasts.
    void finish_stage(Stage &g, const std::vector<int32_t> &cs) const
    {
        std::vector<int32_t> rest;
        g.saved = 0;
        for (int32_t c : cs) {
            if (in_runs(g, c)) g.saved += cnt[c];
            else if (cnt[c] >= cfg.list_min) rest.push_back(c);
        }
        g.run2_at = g.run2len > 0 ? (g.runlen + cfg.align - 1) / cfg.align * cfg.align
                                  : g.runlen;
        const int64_t room = (int64_t)cfg.W - g.run2_at - g.run2len;
        if ((int64_t)rest.size() > room) {
            const size_t keep = (size_t)std::max<int64_t>(room, 0);
            std::nth_element(rest.begin(), rest.begin() + keep, rest.end(),
                             [&](int32_t x, int32_t y) {
                                 return cnt[x] != cnt[y] ? cnt[x] > cnt[y] : x < y;
                             });
            rest.resize(keep);
        }
        std::sort(rest.begin(), rest.end());
        for (int32_t c : rest) g.saved += cnt[c];
        g.list.swap(rest);
        g.cost = (double)(g.runlen + g.run2len) * lam() + (double)g.list.size();
    }

    // Close the tile made of plan rows `rows`; its columns carry mark == stamp
    // and their use counts in cnt.
    void emit(const std::vector<int32_t> &rows, int64_t tile_nnz, int32_t h0, int32_t h1,
              bool force_global)
    {
        if (rows.empty()) return;
        Tile t{};
        t.kind = TILE_GLOBAL;
        if (cfg.stage && !force_global && tile_nnz > 0) {
            std::vector<int32_t> cs(used);
            std::sort(cs.begin(), cs.end());
            const int32_t slack = 2 * (cfg.align - 1);
            std::vector<Stage> cand;
            // (a) the span of home columns the tile uses (the C_k of its
            // parts, consecutive in x_hat) when it fits, plus the list
            {
                int32_t lo = INT32_MAX, hi = -1;
                for (int32_t c : cs)
                    if (c >= h0 && c < h1) {
                        lo = std::min(lo, c);
                        hi = std::max(hi, c);
                    }
                Stage g;
                if (hi >= 0) aligned_run(lo, hi, &g.run0, &g.runlen);
                if (g.runlen <= cfg.W) {
                    finish_stage(g, cs);
                    if (g.entries() <= cfg.W) cand.push_back(std::move(g));
                }
            }
            // (b) the list alone: the most used columns
            {
                Stage g;
                finish_stage(g, cs);
                cand.push_back(std::move(g));
            }
            // (c) the densest window of x_hat, then the densest window of
            // what is left, then the list
            {
                Stage g;
                int32_t lo, hi;
                if (best_window(cs, cfg.W - slack, lam(), 0, 0, &lo, &hi) > 0) {
                    aligned_run(lo, hi, &g.run0, &g.runlen);
                    if (best_window(cs, cfg.W - g.runlen - cfg.align - slack, lam(), g.run0,
                                    g.run0 + g.runlen, &lo, &hi) > 0)
                        aligned_run(lo, hi, &g.run2_0, &g.run2len);
                    // aligned runs may touch; they never overlap (the second
                    // avoids the first's columns, and alignment rounds both
                    // outward only to the same boundaries)
                    if (g.run2len > 0 && g.run2_0 < g.run0 + g.runlen &&
                        g.run0 < g.run2_0 + g.run2len) {
                        g.run2_0 = g.run2len = 0;
                    }
                    finish_stage(g, cs);
                    if (g.entries() <= cfg.W) cand.push_back(std::move(g));
                }
            }
            const Stage *best = nullptr;
            for (const Stage &g : cand)
                if (g.entries() <= cfg.W && (!best || g.gain() > best->gain())) best = &g;
            // stage when it saves at least as many gathers as it costs (a
            // staged entry is fetched before the tile's rows start, where its
            // latency is not hidden) and covers a quarter of the tile's
            // uses: a tile that stages and still gathers issues a shared-
            // memory load beside the gather in the slots that gather
            if (best && best->gain() > 0.0 && best->gain() >= best->cost &&
                4 * best->saved >= tile_nnz) {
                const Stage &g = *best;
                int32_t listlen = 0;
                int64_t direct = 0;
                t.list0 = (int32_t)P.xlist.size();
                for (int32_t c : cs) {
                    if (c >= g.run0 && c < g.run0 + g.runlen) loc[c] = c - g.run0;
                    else if (c >= g.run2_0 && c < g.run2_0 + g.run2len)
                        loc[c] = g.run2_at + (c - g.run2_0);
                    else loc[c] = -1;
                }
                for (int32_t c : g.list) {
                    loc[c] = g.run2_at + g.run2len + listlen++;
                    P.xlist.push_back(c);
                }
                for (int32_t c : cs)
                    if (loc[c] < 0) direct += cnt[c];
                t.kind = direct == 0 ? TILE_NARROW : TILE_MIXED;
                t.run0 = g.run0;
                t.runlen = g.runlen;
                t.run2_0 = g.run2_0;
                t.run2len = g.run2len;
                t.run2_at = g.run2_at;
                t.listlen = listlen;
                const int32_t staged = g.entries();
                P.max_staged = std::max(P.max_staged, staged);
                P.staged_entries += staged;
                P.list_entries += listlen;
                P.direct_nnz += direct;
                if (t.kind == TILE_NARROW) P.narrow_nnz += tile_nnz;
                P.n_staged_tiles++;
            }
        }
        if (t.kind == TILE_GLOBAL) {
            P.n_global_tiles++;
            P.direct_nnz += tile_nnz;
        }
        // rows longer than cfg.vrow_len are reduced by a whole warp; the rest
        // go by decreasing length (stable) into chunks of 32, column-major
        auto put = [&](size_t e, int32_t q) {
            const int32_t cg = col[q];
            P.val[e] = pval[q];
            if (t.kind == TILE_NARROW) P.col16[e] = (uint16_t)loc[cg];
            else if (t.kind == TILE_MIXED) P.col32[e] = loc[cg] >= 0 ? loc[cg] : ~cg;
            else P.col32[e] = cg;
        };
        order.clear();
        t.vrow0 = (int32_t)P.vrows.size();
        // the warp rows longest first: the warps take them round-robin, so
        // this keeps the warps of the CTA about equally busy
        std::vector<int32_t> wide_rows;
        for (int32_t r : rows) {
            if (prp[r + 1] - prp[r] <= cfg.vrow_len) order.push_back(r);
            else wide_rows.push_back(r);
        }
        std::stable_sort(wide_rows.begin(), wide_rows.end(), [&](int32_t a, int32_t b) {
            return prp[a + 1] - prp[a] > prp[b + 1] - prp[b];
        });
        for (int32_t r : wide_rows) {
            const int32_t a = prp[r], len = prp[r + 1] - a;
            const size_t e0 = P.val.size();
            P.val.resize(e0 + len, 0.0);
            P.col32.resize(e0 + len, 0);
            P.col16.resize(e0 + len, 0);
            for (int32_t k = 0; k < len; ++k) put(e0 + k, a + k);
            P.vrows.push_back(VRow{(int32_t)e0, len, pdst[r], 0});
            P.padded_elems += len;
            P.fma_slots += ((len + 31) / 32) * 32;
        }
        t.nvrows = (int32_t)P.vrows.size() - t.vrow0;
        // chunk rows by decreasing length; in MIXED tiles rows of equal
        // length by decreasing count of gathered elements, so that the rows
        // that gather share chunks and the others' chunks read shared memory
        // only
        std::vector<int32_t> ng;
        if (t.kind == TILE_MIXED) {
            ng.assign(order.size(), 0);
            for (size_t k = 0; k < order.size(); ++k)
                for (int32_t q = prp[order[k]]; q < prp[order[k] + 1]; ++q)
                    ng[k] += loc[col[q]] < 0;
            std::vector<int32_t> idx(order.size());
            std::iota(idx.begin(), idx.end(), 0);
            std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
                const int32_t la = prp[order[a] + 1] - prp[order[a]];
                const int32_t lb = prp[order[b] + 1] - prp[order[b]];
                return la != lb ? la > lb : ng[a] > ng[b];
            });
            std::vector<int32_t> o2(order.size());
            for (size_t k = 0; k < idx.size(); ++k) o2[k] = order[idx[k]];
            order.swap(o2);
        } else {
            std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
                return prp[a + 1] - prp[a] > prp[b + 1] - prp[b];
            });
        }
        t.chunk0 = (int32_t)P.chunk_off.size();
        const int32_t nrows = (int32_t)order.size();
        t.nchunks = (nrows + 31) / 32;
        std::vector<int32_t> seq;
        const bool delta = cfg.delta && t.kind == TILE_GLOBAL;
        int32_t n_delta = 0;
        for (int32_t c = 0; c < t.nchunks; ++c) {
            const int32_t first = c * 32;
            const int32_t L = prp[order[first] + 1] - prp[order[first]];
            if (delta && (P.val.size() & 1)) {
                // increments are read in 32-bit pairs: the chunk starts on
                // an even element
                P.val.push_back(0.0);
                P.col32.push_back(0);
                P.col16.push_back(0);
            }
            const size_t off = P.val.size();
            P.chunk_off.push_back((int32_t)off);
            P.val.resize(off + (size_t)L * 32, 0.0);
            P.col32.resize(off + (size_t)L * 32, 0);
            P.col16.resize(off + (size_t)L * 32, 0);
            P.padded_elems += (int64_t)L * 32;
            P.fma_slots += (int64_t)L * 32;
            int32_t G = 0;
            for (int32_t i = 0; i < 32; ++i) {
                const int32_t idx = first + i;
                if (idx >= nrows) {
                    P.slot_dst.push_back(-1);
                    P.slot_len.push_back(0);
                    continue;
                }
                const int32_t r = order[idx];
                const int32_t a = prp[r], len = prp[r + 1] - a;
                P.slot_dst.push_back(pdst[r]);
                P.slot_len.push_back(len);
                // in MIXED tiles a row stores its gathered elements first, so
                // that from slot G on (G = the most any row of the chunk
                // gathers) every lane reads shared memory only
                seq.clear();
                if (t.kind == TILE_MIXED) {
                    for (int32_t k = 0; k < len; ++k)
                        if (loc[col[a + k]] < 0) seq.push_back(a + k);
                    G = std::max(G, (int32_t)seq.size());
                    for (int32_t k = 0; k < len; ++k)
                        if (loc[col[a + k]] >= 0) seq.push_back(a + k);
                } else {
                    for (int32_t k = 0; k < len; ++k) seq.push_back(a + k);
                }
                for (int32_t k = 0; k < len; ++k) put(off + (size_t)k * 32 + i, seq[k]);
            }
            if (delta) {
                // base column: the smallest first column of the chunk's
                // rows; every increment (from the base to a row's first
                // column, then between successive columns of the row) must
                // fit 16 bits
                int32_t B = INT32_MAX;
                bool fits = true;
                for (int32_t i = 0; i < 32 && first + i < nrows; ++i) {
                    const int32_t r = order[first + i];
                    if (prp[r + 1] > prp[r]) B = std::min(B, col[prp[r]]);
                }
                if (B == INT32_MAX) B = 0;
                for (int32_t i = 0; i < 32 && first + i < nrows && fits; ++i) {
                    const int32_t r = order[first + i];
                    int32_t prev = B;
                    for (int32_t q = prp[r]; q < prp[r + 1]; ++q) {
                        const int64_t d = (int64_t)col[q] - prev;
                        if (d < 0 || d > 65535) {
                            fits = false;
                            break;
                        }
                        prev = col[q];
                    }
                }
                if (fits) {
                    for (int32_t i = 0; i < 32 && first + i < nrows; ++i) {
                        const int32_t r = order[first + i];
                        int32_t prev = B;
                        for (int32_t k = 0; k < prp[r + 1] - prp[r]; ++k) {
                            const int32_t cg = col[prp[r] + k];
                            P.col16[(size_t)delta_pos((int64_t)off, L, k, i)] =
                                (uint16_t)(cg - prev);
                            prev = cg;
                        }
                        P.delta_nnz += prp[r + 1] - prp[r];
                    }
                    ++n_delta;
                }
                G = fits ? B : -1;
            }
            P.chunk_mix.push_back(G);
            if (!delta) P.mixed_slots += (int64_t)G * 32;
        }
        if (delta && n_delta > 0) {
            t.kind = TILE_DELTA;
        } else if (delta) {
            // no chunk fits: a plain GLOBAL tile
            std::fill(P.chunk_mix.begin() + t.chunk0, P.chunk_mix.end(), 0);
        }
        P.tiles.push_back(t);
    }

    // Tile plan rows [rb, re) of one part (or consecutive parts) with home
    // columns [h0, h1): consecutive rows up to the nonzero budget; emit()
    // then stages what fits the capacity.  chunked[r] marks rows handled as
    // chunks (left out of the tiles).
    void tile_rows(int32_t rb, int32_t re, int32_t h0, int32_t h1,
                   const std::vector<char> &chunked, bool force_global)
    {
        const int32_t limit = cfg.tnnz;
        int64_t cur_nnz = 0;
        std::vector<int32_t> rows;
        auto close = [&]() {
            emit(rows, cur_nnz, h0, h1, force_global);
            rows.clear();
            cur_nnz = 0;
            used.clear();
            ++stamp;
        };
        for (int32_t r = rb; r < re; ++r) {
            if (chunked[r]) continue;
            const int32_t a = prp[r], b = prp[r + 1], len = b - a;
            // fill to the budget: the row goes to the next tile when it would
            // take this one more than half its length past it
            if (!rows.empty() &&
                ((int32_t)rows.size() >= cfg.max_rows || cur_nnz + len / 2 > limit))
                close();
            rows.push_back(r);
            for (int32_t q = a; q < b; ++q) {
                const int32_t c = col[q];
                if (mark[c] != stamp) {
                    mark[c] = stamp;
                    cnt[c] = 1;
                    used.push_back(c);
                } else {
                    ++cnt[c];
                }
            }
            cur_nnz += len;
        }
        close();
    }
};

int32_t pow2_at_least(double want, int32_t lo)
{
    int32_t l = lo;
    while (l < 32 && l < want) l *= 2;
    return l;
}

}  // namespace

// --------------------------------------------------------------- the plan --
spmv_status build_host_plan(const spmv_csr *A, const spmv_perm *perm,
                            const spmv_splits *splits, const spmv_opts *opts,
                            int32_t n_sm, HostPlan *P)
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
    if (o.warp_rows < 0) {
        set_error("warp_rows=%d must be >= 0", o.warp_rows);
        return SPMV_E_INVALID;
    }
    if (o.lanes != 0 && o.lanes != 1 && o.lanes != 2 && o.lanes != 4 && o.lanes != 8 &&
        o.lanes != 16 && o.lanes != 32) {
        set_error("lanes=%d: must be 0, 1, 2, 4, 8, 16 or 32", o.lanes);
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
    const int r = o.nrhs;
    // CTA shape: 6 CTAs of 256 threads per SM (fewer for 4 or 8 right-hand
    // sides), each staging up to 36 KB of x (they fit an SM's 228 KB next to some L1), or one wide
    // CTA of 1024 threads per SM staging up to 200 KB
    if (o.cta_threads != 0 && o.cta_threads != 256 && o.cta_threads != 512 &&
        o.cta_threads != 1024) {
        set_error("cta_threads=%d: must be 0, 256, 512 or 1024", o.cta_threads);
        return SPMV_E_INVALID;
    }
    const bool wide = o.cta_threads == 1024, mid = o.cta_threads == 512;
    if ((wide || mid) && (o.flags & (SPMV_FLAG_SM_AFFINE | SPMV_FLAG_PERSISTENT))) {
        set_error("cta_threads=%d runs one CTA per tile (no persistent or SM-affine launch)",
                  o.cta_threads);
        return SPMV_E_INVALID;
    }
    // tiles per SM of a launch: one wave of the 256-thread CTAs, two waves
    // of the 512-thread CTAs (two per SM) and of the wide ones (one per SM).
    // Windows: 96 KB for the wide CTAs and 48 KB for each 512-thread CTA,
    // which leaves L1 about 128 KB for the entries gathered and for the
    // matrix stream in flight (measured on GB300: the blocks matrix in SB
    // form, one wide CTA per SM, 126.9 us with 128 KB windows, 122.6 us with
    // 96 KB windows in twice larger tiles, 198.6 us with 200 KB windows)
    const int32_t ctas_per_sm = wide ? 2 : (mid ? 4 : tile_ctas_per_sm_for(r));
    int32_t W = o.tile_cols > 0
                    ? o.tile_cols
                    : std::min<int32_t>(65535, ((wide ? 96 : (mid ? 48 : 36)) * 1024) / (xb * r));
    if ((int64_t)W * xb * r > 220 * 1024 || W > 65535) {
        set_error("tile_cols=%d does not fit shared memory (x entries of %d bytes, r=%d)", W,
                  xb, r);
        return SPMV_E_UNSUPPORTED;
    }
    P->m = m;
    P->n = n;
    P->nnz = nnz;
    P->form = form;
    P->dtype = o.dtype;
    P->nrhs = r;
    if (o.flags & ~(SPMV_FLAG_NO_STAGING | SPMV_FLAG_TILED_NATURAL | SPMV_FLAG_SM_AFFINE |
                    SPMV_FLAG_PERSISTENT | SPMV_FLAG_STAGE | SPMV_FLAG_TEST_WAIT_EXPIRES |
                    SPMV_FLAG_COL_DELTA)) {
        set_error("unknown flag bits 0x%x", o.flags);
        return SPMV_E_INVALID;
    }
    if ((o.flags & SPMV_FLAG_SM_AFFINE) && (o.flags & SPMV_FLAG_PERSISTENT)) {
        set_error("SPMV_FLAG_SM_AFFINE and SPMV_FLAG_PERSISTENT exclude each other");
        return SPMV_E_INVALID;
    }
    P->flags = o.flags;
    P->cta_threads = o.cta_threads == 1024 ? 1024 : (o.cta_threads == 512 ? 512 : 256);
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
        P->lanes = o.lanes ? o.lanes : pow2_at_least(mean_len / 6.0, 2);
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

    TileCfg cfg;
    cfg.W = W;
    cfg.n = n;
    cfg.entry_bytes = xb * r;
    cfg.align = std::max(1, 16 / (xb * r));
    cfg.list_min = 3;
    cfg.max_rows = 4096;
    cfg.vrow_len = o.warp_rows > 0 ? o.warp_rows : 64;
    // tiles sized so that one launch is about one wave of resident CTAs
    // (ctas_per_sm per SM): every CTA starts at once and none waits for
    // a slot, so there is no tail wave.  Rows longer than long_t are cut into
    // chunk tiles (at least 4096 nonzeros); the fix-up kernel adds their
    // pieces.
    {
        const int64_t slots = (int64_t)(n_sm > 0 ? n_sm : 152) * ctas_per_sm;
        const int64_t want = std::max<int64_t>((nnz + slots - 1) / slots, 1024);
        cfg.tnnz = o.tile_nnz > 0 ? o.tile_nnz : (int32_t)std::min<int64_t>(want, 1 << 26);
        // chunk tiles of a quarter of a tile's budget, rows over a sixteenth
        // of it cut into them (the rest stay in the tiles, reduced by a warp
        // or a lane): on power-law matrices the small chunks fill the slots
        // the row tiles leave at the end of the wave (R-MAT SB K=1024:
        // 90.8 us against 103.1 us with whole-tile chunks of rows over a
        // quarter)
        cfg.chunk = std::max<int32_t>(4096, cfg.tnnz / 4);
        cfg.long_t = o.long_row > 0 ? o.long_row : std::max<int32_t>(1024, cfg.tnnz / 16);
    }
    cfg.stage = !(o.flags & SPMV_FLAG_NO_STAGING) && (wide || mid || (o.flags & SPMV_FLAG_STAGE));
    cfg.delta = (o.flags & SPMV_FLAG_COL_DELTA) != 0;
    P->lanes = 32;                 // one lane per row, 32 rows per chunk
    P->long_thresh = cfg.long_t;

    // pieces per plan row, slots and fix-ups (split rows shared by several
    // parts and chunked long rows are summed in part / chunk order)
    std::vector<char> chunked((size_t)R, 0), has_chunk((size_t)m, 0);
    std::vector<int32_t> pieces((size_t)R, 1), tot((size_t)m, 0);
    for (int32_t q = 0; q < R; ++q) {
        int32_t len = prp[q + 1] - prp[q];
        if (len > cfg.long_t) {
            chunked[q] = 1;
            has_chunk[prow[q]] = 1;
            pieces[q] = (len + cfg.chunk - 1) / cfg.chunk;
        }
        tot[prow[q]] += pieces[q];
    }
    std::vector<int32_t> base((size_t)m, -1);
    int64_t slots = 0;
    for (int32_t i = 0; i < m; ++i)
        if (tot[i] != 1 || has_chunk[i]) {
            base[i] = (int32_t)slots;
            P->fixups.push_back(Fixup{i, (int32_t)slots, tot[i], 0});
            slots += tot[i];
        }
    if (slots >= INT32_MAX / 2) {
        set_error("too many partial sums");
        return SPMV_E_UNSUPPORTED;
    }
    P->partial_slots = slots;
    std::vector<int32_t> run((size_t)m, 0), pdst((size_t)R, -1);
    std::vector<std::pair<int32_t, int32_t>> chunk_rows;   // (plan row, first slot)
    for (int32_t q = 0; q < R; ++q) {
        int32_t i = prow[q];
        int32_t slot = base[i] >= 0 ? base[i] + run[i] : -1;
        run[i] += pieces[q];
        pdst[q] = (slot >= 0) ? dst_partial(slot) : i;
        if (chunked[q]) chunk_rows.emplace_back(q, slot);
    }
    std::vector<double> pval((size_t)nnz);
    for (int64_t q = 0; q < nnz; ++q) pval[q] = A->vals[psrc[q]];

    Tiler tiler(cfg, prp, pcol, pval, pdst, *P, n);
    // the parts' home columns C_1 .. C_K are consecutive ranges of x_hat, so
    // a tile may run across part boundaries and still stage one contiguous
    // run: the union of the C_k of the parts it covers
    {
        int32_t h0 = 0, h1 = 0;
        if (!cp_part.empty()) {
            h0 = cp_part[0];
            h1 = cp_part[K];
        } else if (form == SPMV_NATURAL) {
            h0 = 0;
            h1 = n;
        }
        tiler.tile_rows(pr_part[0], pr_part[K], h0, h1, chunked, false);
    }
    // DB row border R_B: no home columns (the paper charges every border
    // nonzero a miss, eq. 6); columns it reuses may still be staged
    if (pr_part[K + 1] > pr_part[K])
        tiler.tile_rows(pr_part[K], pr_part[K + 1], 0, 0, chunked, false);

    // long rows: contiguous, global indices, one CTA per chunk of nonzeros;
    // chunk tiles go first so the longest work starts early
    std::vector<Tile> chunk_tiles;
    for (auto &cr : chunk_rows) {
        const int32_t q = cr.first, slot = cr.second;
        const size_t e0 = P->val.size();
        const int32_t a = prp[q], len = prp[q + 1] - a;
        if (e0 + (size_t)len >= (size_t)INT32_MAX) {
            set_error("too many stored elements");
            return SPMV_E_UNSUPPORTED;
        }
        for (int32_t k = 0; k < len; ++k) {
            P->val.push_back(pval[a + k]);
            P->col32.push_back(pcol[a + k]);
            P->col16.push_back(0);
        }
        for (int32_t c = 0; c < pieces[q]; ++c) {
            Tile t{};
            t.kind = TILE_CHUNK;
            t.e0 = (int32_t)e0 + c * cfg.chunk;
            t.e1 = std::min((int32_t)(e0 + len), t.e0 + cfg.chunk);
            t.slot = slot + c;
            chunk_tiles.push_back(t);
        }
    }
    // row tiles first, then the chunk tiles, longest first: the smaller
    // pieces fill the slots that free up last
    P->n_chunk_tiles = (int32_t)chunk_tiles.size();
    std::stable_sort(chunk_tiles.begin(), chunk_tiles.end(),
                     [](const Tile &a, const Tile &b) { return a.e1 - a.e0 > b.e1 - b.e0; });
    P->tiles.insert(P->tiles.end(), chunk_tiles.begin(), chunk_tiles.end());
    if (P->val.size() >= (size_t)INT32_MAX) {
        set_error("too many stored elements");
        return SPMV_E_UNSUPPORTED;
    }
    if (P->narrow_nnz == 0 && P->delta_nnz == 0) {
        P->col16.clear();
        P->col16.shrink_to_fit();
    }

    // coverage: every y row is written exactly once (by a tile slot or a fix-up)
    {
        std::vector<int32_t> cover((size_t)m, 0);
        for (int32_t d : P->slot_dst)
            if (d >= 0) cover[d]++;
        for (const VRow &v : P->vrows)
            if (v.dst >= 0) cover[v.dst]++;
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
        // The border's coupling columns go by the part holding most of their
        // nonzeros (the lower part on ties), then by index: columns used
        // mostly by the same part sit together (Sec. 3 places columns with
        // similar sparsity patterns near each other), so a part's border
        // columns form a few contiguous ranges of x_hat that a tile can
        // stage in bulk.  Untouched columns follow, by index.
        std::vector<int32_t> maj((size_t)n, K);
        {
            std::vector<int64_t> cstart((size_t)n + 1, 0);
            for (int32_t i = 0; i < m; ++i)
                if (labels[i] < K)
                    for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
                        if (multi[A->colidx[p]]) cstart[A->colidx[p] + 1]++;
            for (int32_t c = 0; c < n; ++c) cstart[c + 1] += cstart[c];
            std::vector<int32_t> lab((size_t)cstart[n]);
            std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
            for (int32_t i = 0; i < m; ++i)
                if (labels[i] < K)
                    for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
                        if (multi[A->colidx[p]]) lab[(size_t)fill[A->colidx[p]]++] = labels[i];
            for (int32_t c = 0; c < n; ++c) {
                if (!multi[c]) continue;
                auto a = lab.begin() + cstart[c], b = lab.begin() + cstart[c + 1];
                std::sort(a, b);
                int64_t best = 0;
                for (auto q = a; q != b;) {
                    auto r = q;
                    while (r != b && *r == *q) ++r;
                    if (r - q > best) {
                        best = r - q;
                        maj[c] = *q;
                    }
                    q = r;
                }
            }
        }
        std::vector<int32_t> pos(ccnt.begin(), ccnt.end() - 1);
        for (int32_t c = 0; c < n; ++c)
            if (cls(c) != K) col_perm[pos[cls(c)]++] = c;
        {
            std::vector<int32_t> mc((size_t)K + 1, 0);
            for (int32_t c = 0; c < n; ++c)
                if (cls(c) == K) mc[maj[c] + 1]++;
            for (int32_t k = 0; k < K; ++k) mc[k + 1] += mc[k];
            for (int32_t c = 0; c < n; ++c)
                if (cls(c) == K) col_perm[ccnt[K] + mc[maj[c]]++] = c;
        }
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
