// Host emulation of a plan's device image (diagnostics and tests).
//
// spmv_plan_emulate builds the host image of a plan exactly as
// spmv_plan_create does (the same build_host_plan, for a given SM count) and
// evaluates y_hat = A_hat x_hat (Sec. 3) or the split's sum of A^k x_hat
// (Sec. 4) by walking that image the way the kernels do: the staged window
// of each tile, the warp rows, the chunks of 32 rows with their slot
// destinations, the chunk tiles of long rows, the partial slots and the
// fix-ups.  Every index is checked against its array, and every row of y and
// every partial slot must be written exactly once (the device path has no
// clearing pass: a row nobody writes keeps whatever y held).  It needs no
// GPU, so the tiling of full-size matrices in every launch shape can be
// checked on the host; sums run in FP64 in the order the image stores them.
#include <cmath>
#include <limits>
#include <new>
#include <vector>

#include "spmv_internal.h"

using namespace spmv;

namespace {

struct Emu {
    const HostPlan &P;
    const int32_t r;
    std::vector<double> xh;          // x_hat, n x r
    std::vector<double> yh;          // y_hat, m x r
    std::vector<uint8_t> y_done;
    std::vector<double> partial;     // partial_slots x r
    std::vector<uint8_t> p_done;
    std::vector<double> win;         // a tile's staged window, entries x r
    int32_t n_win = 0;

    explicit Emu(const HostPlan &p) : P(p), r(p.nrhs) {}

    bool fail(const char *what, long long a, long long b)
    {
        set_error("plan image check: %s (%lld, %lld)", what, a, b);
        return false;
    }

    // x row of element e of a tile of the given kind, into o[r]
    bool xrow(int32_t kind, int64_t e, double *o)
    {
        if (kind == TILE_NARROW) {
            if (e < 0 || e >= (int64_t)P.col16.size()) return fail("col16 element", e, 0);
            const int32_t c = P.col16[(size_t)e];
            if (c >= n_win) return fail("narrow index beyond the staged window", c, n_win);
            for (int32_t k = 0; k < r; ++k) o[k] = win[(size_t)c * r + k];
            return true;
        }
        if (e < 0 || e >= (int64_t)P.col32.size()) return fail("col32 element", e, 0);
        const int32_t c = P.col32[(size_t)e];
        if (kind == TILE_MIXED && c >= 0) {
            if (c >= n_win) return fail("mixed index beyond the staged window", c, n_win);
            for (int32_t k = 0; k < r; ++k) o[k] = win[(size_t)c * r + k];
            return true;
        }
        const int64_t g = (kind == TILE_MIXED) ? (int64_t)~c : (int64_t)c;
        if (g < 0 || g >= P.n) return fail("x index", g, P.n);
        for (int32_t k = 0; k < r; ++k) o[k] = xh[(size_t)g * r + k];
        return true;
    }

    bool store(int32_t dst, const double *s)
    {
        if (dst == -1) return true;
        if (dst >= 0) {
            if (dst >= P.m) return fail("y row", dst, P.m);
            if (y_done[(size_t)dst]) return fail("y row written twice", dst, 0);
            y_done[(size_t)dst] = 1;
            for (int32_t k = 0; k < r; ++k) yh[(size_t)dst * r + k] = s[k];
            return true;
        }
        const int64_t slot = (int64_t)(-dst) - 2;
        if (slot < 0 || slot >= P.partial_slots) return fail("partial slot", slot, 0);
        if (p_done[(size_t)slot]) return fail("partial slot written twice", slot, 0);
        p_done[(size_t)slot] = 1;
        for (int32_t k = 0; k < r; ++k) partial[(size_t)slot * r + k] = s[k];
        return true;
    }

    // sum of val[e] * x(e) over the given elements, into s[r]
    template <class Elements>
    bool row_sum(int32_t kind, Elements elems, int32_t len, double *s)
    {
        std::vector<double> o((size_t)r);
        for (int32_t k = 0; k < r; ++k) s[k] = 0.0;
        for (int32_t j = 0; j < len; ++j) {
            const int64_t e = elems(j);
            if (e < 0 || e >= (int64_t)P.val.size()) return fail("value element", e, 0);
            if (!xrow(kind, e, o.data())) return false;
            for (int32_t k = 0; k < r; ++k) s[k] += P.val[(size_t)e] * o[k];
        }
        return true;
    }
};

bool run_plain(Emu &E)
{
    const HostPlan &P = E.P;
    if ((int64_t)P.rowptr.size() != (int64_t)P.m + 1)
        return E.fail("rowptr size", (long long)P.rowptr.size(), P.m);
    std::vector<double> s((size_t)E.r);
    for (int32_t i = 0; i < P.m; ++i) {
        const int32_t a = P.rowptr[(size_t)i], b = P.rowptr[(size_t)i + 1];
        if (a > b) return E.fail("rowptr not monotone", i, a);
        if (!E.row_sum(TILE_GLOBAL, [a](int32_t j) { return (int64_t)a + j; }, b - a, s.data()))
            return false;
        if (!E.store(i, s.data())) return false;
    }
    return true;
}

// A chunk of column increments (DELTA tiles), as the kernel reads it: lane
// i's running column starts at the base B and adds the increment of every
// element slot up to the chunk's longest row L, padding included; the kernel
// gathers x at every such column, so each must lie in [0, n).  Padding adds
// 0, so a lane's column stays at its row's last one.
bool run_delta_chunk(Emu &E, int64_t off, int32_t L, int32_t B, int64_t ch)
{
    const HostPlan &P = E.P;
    const int32_t r = E.r;
    if (off & 1) return E.fail("increment chunk at an odd element", ch, off);
    if (off + 32 * (int64_t)L > (int64_t)P.col16.size())
        return E.fail("increment chunk storage", ch, off);
    std::vector<double> s((size_t)r);
    for (int32_t i = 0; i < 32; ++i) {
        const int32_t len = P.slot_len[(size_t)ch * 32 + i];
        const int32_t dst = P.slot_dst[(size_t)ch * 32 + i];
        if (len < 0 || len > L) return E.fail("chunk rows not sorted by length", ch, i);
        if (dst == -1 && len != 0) return E.fail("empty slot with elements", ch, i);
        int64_t c = B;
        for (int32_t k = 0; k < r; ++k) s[k] = 0.0;
        for (int32_t k = 0; k < L; ++k) {
            const uint16_t d = P.col16[(size_t)delta_pos(off, L, k, i)];
            if (k >= len && d != 0) return E.fail("padding increment is not 0", ch, k);
            c += d;
            if (c >= P.n) return E.fail("running column beyond n", ch, c);
            if (k >= len) continue;
            const int64_t e = off + 32 * (int64_t)k + i;
            for (int32_t q = 0; q < r; ++q) s[q] += P.val[(size_t)e] * E.xh[(size_t)c * r + q];
        }
        if (!E.store(dst, s.data())) return false;
    }
    return true;
}

bool run_tile(Emu &E, const Tile &t)
{
    const HostPlan &P = E.P;
    const int32_t r = E.r;
    std::vector<double> s((size_t)r);
    if (t.kind == TILE_CHUNK) {
        if (t.e0 > t.e1) return E.fail("chunk tile range", t.e0, t.e1);
        if (!E.row_sum(TILE_GLOBAL, [&t](int32_t j) { return (int64_t)t.e0 + j; }, t.e1 - t.e0,
                       s.data()))
            return false;
        return E.store(dst_partial(t.slot), s.data());
    }
    if (t.kind != TILE_NARROW && t.kind != TILE_MIXED && t.kind != TILE_GLOBAL &&
        t.kind != TILE_DELTA)
        return E.fail("tile kind", t.kind, 0);
    // the staged window: the first run, the second run (at run2_at), then
    // the gathered list
    if (t.runlen < 0 || t.run2len < 0 || t.listlen < 0)
        return E.fail("window lengths", t.runlen, t.listlen);
    if (t.run2_at < t.runlen) return E.fail("second run overlaps the first", t.run2_at, t.runlen);
    E.n_win = t.run2_at + t.run2len + t.listlen;
    if (t.kind == TILE_NARROW && E.n_win > 65536) return E.fail("narrow window", E.n_win, 0);
    // the device's preconditions: the window fits the dynamic shared memory
    // the launch reserves (max_staged entries); each run's bulk copy starts
    // on a 16-byte boundary of x_hat and of shared memory
    if (E.n_win > P.max_staged) return E.fail("window beyond the reserved shared memory",
                                              E.n_win, P.max_staged);
    {
        const int64_t xb = P.dtype == SPMV_F64 ? 8 : 4;
        const int64_t body1 = ((int64_t)t.runlen * r * xb) & ~(int64_t)15;
        const int64_t body2 = ((int64_t)t.run2len * r * xb) & ~(int64_t)15;
        if (body1 > 0 && ((int64_t)t.run0 * r * xb) % 16 != 0)
            return E.fail("bulk copy source not 16-byte aligned", t.run0, r);
        if (body2 > 0 && (((int64_t)t.run2_0 * r * xb) % 16 != 0 ||
                          ((int64_t)t.run2_at * r * xb) % 16 != 0))
            return E.fail("second bulk copy not 16-byte aligned", t.run2_0, t.run2_at);
        if ((int64_t)P.max_staged * r * xb > 227 * 1024)
            return E.fail("reserved shared memory beyond 227 KB", P.max_staged, r);
    }
    E.win.assign((size_t)E.n_win * r, 0.0);
    for (int32_t i = 0; i < t.runlen; ++i) {
        const int64_t g = (int64_t)t.run0 + i;
        if (g < 0 || g >= P.n) return E.fail("staged run", g, P.n);
        for (int32_t k = 0; k < r; ++k) E.win[(size_t)i * r + k] = E.xh[(size_t)g * r + k];
    }
    for (int32_t i = 0; i < t.run2len; ++i) {
        const int64_t g = (int64_t)t.run2_0 + i;
        if (g < 0 || g >= P.n) return E.fail("second staged run", g, P.n);
        for (int32_t k = 0; k < r; ++k)
            E.win[(size_t)(t.run2_at + i) * r + k] = E.xh[(size_t)g * r + k];
    }
    const int32_t lat = t.run2_at + t.run2len;
    for (int32_t i = 0; i < t.listlen; ++i) {
        const int64_t q = (int64_t)t.list0 + i;
        if (q < 0 || q >= (int64_t)P.xlist.size()) return E.fail("staging list", q, 0);
        const int32_t g = P.xlist[(size_t)q];
        if (g < 0 || g >= P.n) return E.fail("staged list entry", g, P.n);
        for (int32_t k = 0; k < r; ++k)
            E.win[(size_t)(lat + i) * r + k] = E.xh[(size_t)g * r + k];
    }
    if ((t.kind == TILE_GLOBAL || t.kind == TILE_DELTA) && E.n_win != 0)
        return E.fail("unstaged tile stages", E.n_win, 0);
    // warp rows and col32 chunks of a DELTA tile read x as a GLOBAL tile does
    const int32_t kind32 = t.kind == TILE_DELTA ? TILE_GLOBAL : t.kind;
    // rows reduced by a warp
    for (int32_t w = 0; w < t.nvrows; ++w) {
        const int64_t vi = (int64_t)t.vrow0 + w;
        if (vi < 0 || vi >= (int64_t)P.vrows.size()) return E.fail("warp row", vi, 0);
        const VRow v = P.vrows[(size_t)vi];
        if (v.len < 0) return E.fail("warp row length", vi, v.len);
        if (!E.row_sum(kind32, [&v](int32_t j) { return (int64_t)v.e0 + j; }, v.len, s.data()))
            return false;
        if (!E.store(v.dst, s.data())) return false;
    }
    // chunks of 32 rows, one lane per row, element k of lane i at off + 32 k + i
    for (int32_t c = 0; c < t.nchunks; ++c) {
        const int64_t ch = (int64_t)t.chunk0 + c;
        if (ch < 0 || ch >= (int64_t)P.chunk_off.size() ||
            (ch + 1) * 32 > (int64_t)P.slot_len.size() ||
            (ch + 1) * 32 > (int64_t)P.slot_dst.size())
            return E.fail("chunk", ch, 0);
        const int64_t off = P.chunk_off[(size_t)ch];
        const int32_t longest = P.slot_len[(size_t)ch * 32];
        // the kernel reads every lane up to the longest row (padding included)
        if (off < 0 || off + 32 * (int64_t)longest > (int64_t)P.val.size())
            return E.fail("chunk storage", ch, off);
        if (ch >= (int64_t)P.chunk_mix.size()) return E.fail("chunk mix prefix", ch, 0);
        const int32_t G = P.chunk_mix[(size_t)ch];
        if (t.kind == TILE_DELTA) {
            if (G < -1 || G >= P.n) return E.fail("chunk base column", ch, G);
            if (G >= 0 && !run_delta_chunk(E, off, longest, G, ch)) return false;
            if (G >= 0) continue;
        } else if (G < 0 || G > longest || (t.kind != TILE_MIXED && G != 0)) {
            return E.fail("chunk mix prefix", ch, G);
        }
        if (t.kind == TILE_MIXED) {
            // from slot G on the kernel reads shared memory only: every
            // stored element there (padding included) must be a staged index
            for (int64_t k = G; k < longest; ++k)
                for (int32_t i = 0; i < 32; ++i) {
                    const int32_t c = P.col32[(size_t)(off + 32 * k + i)];
                    if (c < 0 || c >= E.n_win)
                        return E.fail("element past the mix prefix is not staged", ch, k);
                }
        }
        for (int32_t i = 0; i < 32; ++i) {
            const int32_t len = P.slot_len[(size_t)ch * 32 + i];
            const int32_t dst = P.slot_dst[(size_t)ch * 32 + i];
            if (len < 0 || len > longest) return E.fail("chunk rows not sorted by length", ch, i);
            if (dst == -1 && len != 0) return E.fail("empty slot with elements", ch, i);
            if (!E.row_sum(kind32, [off, i](int32_t k) { return off + 32 * (int64_t)k + i; },
                           len, s.data()))
                return false;
            if (!E.store(dst, s.data())) return false;
        }
    }
    return true;
}

bool run_fixups(Emu &E)
{
    const HostPlan &P = E.P;
    for (const Fixup &f : P.fixups) {
        if (f.count < 0 || f.slot0 < 0 || (int64_t)f.slot0 + f.count > P.partial_slots)
            return E.fail("fix-up slots", f.slot0, f.count);
        std::vector<double> s((size_t)E.r, 0.0);
        for (int32_t t = 0; t < f.count; ++t) {
            const size_t slot = (size_t)f.slot0 + t;
            if (!E.p_done[slot])
                return E.fail("fix-up reads an unwritten slot", (long long)slot, f.row);
            for (int32_t k = 0; k < E.r; ++k) s[k] += E.partial[slot * E.r + k];
        }
        if (!E.store(f.row, s.data())) return false;
    }
    for (int64_t q = 0; q < P.partial_slots; ++q)
        if (!E.p_done[(size_t)q]) return E.fail("partial slot never written", q, 0);
    return true;
}

}  // namespace

extern "C" spmv_status spmv_plan_emulate(const spmv_csr *A, const spmv_perm *perm,
                                         const spmv_splits *splits, const spmv_opts *opts,
                                         int32_t n_sm, const double *x, double *y,
                                         int64_t *stats)
{
    clear_error();
    if (!A || (!x && A->n > 0) || (!y && A->m > 0)) {
        set_error("A, x and y are required");
        return SPMV_E_INVALID;
    }
    try {
        HostPlan P;
        spmv_status st = build_host_plan(A, perm, splits, opts, n_sm, &P);
        if (st != SPMV_OK) return st;
        Emu E(P);
        const int32_t r = P.nrhs;
        E.xh.resize((size_t)P.n * r);
        for (int32_t j = 0; j < P.n; ++j) {
            const int32_t src = P.col_perm.empty() ? j : P.col_perm[(size_t)j];
            for (int32_t k = 0; k < r; ++k) E.xh[(size_t)j * r + k] = x[(size_t)src * r + k];
        }
        E.yh.assign((size_t)P.m * r, std::numeric_limits<double>::quiet_NaN());
        E.y_done.assign((size_t)P.m, 0);
        E.partial.assign((size_t)P.partial_slots * r, 0.0);
        E.p_done.assign((size_t)P.partial_slots, 0);
        bool ok = true;
        if (P.use_k1) {
            ok = run_plain(E);
        } else {
            for (size_t t = 0; ok && t < P.tiles.size(); ++t) ok = run_tile(E, P.tiles[t]);
            ok = ok && run_fixups(E);
        }
        for (int32_t i = 0; ok && i < P.m; ++i)
            if (!E.y_done[(size_t)i]) ok = E.fail("y row never written", i, 0);
        if (!ok) return SPMV_E_INTERNAL;
        for (int32_t i = 0; i < P.m; ++i) {
            const int32_t dst = P.row_perm.empty() ? i : P.row_perm[(size_t)i];
            for (int32_t k = 0; k < r; ++k) y[(size_t)dst * r + k] = E.yh[(size_t)i * r + k];
        }
        if (stats) {
            int32_t nvr = 0;
            int64_t two_runs = 0;
            for (const Tile &t : P.tiles) {
                nvr += t.kind == TILE_CHUNK ? 0 : t.nvrows;
                two_runs += t.kind != TILE_CHUNK && t.run2len > 0;
            }
            const int64_t v[SPMV_EMULATE_STATS] = {
                (int64_t)P.tiles.size(), P.n_chunk_tiles, P.n_staged_tiles, P.partial_slots,
                (int64_t)P.fixups.size(), nvr, P.padded_elems, P.use_k1 ? 1 : 0,
                P.direct_nnz, P.fma_slots, P.mixed_slots, P.staged_entries, two_runs,
                P.delta_nnz};
            for (int k = 0; k < SPMV_EMULATE_STATS; ++k) stats[k] = v[k];
        }
        return SPMV_OK;
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        return SPMV_E_NOMEM;
    }
}
