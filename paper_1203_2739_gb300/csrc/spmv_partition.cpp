// Recursive hypergraph bisection for the three models of the paper:
//
//  * column-net (CN, Sec. 3.1): vertices = rows, nets = columns, connectivity
//    metric with cut-net splitting; the bisection tree's leaves are the row
//    parts of the SB form and the cut size plus the number of non-empty
//    columns is the bound of eq. (4);
//  * row-column-net (RCN, Sec. 4.1): vertices = nonzeros, nets = rows and
//    columns, connectivity metric on both -> a split whose cut size plus the
//    number of non-empty rows and columns is the bound of eq. (7);
//  * enhanced row-column-net (eRCN, Sec. 3.2): as RCN, but a row net costs
//    nnz(r_i) under the cut-net metric: when it is cut, the row goes to the
//    row border R_B and its nonzeros are removed from both halves (cut-net
//    removal), while column nets keep cost 1 and are split (cut-net
//    splitting).  The accounting gives eq. (6).
//
// Each bisection is multilevel: heavy-connectivity matching (or a linear
// net-based matching on very large levels), contraction, greedy growing plus
// FM refinement on the coarsest level, and boundary FM while uncoarsening.
// Recursion stops at a fixed depth log2(K), or when a part "fits" (Sec. 5.1):
// its CSR storage with its x and y subvectors (or, for the GPU adaptation,
// its x subvector) drops below a byte budget.  Subtrees run on separate
// threads; every random choice is seeded from (seed, tree path), so the
// result does not depend on the thread count.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <numeric>
#include <queue>
#include <random>
#include <thread>
#include <tuple>
#include <vector>

#include "spmv_internal.h"

namespace spmv {
namespace {

using i32 = int32_t;
using i64 = int64_t;
using u64 = uint64_t;

enum NetType : uint8_t { NET_CONN = 0, NET_REMOVE = 1 };
enum NetKind : uint8_t { KIND_ROW = 0, KIND_COL = 1 };

u64 splitmix(u64 z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

struct HG {
    i32 nv = 0, nn = 0;
    std::vector<i64> xpins;      // nn + 1
    std::vector<i32> pins;
    std::vector<i64> xnets;      // nv + 1
    std::vector<i32> nets;
    std::vector<i64> vw;         // vertex weight (balance)
    std::vector<i32> nc;         // net cost
    std::vector<uint8_t> nt;     // NetType
    std::vector<uint8_t> nk;     // NetKind
    std::vector<i32> nid;        // original row / column index of the net
    std::vector<i32> vid;        // original vertex id (finest level only)
    std::vector<i32> vz;         // nonzeros carried by the vertex (finest level only)

    i64 pins_of(i32 n) const { return xpins[n + 1] - xpins[n]; }

    // The transpose: the nets of each vertex in increasing order.  With
    // several threads each takes a range of nets, counts its pins per
    // vertex and writes after the threads before it, so the result is the
    // serial one (used on coarse levels: few vertices, many pins).
    void build_vertex_side(int threads = 1)
    {
        const i64 np = (i64)pins.size();
        xnets.assign((size_t)nv + 1, 0);
        nets.resize((size_t)np);
        int T = std::max(1, threads);
        if (np < (1 << 20)) T = 1;
        T = (int)std::min<i64>(T, std::max<i64>(1, ((i64)64 << 20) / (8 * std::max<i32>(nv, 1))));
        if (T == 1) {
            for (i64 q = 0; q < np; ++q) xnets[pins[q] + 1]++;
            for (i32 v = 0; v < nv; ++v) xnets[v + 1] += xnets[v];
            std::vector<i64> pos(xnets.begin(), xnets.end() - 1);
            for (i32 n = 0; n < nn; ++n)
                for (i64 q = xpins[n]; q < xpins[n + 1]; ++q) nets[pos[pins[q]]++] = n;
            return;
        }
        // net ranges of about np / T pins each
        std::vector<i32> nb((size_t)T + 1, nn);
        nb[0] = 0;
        for (int t = 1; t < T; ++t)
            nb[t] = (i32)(std::lower_bound(xpins.begin(), xpins.begin() + nn, np * t / T) -
                          xpins.begin());
        std::vector<std::vector<i64>> off((size_t)T, std::vector<i64>((size_t)nv, 0));
        auto run = [&](auto &&body) {
            std::vector<std::thread> ts;
            for (int t = 1; t < T; ++t) ts.emplace_back(body, t);
            body(0);
            for (auto &th : ts) th.join();
        };
        run([&](int t) {
            std::vector<i64> &c = off[t];
            for (i64 q = xpins[nb[t]]; q < xpins[nb[t + 1]]; ++q) c[pins[q]]++;
        });
        for (i32 v = 0; v < nv; ++v) {
            i64 at = xnets[v];
            for (int t = 0; t < T; ++t) {
                const i64 c = off[t][v];
                off[t][v] = at;
                at += c;
            }
            xnets[v + 1] = at;
        }
        run([&](int t) {
            std::vector<i64> &o = off[t];
            for (i32 n = nb[t]; n < nb[t + 1]; ++n)
                for (i64 q = xpins[n]; q < xpins[n + 1]; ++q) nets[o[pins[q]]++] = n;
        });
    }
};

// ------------------------------------------------------------- coarsening --
struct Coarsen {
    static constexpr i32 kNetMax = 1024;     // nets above this are ignored by matching
    static constexpr i64 kBudget = 128;      // pins scanned per vertex in HCM

    // heavy-connectivity matching: pair each vertex with the unmatched
    // neighbour sharing the most net weight c(n)/(|n|-1)
    static i32 hcm(const HG &G, i64 maxw, std::mt19937_64 &rng, std::vector<i32> &cmap)
    {
        const i32 nv = G.nv;
        std::vector<i32> order((size_t)nv);
        std::iota(order.begin(), order.end(), 0);
        std::shuffle(order.begin(), order.end(), rng);
        std::vector<i32> match((size_t)nv, -1);
        std::vector<double> score((size_t)nv, 0.0);
        std::vector<i32> touched;
        for (i32 u : order) {
            if (match[u] >= 0) continue;
            touched.clear();
            i64 budget = 0;
            for (i64 a = G.xnets[u]; a < G.xnets[u + 1] && budget < kBudget; ++a) {
                const i32 n = G.nets[a];
                const i64 sz = G.pins_of(n);
                if (sz < 2 || sz > kNetMax) continue;
                const double w = (double)G.nc[n] / (double)(sz - 1);
                for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) {
                    const i32 v = G.pins[q];
                    if (v == u || match[v] >= 0) continue;
                    if (score[v] == 0.0) touched.push_back(v);
                    score[v] += w;
                }
                budget += sz;
            }
            i32 best = -1;
            double bs = 0.0;
            for (i32 v : touched) {
                if (score[v] > bs && G.vw[u] + G.vw[v] <= maxw) {
                    bs = score[v];
                    best = v;
                }
                score[v] = 0.0;
            }
            if (best >= 0) {
                match[u] = best;
                match[best] = u;
            } else {
                match[u] = u;
            }
        }
        pair_leftovers(G, maxw, match);
        return number(match, cmap);
    }

    // Vertices left alone (joined only through nets too large to scan) would
    // stall the coarsening; pair them in visiting order so the hierarchy
    // keeps shrinking.  Only done when they are a large share of the level.
    static void pair_leftovers(const HG &G, i64 maxw, std::vector<i32> &match)
    {
        std::vector<i32> alone;
        for (i32 v = 0; v < G.nv; ++v)
            if (match[v] == v) alone.push_back(v);
        if ((double)alone.size() < 0.15 * (double)G.nv) return;
        i32 prev = -1;
        for (i32 v : alone) {
            if (prev < 0) {
                prev = v;
            } else if (G.vw[prev] + G.vw[v] <= maxw) {
                match[prev] = v;
                match[v] = prev;
                prev = -1;
            } else {
                prev = v;
            }
        }
    }

    // linear-time matching for very large levels: walk nets from the smallest
    // and pair consecutive unmatched pins
    static i32 net_matching(const HG &G, i64 maxw, std::mt19937_64 &rng, std::vector<i32> &cmap)
    {
        const i32 nv = G.nv;
        std::vector<i32> match((size_t)nv, -1);
        std::vector<std::tuple<double, u64, i32>> order;
        order.reserve((size_t)G.nn);
        for (i32 n = 0; n < G.nn; ++n) {
            i64 sz = G.pins_of(n);
            if (sz < 2 || sz > 4 * kNetMax) continue;
            // heaviest connectivity c(n)/(|n|-1) first, random ties
            order.emplace_back(-(double)G.nc[n] / (double)(sz - 1), rng(), n);
        }
        std::sort(order.begin(), order.end());
        for (auto &o : order) {
            const i32 n = std::get<2>(o);
            i32 prev = -1;
            for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) {
                const i32 v = G.pins[q];
                if (match[v] >= 0) continue;
                if (prev < 0) {
                    prev = v;
                } else if (G.vw[prev] + G.vw[v] <= maxw) {
                    match[prev] = v;
                    match[v] = prev;
                    prev = -1;
                } else {
                    prev = v;
                }
            }
        }
        for (i32 v = 0; v < nv; ++v)
            if (match[v] < 0) match[v] = v;
        return number(match, cmap);
    }

    static i32 number(const std::vector<i32> &match, std::vector<i32> &cmap)
    {
        const i32 nv = (i32)match.size();
        cmap.assign((size_t)nv, -1);
        i32 nc = 0;
        for (i32 v = 0; v < nv; ++v) {
            if (cmap[v] >= 0) continue;
            cmap[v] = nc;
            if (match[v] != v) cmap[match[v]] = nc;
            ++nc;
        }
        return nc;
    }

    static HG contract(const HG &G, const std::vector<i32> &cmap, i32 ncv, int threads)
    {
        HG C;
        C.nv = ncv;
        C.vw.assign((size_t)ncv, 0);
        for (i32 v = 0; v < G.nv; ++v) C.vw[cmap[v]] += G.vw[v];
        threads = std::max(1, std::min(threads, (int)(G.pins.size() / 200000) + 1));
        struct Part {
            std::vector<i64> sizes;
            std::vector<i32> pins, nc, nid;
            std::vector<uint8_t> nt, nk;
        };
        std::vector<Part> parts((size_t)threads);
        auto work = [&](int t) {
            Part &P = parts[t];
            const i32 b = (i32)((i64)G.nn * t / threads), e = (i32)((i64)G.nn * (t + 1) / threads);
            std::vector<i32> buf;
            for (i32 n = b; n < e; ++n) {
                buf.clear();
                for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) buf.push_back(cmap[G.pins[q]]);
                std::sort(buf.begin(), buf.end());
                buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
                if (buf.size() < 2) continue;
                P.sizes.push_back((i64)buf.size());
                P.pins.insert(P.pins.end(), buf.begin(), buf.end());
                P.nc.push_back(G.nc[n]);
                P.nt.push_back(G.nt[n]);
                P.nk.push_back(G.nk[n]);
                P.nid.push_back(G.nid[n]);
            }
        };
        if (threads == 1) {
            work(0);
        } else {
            std::vector<std::thread> ts;
            for (int t = 0; t < threads; ++t) ts.emplace_back(work, t);
            for (auto &t : ts) t.join();
        }
        i64 nn = 0, np = 0;
        for (auto &P : parts) {
            nn += (i64)P.sizes.size();
            np += (i64)P.pins.size();
        }
        C.nn = (i32)nn;
        C.xpins.resize((size_t)nn + 1);
        C.pins.reserve((size_t)np);
        C.nc.reserve((size_t)nn);
        C.nt.reserve((size_t)nn);
        C.nk.reserve((size_t)nn);
        C.nid.reserve((size_t)nn);
        C.xpins[0] = 0;
        i64 k = 0;
        for (auto &P : parts) {
            for (i64 s : P.sizes) {
                C.xpins[k + 1] = C.xpins[k] + s;
                ++k;
            }
            C.pins.insert(C.pins.end(), P.pins.begin(), P.pins.end());
            C.nc.insert(C.nc.end(), P.nc.begin(), P.nc.end());
            C.nt.insert(C.nt.end(), P.nt.begin(), P.nt.end());
            C.nk.insert(C.nk.end(), P.nk.begin(), P.nk.end());
            C.nid.insert(C.nid.end(), P.nid.begin(), P.nid.end());
            P = Part();
        }
        merge_identical(C, threads);
        C.build_vertex_side(threads);
        return C;
    }

    // Nets with the same pin set are cut together: keep one with the summed
    // cost (coarse levels only; the split bookkeeping uses the finest level).
    static void merge_identical(HG &C, int threads = 1)
    {
        if (C.nn < 2) return;
        std::vector<std::pair<u64, i32>> key((size_t)C.nn);
        auto hash = [&](int t, int T) {
            const i32 b = (i32)((i64)C.nn * t / T), e = (i32)((i64)C.nn * (t + 1) / T);
            for (i32 n = b; n < e; ++n) {
                u64 h = 1469598103934665603ULL ^ (u64)C.pins_of(n);
                for (i64 q = C.xpins[n]; q < C.xpins[n + 1]; ++q)
                    h = (h ^ (u64)C.pins[q]) * 1099511628211ULL;
                key[n] = {h, n};
            }
        };
        const int T = C.pins.size() > (1u << 20) ? std::max(1, threads) : 1;
        if (T == 1) {
            hash(0, 1);
        } else {
            std::vector<std::thread> ts;
            for (int t = 1; t < T; ++t) ts.emplace_back(hash, t, T);
            hash(0, T);
            for (auto &th : ts) th.join();
        }
        std::sort(key.begin(), key.end());
        std::vector<i32> keep_of((size_t)C.nn, -1);
        i64 merged = 0;
        for (size_t a = 0; a < key.size();) {
            size_t b = a;
            while (b < key.size() && key[b].first == key[a].first) ++b;
            for (size_t i = a; i < b; ++i) {
                const i32 n = key[i].second;
                if (keep_of[n] >= 0) continue;
                keep_of[n] = n;
                for (size_t j = i + 1; j < b; ++j) {
                    const i32 o = key[j].second;
                    if (keep_of[o] >= 0 || C.pins_of(o) != C.pins_of(n)) continue;
                    if (!std::equal(C.pins.begin() + C.xpins[n], C.pins.begin() + C.xpins[n + 1],
                                    C.pins.begin() + C.xpins[o]))
                        continue;
                    keep_of[o] = n;
                    C.nc[n] += C.nc[o];
                    ++merged;
                }
            }
            a = b;
        }
        if (merged == 0) return;
        HG M;
        M.nv = C.nv;
        M.vw.swap(C.vw);
        M.xpins.assign(1, 0);
        M.pins.reserve(C.pins.size());
        for (i32 n = 0; n < C.nn; ++n) {
            if (keep_of[n] != n) continue;
            M.pins.insert(M.pins.end(), C.pins.begin() + C.xpins[n], C.pins.begin() + C.xpins[n + 1]);
            M.xpins.push_back((i64)M.pins.size());
            M.nc.push_back(C.nc[n]);
            M.nt.push_back(C.nt[n]);
            M.nk.push_back(C.nk[n]);
            M.nid.push_back(C.nid[n]);
        }
        M.nn = (i32)M.nc.size();
        C = std::move(M);
    }
};

// -------------------------------------------------------------- 2-way FM --
// Indexed binary max-heap of vertices keyed by FM gain (ties broken by a
// per-pass random priority), with O(log n) updates and no stale entries.
struct GainHeap {
    std::vector<i32> h;
    std::vector<i32> *pos;
    const std::vector<i64> *gain;
    const std::vector<uint32_t> *tb;

    // a strict total order, so the top does not depend on the heap's layout
    bool above(i32 a, i32 b) const
    {
        const i64 ga = (*gain)[a], gb = (*gain)[b];
        if (ga != gb) return ga > gb;
        const uint32_t ta = (*tb)[a], tbb = (*tb)[b];
        return ta != tbb ? ta > tbb : a < b;
    }
    void up(size_t i)
    {
        const i32 v = h[i];
        while (i > 0) {
            size_t p = (i - 1) / 2;
            if (!above(v, h[p])) break;
            h[i] = h[p];
            (*pos)[h[i]] = (i32)i;
            i = p;
        }
        h[i] = v;
        (*pos)[v] = (i32)i;
    }
    void down(size_t i)
    {
        const i32 v = h[i];
        const size_t n = h.size();
        for (;;) {
            size_t c = 2 * i + 1;
            if (c >= n) break;
            if (c + 1 < n && above(h[c + 1], h[c])) ++c;
            if (!above(h[c], v)) break;
            h[i] = h[c];
            (*pos)[h[i]] = (i32)i;
            i = c;
        }
        h[i] = v;
        (*pos)[v] = (i32)i;
    }
    void push(i32 v)
    {
        h.push_back(v);
        up(h.size() - 1);
    }
    void update(i32 v)
    {
        const size_t i = (size_t)(*pos)[v];
        up(i);
        down((size_t)(*pos)[v]);
    }
    void erase(i32 v)
    {
        const size_t i = (size_t)(*pos)[v];
        (*pos)[v] = -1;
        const i32 last = h.back();
        h.pop_back();
        if (i < h.size()) {
            h[i] = last;
            (*pos)[last] = (i32)i;
            up(i);
            down((size_t)(*pos)[last]);
        }
    }
    bool empty() const { return h.empty(); }
    i32 top() const { return h[0]; }
};

struct FM {
    static constexpr i64 kBigNet = 4096;
    const HG &G;
    std::vector<uint8_t> &side;
    i64 maxw[2];
    std::vector<i32> cnt;        // 2 per net
    i64 w[2] = {0, 0};
    std::vector<i64> gain;
    std::vector<uint8_t> locked;
    std::vector<i32> pos;        // heap position, -1 = not in a heap
    std::vector<uint32_t> tb;    // random tie-break per vertex
    GainHeap heap[2];

    FM(const HG &g, std::vector<uint8_t> &s, i64 m0, i64 m1) : G(g), side(s)
    {
        maxw[0] = m0;
        maxw[1] = m1;
        for (int k = 0; k < 2; ++k) {
            heap[k].pos = &pos;
            heap[k].gain = &gain;
            heap[k].tb = &tb;
        }
    }

    void init_counts()
    {
        cnt.assign((size_t)G.nn * 2, 0);
        tracked = true;
        for (i32 n = 0; n < G.nn && tracked; ++n) tracked = G.pins_of(n) <= kBigNet;
        w[0] = w[1] = 0;
        for (i32 v = 0; v < G.nv; ++v) w[side[v]] += G.vw[v];
        for (i32 n = 0; n < G.nn; ++n)
            for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) cnt[2 * n + side[G.pins[q]]]++;
    }

    i64 vgain(i32 v) const
    {
        const int s = side[v], t = 1 - s;
        i64 g = 0;
        for (i64 a = G.xnets[v]; a < G.xnets[v + 1]; ++a) {
            const i32 n = G.nets[a];
            if (cnt[2 * n + s] == 1) g += G.nc[n];
            if (cnt[2 * n + t] == 0) g -= G.nc[n];
        }
        return g;
    }

    i64 cut() const
    {
        i64 c = 0;
        for (i32 n = 0; n < G.nn; ++n)
            if (cnt[2 * n] > 0 && cnt[2 * n + 1] > 0) c += G.nc[n];
        return c;
    }

    std::vector<i32> pending;        // vertices entering the candidate set
    std::vector<uint8_t> is_pending;
    // gain_ok[u]: gain[u] is exact although u is not in a heap (it left one
    // as infeasible, or entered the candidate set earlier in the pass), so
    // re-entering costs no recount of its nets.  Kept only when every net
    // gets the per-move updates (none above kBigNet pins).
    std::vector<uint8_t> gain_ok;
    bool tracked = true;
    // gain changes of one move, summed per vertex before the heaps see them
    // (at coarse levels a move touches the same few vertices through
    // thousands of nets)
    std::vector<i64> delta;
    std::vector<i32> touched;
    std::vector<uint8_t> is_touched;

    void bump(i32 u, i64 d)
    {
        if (locked[u]) return;
        if (!is_touched[u]) {
            is_touched[u] = 1;
            touched.push_back(u);
        }
        delta[u] += d;
    }

    void flush_bumps()
    {
        for (i32 u : touched) {
            is_touched[u] = 0;
            const i64 d = delta[u];
            delta[u] = 0;
            if (locked[u]) continue;
            if (pos[u] >= 0) {
                if (d != 0) {
                    gain[u] += d;
                    heap[side[u]].update(u);
                }
            } else {
                if (gain_ok[u]) gain[u] += d;
                if (!is_pending[u]) {
                    // not in a heap: it re-enters once the move is complete
                    // (with its gain counted then if it was never known)
                    is_pending[u] = 1;
                    pending.push_back(u);
                }
            }
        }
        touched.clear();
    }

    void flush_pending()
    {
        for (i32 u : pending) {
            is_pending[u] = 0;
            if (locked[u] || pos[u] >= 0) continue;
            if (!gain_ok[u]) {
                gain[u] = vgain(u);
                gain_ok[u] = tracked;
            }
            heap[side[u]].push(u);
        }
        pending.clear();
    }

    // One or more FM passes; returns the total cut reduction.
    i64 refine(int passes, i64 max_stall, std::mt19937_64 &rng, bool boundary_only)
    {
        init_counts();
        gain.assign((size_t)G.nv, 0);
        pos.assign((size_t)G.nv, -1);
        tb.resize((size_t)G.nv);
        is_pending.assign((size_t)G.nv, 0);
        delta.assign((size_t)G.nv, 0);
        is_touched.assign((size_t)G.nv, 0);
        touched.clear();
        i64 total = 0;
        for (int pass = 0; pass < passes; ++pass) {
            locked.assign((size_t)G.nv, 0);
            gain_ok.assign((size_t)G.nv, 0);
            for (i32 v = 0; v < G.nv; ++v) tb[v] = (uint32_t)rng();
            heap[0].h.clear();
            heap[1].h.clear();
            std::fill(pos.begin(), pos.end(), -1);
            for (i32 v = 0; v < G.nv; ++v) {
                bool cand = !boundary_only;
                if (boundary_only)
                    for (i64 a = G.xnets[v]; a < G.xnets[v + 1] && !cand; ++a) {
                        const i32 n = G.nets[a];
                        cand = cnt[2 * n] > 0 && cnt[2 * n + 1] > 0;
                    }
                if (!cand) continue;
                gain[v] = vgain(v);
                gain_ok[v] = tracked;
                heap[side[v]].push(v);
            }
            std::vector<i32> moves;
            i64 cum = 0, best = 0, best_imb = std::llabs(w[0] - w[1]);
            size_t best_len = 0;
            i64 stall = 0;
            while (stall < max_stall) {
                i32 cand[2] = {-1, -1};
                for (int s = 0; s < 2; ++s) {
                    while (!heap[s].empty()) {
                        const i32 v = heap[s].top();
                        if (w[1 - s] + G.vw[v] > maxw[1 - s]) {
                            heap[s].erase(v);     // infeasible now; may come back on a bump
                            continue;
                        }
                        cand[s] = v;
                        break;
                    }
                }
                int s;
                if (cand[0] < 0 && cand[1] < 0) break;
                if (cand[0] < 0) s = 1;
                else if (cand[1] < 0) s = 0;
                else if (gain[cand[0]] != gain[cand[1]]) s = gain[cand[0]] > gain[cand[1]] ? 0 : 1;
                else s = w[0] >= w[1] ? 0 : 1;
                const i32 v = cand[s];
                heap[s].erase(v);
                cum += gain[v];
                move(v, s, 1 - s);
                flush_pending();
                moves.push_back(v);
                const i64 imb = std::llabs(w[0] - w[1]);
                if (cum > best || (cum == best && imb < best_imb)) {
                    best = cum;
                    best_imb = imb;
                    best_len = moves.size();
                    stall = 0;
                } else {
                    ++stall;
                }
            }
            // roll back past the best prefix
            for (size_t i = moves.size(); i > best_len; --i) {
                const i32 v = moves[i - 1];
                const int s = side[v], t = 1 - s;
                for (i64 a = G.xnets[v]; a < G.xnets[v + 1]; ++a) {
                    const i32 n = G.nets[a];
                    cnt[2 * n + s]--;
                    cnt[2 * n + t]++;
                }
                w[s] -= G.vw[v];
                w[t] += G.vw[v];
                side[v] = (uint8_t)t;
            }
            total += best;
            if (best <= 0) break;
        }
        return total;
    }

    // Move v from s to t with the classical FM gain updates on its nets.
    void move(i32 v, int s, int t)
    {
        locked[v] = 1;
        for (i64 a = G.xnets[v]; a < G.xnets[v + 1]; ++a) {
            const i32 n = G.nets[a];
            const i64 c = G.nc[n];
            if (G.pins_of(n) > kBigNet) {
                // too large to update every pin per move: counts stay exact,
                // the pins' gains are refreshed at the next pass
                cnt[2 * n + s]--;
                cnt[2 * n + t]++;
                continue;
            }
            const i32 T = cnt[2 * n + t];
            if (T == 0) {
                for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) {
                    const i32 u = G.pins[q];
                    if (u != v) bump(u, c);
                }
            } else if (T == 1) {
                for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) {
                    const i32 u = G.pins[q];
                    if (side[u] == t) {
                        bump(u, -c);
                        break;
                    }
                }
            }
            cnt[2 * n + s]--;
            cnt[2 * n + t]++;
            const i32 F = cnt[2 * n + s];
            if (F == 0) {
                for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) {
                    const i32 u = G.pins[q];
                    if (u != v) bump(u, -c);
                }
            } else if (F == 1) {
                for (i64 q = G.xpins[n]; q < G.xpins[n + 1]; ++q) {
                    const i32 u = G.pins[q];
                    if (u != v && side[u] == s) {
                        bump(u, c);
                        break;
                    }
                }
            }
        }
        w[s] -= G.vw[v];
        w[t] += G.vw[v];
        side[v] = (uint8_t)t;
        flush_bumps();
    }
};

// greedy growing of side 0 from a random seed, by best FM gain
void grow(const HG &G, i64 target0, std::mt19937_64 &rng, std::vector<uint8_t> &side)
{
    side.assign((size_t)G.nv, 1);
    if (G.nv == 0) return;
    if (G.nv > 2000) {
        // coarsening stalled on a large level: start from a random balanced
        // split and leave the work to FM
        std::vector<i32> order((size_t)G.nv);
        std::iota(order.begin(), order.end(), 0);
        std::shuffle(order.begin(), order.end(), rng);
        i64 w0 = 0;
        for (i32 v : order) {
            if (w0 >= target0) break;
            side[v] = 0;
            w0 += G.vw[v];
        }
        return;
    }
    // moves by best gain, kept exact by the FM update rules (O(pins) per try)
    FM fm(G, side, std::numeric_limits<i64>::max(), std::numeric_limits<i64>::max());
    fm.init_counts();
    fm.gain.assign((size_t)G.nv, 0);
    fm.pos.assign((size_t)G.nv, -1);
    fm.tb.resize((size_t)G.nv);
    fm.is_pending.assign((size_t)G.nv, 0);
    fm.delta.assign((size_t)G.nv, 0);
    fm.is_touched.assign((size_t)G.nv, 0);
    fm.locked.assign((size_t)G.nv, 0);
    fm.gain_ok.assign((size_t)G.nv, 0);
    for (i32 v = 0; v < G.nv; ++v) {
        fm.tb[v] = (uint32_t)rng();
        fm.gain[v] = fm.vgain(v);
        fm.gain_ok[v] = fm.tracked;
        fm.heap[1].push(v);
    }
    i32 v = (i32)(rng() % (u64)G.nv);       // random seed vertex first
    while (fm.w[0] < target0) {
        fm.heap[1].erase(v);
        fm.move(v, 1, 0);
        fm.flush_pending();
        if (fm.heap[1].empty()) break;
        v = fm.heap[1].top();
    }
}

// Multilevel bisection of G into sides 0/1 with weights near half.
// Copy of G without the nets above `limit` pins.  Such nets are cut by almost
// any balanced bisection; leaving them out keeps coarsening and FM fast on
// power-law matrices (their cost is still counted exactly by the caller).
bool drop_large_nets(const HG &G, i64 limit, HG &out)
{
    i64 big = 0;
    for (i32 n = 0; n < G.nn; ++n) big += G.pins_of(n) > limit;
    if (big == 0) return false;
    out.nv = G.nv;
    out.vw = G.vw;
    out.xpins.assign(1, 0);
    for (i32 n = 0; n < G.nn; ++n) {
        if (G.pins_of(n) > limit) continue;
        out.pins.insert(out.pins.end(), G.pins.begin() + G.xpins[n], G.pins.begin() + G.xpins[n + 1]);
        out.xpins.push_back((i64)out.pins.size());
        out.nc.push_back(G.nc[n]);
        out.nt.push_back(G.nt[n]);
        out.nk.push_back(G.nk[n]);
        out.nid.push_back(G.nid[n]);
    }
    out.nn = (i32)out.nc.size();
    out.build_vertex_side();
    return true;
}

void bisect_core(const HG &G, double eps, u64 seed, int threads, std::vector<uint8_t> &side);

void bisect(const HG &G, double eps, u64 seed, int threads, std::vector<uint8_t> &side)
{
    HG small;
    if (drop_large_nets(G, 1024, small)) bisect_core(small, eps, seed, threads, side);
    else bisect_core(G, eps, seed, threads, side);
}

void bisect_core(const HG &G, double eps, u64 seed, int threads, std::vector<uint8_t> &side)
{
    std::mt19937_64 rng(seed);
    const i64 total = std::accumulate(G.vw.begin(), G.vw.end(), (i64)0);
    const i64 half = total / 2;
    const i64 maxw = (i64)std::ceil((1.0 + eps) * (double)total / 2.0);
    i64 vmax = 0;
    for (i64 x : G.vw) vmax = std::max(vmax, x);
    const i64 mw0 = std::max(maxw, half + vmax), mw1 = std::max(maxw, total - half + vmax);

    std::vector<HG> levels;
    std::vector<std::vector<i32>> maps;
    const HG *cur = &G;
    const i32 coarse_to = 160;
    const i64 cap = std::max<i64>(vmax, total / 96);
    while (cur->nv > coarse_to && levels.size() < 48) {
        std::vector<i32> cmap;
        i32 ncv;
        if (cur->nv > 200000) ncv = Coarsen::net_matching(*cur, cap, rng, cmap);
        else ncv = Coarsen::hcm(*cur, cap, rng, cmap);
        if (ncv > (i32)(0.92 * cur->nv)) break;
        levels.push_back(Coarsen::contract(*cur, cmap, ncv, threads));
        maps.push_back(std::move(cmap));
        cur = &levels.back();
    }
    // initial bisection: several greedy growings refined by FM; keep the best
    std::vector<uint8_t> best_side;
    i64 best_cut = std::numeric_limits<i64>::max();
    i64 best_imb = std::numeric_limits<i64>::max();
    const int tries = cur->pins.size() > 200000 ? 3 : 6;
    for (int t = 0; t < tries; ++t) {
        std::vector<uint8_t> s;
        grow(*cur, half, rng, s);
        FM fm(*cur, s, mw0, mw1);
        fm.refine(2, std::max<i64>(cur->nv, 50), rng, false);
        const bool ok = fm.w[0] <= mw0 && fm.w[1] <= mw1;
        const i64 c = fm.cut(), imb = std::llabs(fm.w[0] - fm.w[1]);
        if (!ok) continue;
        if (c < best_cut || (c == best_cut && imb < best_imb)) {
            best_cut = c;
            best_imb = imb;
            best_side = s;
        }
    }
    if (best_side.empty()) {
        // no balanced growing (should not happen): alternate by weight
        best_side.assign((size_t)cur->nv, 0);
        i64 w0 = 0;
        for (i32 v = 0; v < cur->nv; ++v) {
            best_side[v] = w0 >= half;
            if (!best_side[v]) w0 += cur->vw[v];
        }
    }
    std::vector<uint8_t> s = std::move(best_side);
    // uncoarsen with refinement
    for (size_t l = levels.size(); l > 0; --l) {
        const HG &fine = (l >= 2) ? levels[l - 2] : G;
        const std::vector<i32> &cmap = maps[l - 1];
        std::vector<uint8_t> fs((size_t)fine.nv);
        for (i32 v = 0; v < fine.nv; ++v) fs[v] = s[cmap[v]];
        s.swap(fs);
        levels.pop_back();     // the coarse level is no longer needed
        FM fm(fine, s, mw0, mw1);
        const bool big = fine.nv > 200000;
        fm.refine(big ? 1 : 2, big ? 1000 : std::min<i64>(2000, std::max<i64>(100, fine.nv / 50)), rng, true);
    }
    side.swap(s);
}

// ------------------------------------------------------------------ driver --
struct Leaf {
    u64 path;
    int depth;
    std::vector<i32> vids;
};

struct Driver {
    const spmv_csr *A;
    int method;
    int fixed_depth;            // >= 0: bisect exactly to this depth
    i64 part_bytes;
    int fit_rule;
    double eps;
    u64 seed;
    int threads;
    std::mutex mu;
    std::vector<Leaf> leaves;
    std::atomic<i64> cost{0};
    std::atomic<i64> cost_rows{0};
    std::vector<uint8_t> row_cut;        // eRCN: row net cut (row in R_B)
    // Net pieces with a single pin are dropped from the hypergraphs (they can
    // never be cut) but still count for the size rule, and for eRCN a lone
    // column piece disappears when its pin is removed.  single_r / single_c
    // count, per original vertex, the lone row / column pieces it holds.
    std::vector<i32> single_r, single_c;
    std::vector<i32> seg_of;             // RCN/eRCN: vertex (row segment) of each nonzero

    struct Job {
        HG H;
        int depth = 0;
        u64 path = 0;
        i64 single_rows = 0, single_cols = 0;   // lone pieces held by H's vertices
    };

    bool stop(const Job &j) const
    {
        if (fixed_depth >= 0) return j.depth >= fixed_depth;
        if (j.H.nv < 2 || j.depth >= 40) return true;
        i64 rows, cols, nnz;
        if (method == SPMV_PART_CN) {
            rows = j.H.nv;
            nnz = 0;
            for (i32 v : j.H.vz) nnz += v;
            cols = j.H.nn + j.single_cols;
        } else {
            nnz = 0;
            for (i32 v : j.H.vz) nnz += v;
            rows = j.single_rows;
            cols = j.single_cols;
            for (i32 n = 0; n < j.H.nn; ++n) (j.H.nk[n] == KIND_ROW ? rows : cols)++;
        }
        const bool gcsr = (method == SPMV_PART_RCN);
        i64 size;
        if (fit_rule == SPMV_FIT_X) size = cols * 8 + (gcsr ? rows * 8 : 0);
        else size = nnz * 12 + (rows + 1) * 4 + cols * 8 + rows * 8 + (gcsr ? rows * 4 : 0);
        return size < part_bytes;
    }

    void leaf(Job &j)
    {
        Leaf L;
        L.path = j.path;
        L.depth = j.depth;
        L.vids = std::move(j.H.vid);
        std::lock_guard<std::mutex> g(mu);
        leaves.push_back(std::move(L));
    }

    void run(Job j)
    {
        if (stop(j)) {
            leaf(j);
            return;
        }
        const int job_threads = std::max(1, threads >> std::min(j.depth, 20));
        std::vector<uint8_t> side;
        const u64 s = splitmix(seed ^ splitmix((j.path << 6) | (u64)j.depth));
        if (j.H.nv >= 2) bisect(j.H, eps, s, job_threads, side);
        else side.assign((size_t)j.H.nv, 0);
        Job c[2];
        split(j, side, c);
        j = Job();
        const bool spawn = (1 << (c[0].depth)) <= threads && threads > 1;
        if (spawn) {
            std::thread t([this, &c] { run(std::move(c[1])); });
            run(std::move(c[0]));
            t.join();
        } else {
            run(std::move(c[0]));
            run(std::move(c[1]));
        }
    }

    // Build the two halves: split connectivity nets (cost +1 per new piece),
    // remove the vertices of cut removal nets (eRCN, cost nnz(r_i)).
    void split(Job &j, const std::vector<uint8_t> &side, Job *c)
    {
        const HG &H = j.H;
        std::vector<uint8_t> gone((size_t)H.nv, 0);
        i64 dcost = 0, drows = 0;
        // 1. cut removal nets
        for (i32 n = 0; n < H.nn; ++n) {
            if (H.nt[n] != NET_REMOVE) continue;
            i32 p0 = 0, p1 = 0;
            for (i64 q = H.xpins[n]; q < H.xpins[n + 1]; ++q) (side[H.pins[q]] ? p1 : p0)++;
            if (p0 > 0 && p1 > 0) {
                dcost += H.nc[n];
                drows += H.nc[n];
                row_cut[H.nid[n]] = 1;
                for (i64 q = H.xpins[n]; q < H.xpins[n + 1]; ++q) gone[H.pins[q]] = 1;
            }
        }
        // a removed vertex takes its lone column pieces with it
        for (i32 v = 0; v < H.nv; ++v)
            if (gone[v]) dcost -= single_c[H.vid[v]];
        // 2. new vertex numbering per side
        std::vector<i32> nid_of((size_t)H.nv, -1);
        i32 cntv[2] = {0, 0};
        for (i32 v = 0; v < H.nv; ++v)
            if (!gone[v]) nid_of[v] = cntv[side[v]]++;
        for (int s = 0; s < 2; ++s) {
            HG &C = c[s].H;
            C.nv = cntv[s];
            C.vw.resize((size_t)cntv[s]);
            C.vid.resize((size_t)cntv[s]);
            C.vz.resize((size_t)cntv[s]);
            C.xpins.assign(1, 0);
            c[s].depth = j.depth + 1;
            c[s].path = (j.path << 1) | (u64)s;
        }
        for (i32 v = 0; v < H.nv; ++v) {
            if (gone[v]) continue;
            HG &C = c[side[v]].H;
            const i32 u = nid_of[v];
            C.vw[u] = H.vw[v];
            C.vid[u] = H.vid[v];
            C.vz[u] = H.vz[v];
        }
        // 3. nets
        std::vector<i32> buf[2];
        for (i32 n = 0; n < H.nn; ++n) {
            if (H.nt[n] == NET_REMOVE) {
                // uncut removal nets go whole to one side
                bool cut = row_cut[H.nid[n]];
                if (cut) continue;
            }
            buf[0].clear();
            buf[1].clear();
            for (i64 q = H.xpins[n]; q < H.xpins[n + 1]; ++q) {
                const i32 v = H.pins[q];
                if (gone[v]) continue;
                buf[side[v]].push_back(nid_of[v]);
            }
            const int pieces = (!buf[0].empty()) + (!buf[1].empty());
            if (H.nt[n] == NET_CONN) dcost += pieces - 1;
            for (int s = 0; s < 2; ++s) {
                if (buf[s].empty()) continue;
                if (buf[s].size() == 1) {
                    const i32 ov = c[s].H.vid[buf[s][0]];
                    (H.nk[n] == KIND_ROW ? single_r : single_c)[ov]++;
                    continue;
                }
                HG &C = c[s].H;
                C.pins.insert(C.pins.end(), buf[s].begin(), buf[s].end());
                C.xpins.push_back((i64)C.pins.size());
                C.nc.push_back(H.nc[n]);
                C.nt.push_back(H.nt[n]);
                C.nk.push_back(H.nk[n]);
                C.nid.push_back(H.nid[n]);
            }
        }
        for (int s = 0; s < 2; ++s) {
            HG &C = c[s].H;
            C.nn = (i32)C.nc.size();
            C.build_vertex_side();
            for (i32 u = 0; u < C.nv; ++u) {
                c[s].single_rows += single_r[C.vid[u]];
                c[s].single_cols += single_c[C.vid[u]];
            }
        }
        cost += dcost;
        cost_rows += drows;
    }
};

HG build_model(const spmv_csr *A, int method, i32 seg, std::vector<i32> *seg_of)
{
    const i32 m = A->m, n = A->n;
    const i64 nnz = A->nnz;
    HG H;
    if (method == SPMV_PART_CN) {
        // vertices = rows, nets = columns
        H.nv = m;
        H.vw.resize((size_t)m);
        H.vid.resize((size_t)m);
        H.vz.resize((size_t)m);
        std::vector<i64> colcnt((size_t)n + 1, 0);
        for (i32 i = 0; i < m; ++i) {
            const i32 len = A->rowptr[i + 1] - A->rowptr[i];
            H.vw[i] = (i64)len * 12 + 4 + 8;
            H.vid[i] = i;
            H.vz[i] = len;
            for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) colcnt[A->colidx[p] + 1]++;
        }
        std::vector<i32> netof((size_t)n, -1);
        for (i32 j = 0; j < n; ++j)
            if (colcnt[j + 1] >= 2) netof[j] = H.nn++;
        H.xpins.assign((size_t)H.nn + 1, 0);
        for (i32 j = 0; j < n; ++j)
            if (netof[j] >= 0) H.xpins[netof[j] + 1] = colcnt[j + 1];
        for (i32 k = 0; k < H.nn; ++k) H.xpins[k + 1] += H.xpins[k];
        H.pins.resize((size_t)H.xpins[H.nn]);
        std::vector<i64> pos(H.xpins.begin(), H.xpins.end() - 1);
        for (i32 i = 0; i < m; ++i)
            for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
                const i32 k = netof[A->colidx[p]];
                if (k >= 0) H.pins[pos[k]++] = i;
            }
        H.nc.assign((size_t)H.nn, 1);
        H.nt.assign((size_t)H.nn, NET_CONN);
        H.nk.assign((size_t)H.nn, KIND_COL);
        H.nid.resize((size_t)H.nn);
        for (i32 j = 0; j < n; ++j)
            if (netof[j] >= 0) H.nid[netof[j]] = j;
    } else {
        // vertices = nonzeros, nets = rows and columns.  Large matrices start
        // from segments of `seg` consecutive nonzeros of a row (a fixed first
        // coarsening level); seg = 1 is the plain fine-grain model.
        const i64 nseg_max = nnz;
        seg_of->resize((size_t)nnz);
        std::vector<i32> seg_len;
        seg_len.reserve((size_t)std::min<i64>(nseg_max, nnz / std::max(seg, 1) + m + 1));
        std::vector<i32> row_seg0((size_t)m + 1, 0);
        for (i32 i = 0; i < m; ++i) {
            row_seg0[i] = (i32)seg_len.size();
            for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; p += seg) {
                const i32 len = std::min(seg, A->rowptr[i + 1] - p);
                for (i32 q = p; q < p + len; ++q) (*seg_of)[q] = (i32)seg_len.size();
                seg_len.push_back(len);
            }
        }
        row_seg0[m] = (i32)seg_len.size();
        const i32 ns = (i32)seg_len.size();
        H.nv = ns;
        H.vw.resize((size_t)ns);
        H.vid.resize((size_t)ns);
        H.vz.resize((size_t)ns);
        for (i32 v = 0; v < ns; ++v) {
            H.vw[v] = 12LL * seg_len[v];
            H.vid[v] = v;
            H.vz[v] = seg_len[v];
        }
        std::vector<i64> colcnt((size_t)n + 1, 0);
        for (i64 p = 0; p < nnz; ++p) colcnt[A->colidx[p] + 1]++;
        const bool erc = (method == SPMV_PART_ERCN);
        // row nets with >= 2 segments
        H.xpins.assign(1, 0);
        for (i32 i = 0; i < m; ++i) {
            const i32 len = A->rowptr[i + 1] - A->rowptr[i];
            if (row_seg0[i + 1] - row_seg0[i] < 2) continue;
            for (i32 v = row_seg0[i]; v < row_seg0[i + 1]; ++v) H.pins.push_back(v);
            H.xpins.push_back((i64)H.pins.size());
            H.nc.push_back(erc ? len : 1);
            H.nt.push_back(erc ? NET_REMOVE : NET_CONN);
            H.nk.push_back(KIND_ROW);
            H.nid.push_back(i);
        }
        // column nets with >= 2 pins (transpose; a row's columns are distinct,
        // so a column meets each segment at most once)
        for (i32 j = 0; j < n; ++j) colcnt[j + 1] += colcnt[j];
        std::vector<i32> bycol((size_t)nnz);
        {
            std::vector<i64> pos(colcnt.begin(), colcnt.end() - 1);
            for (i64 p = 0; p < nnz; ++p) bycol[pos[A->colidx[p]]++] = (*seg_of)[p];
        }
        for (i32 j = 0; j < n; ++j) {
            const i64 len = colcnt[j + 1] - colcnt[j];
            if (len < 2) continue;
            H.pins.insert(H.pins.end(), bycol.begin() + colcnt[j], bycol.begin() + colcnt[j + 1]);
            H.xpins.push_back((i64)H.pins.size());
            H.nc.push_back(1);
            H.nt.push_back(NET_CONN);
            H.nk.push_back(KIND_COL);
            H.nid.push_back(j);
        }
        H.nn = (i32)H.nc.size();
    }
    H.build_vertex_side();
    return H;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

namespace spmv {
spmv_status order_sbd(const spmv_csr *A, int32_t K, const int32_t *labels, int32_t *row_perm,
                      int32_t *col_perm);
}

// Row-net model (sHP_RN, Sec. 5.1): the columns are the vertices and the rows
// the nets, which is the column-net model of the transpose; the columns are
// ordered by part and the rows into the nested separated block-diagonal
// form (order_sbd).
static spmv_status partition_row_net(const spmv_csr *A, const spmv_partition_opts *opts,
                                     spmv_partition_out *out)
{
    const auto t0 = std::chrono::steady_clock::now();
    const i32 m = A->m, n = A->n;
    const i64 nnz = A->nnz;
    std::vector<i32> tp((size_t)n + 1, 0), ti((size_t)nnz);
    for (i64 p = 0; p < nnz; ++p) tp[(size_t)A->colidx[p] + 1]++;
    for (i32 j = 0; j < n; ++j) tp[(size_t)j + 1] += tp[(size_t)j];
    {
        std::vector<i32> fill(tp.begin(), tp.end() - 1);
        for (i32 i = 0; i < m; ++i)
            for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) ti[(size_t)fill[A->colidx[p]]++] = i;
    }
    std::vector<double> ones((size_t)nnz, 1.0);
    spmv_csr At{n, m, nnz, tp.data(), ti.data(), ones.data()};
    spmv_partition_opts o = *opts;
    o.method = SPMV_PART_CN;
    spmv_partition_out t{};
    spmv_status st = spmv_partition(&At, &o, &t);
    if (st != SPMV_OK) return st;
    const i32 K = t.K;
    std::vector<i32> labels(t.labels, t.labels + n);
    const i64 cost = t.cost;
    spmv_partition_free(&t);
    out->row_perm = (i32 *)std::malloc(sizeof(i32) * (size_t)std::max(m, 1));
    out->col_perm = (i32 *)std::malloc(sizeof(i32) * (size_t)std::max(n, 1));
    out->row_part_ptr = (i32 *)std::malloc(sizeof(i32) * (size_t)(K + 2));
    out->col_part_ptr = (i32 *)std::malloc(sizeof(i32) * (size_t)(K + 2));
    out->labels = (i32 *)std::malloc(sizeof(i32) * std::max<size_t>(labels.size(), 1));
    if (!out->row_perm || !out->col_perm || !out->row_part_ptr || !out->col_part_ptr ||
        !out->labels) {
        spmv_partition_free(out);
        set_error("out of host memory");
        return SPMV_E_NOMEM;
    }
    std::copy(labels.begin(), labels.end(), out->labels);
    st = spmv::order_sbd(A, K, labels.data(), out->row_perm, out->col_perm);
    if (st != SPMV_OK) {
        spmv_partition_free(out);
        return st;
    }
    // column parts: the label ranges; row parts: where each leaf's block
    // of rows starts in the nested order (separators lie between blocks)
    std::vector<i32> cc((size_t)K + 1, 0);
    for (i32 j = 0; j < n; ++j) cc[(size_t)labels[j] + 1]++;
    for (i32 k = 0; k < K; ++k) cc[(size_t)k + 1] += cc[(size_t)k];
    for (i32 k = 0; k <= K; ++k) out->col_part_ptr[k] = cc[(size_t)k];
    out->col_part_ptr[K + 1] = n;
    {
        i32 r = 0;
        for (i32 k = 0; k < K; ++k) {
            // first row (in the new order) whose columns lie in leaves >= k
            while (r < m) {
                const i32 i = out->row_perm[r];
                i32 lo = K;
                for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
                    lo = std::min(lo, labels[A->colidx[p]]);
                if (A->rowptr[i] < A->rowptr[i + 1] && lo < k) ++r;
                else break;
            }
            out->row_part_ptr[k] = r;
        }
        out->row_part_ptr[K] = out->row_part_ptr[K + 1] = m;
    }
    out->form = SPMV_NATURAL;
    out->K = K;
    out->n_labels = n;
    out->cost = cost;
    out->cost_rows = cost;
    out->cost_cols = 0;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return SPMV_OK;
}

extern "C" spmv_status spmv_partition(const spmv_csr *A, const spmv_partition_opts *opts,
                                      spmv_partition_out *out)
{
    clear_error();
    if (!out || !opts) {
        set_error("NULL argument");
        return SPMV_E_INVALID;
    }
    *out = spmv_partition_out{};
    try {
        spmv_status st = validate_csr(A);
        if (st != SPMV_OK) return st;
        const auto t0 = std::chrono::steady_clock::now();
        const int method = opts->method;
        if (method < SPMV_PART_CN || method > SPMV_PART_RN) {
            set_error("unknown partitioning method %d", method);
            return SPMV_E_INVALID;
        }
        if (method == SPMV_PART_RN) return partition_row_net(A, opts, out);
        int depth = -1;
        if (opts->K > 0) {
            if ((opts->K & (opts->K - 1)) != 0) {
                set_error("K=%d must be a power of two", opts->K);
                return SPMV_E_INVALID;
            }
            depth = 0;
            while ((1 << depth) < opts->K) ++depth;
        } else if (opts->part_bytes <= 0) {
            set_error("give K > 0 or part_bytes > 0");
            return SPMV_E_INVALID;
        }
        const i32 m = A->m, n = A->n;
        const i64 nnz = A->nnz;
        std::vector<i32> labels;
        i32 K = 0;
        int form;
        i64 cost = 0, cost_rows = 0, cost_cols = 0;
        if (method == SPMV_PART_RANDOM) {
            K = opts->K > 0 ? opts->K : std::max<i32>(1, (i32)((nnz * 12 + (i64)m * 12 + (i64)n * 8) / std::max<i64>(1, opts->part_bytes)) + 1);
            std::mt19937_64 rng(splitmix(opts->seed));
            labels.resize((size_t)m);
            for (i32 i = 0; i < m; ++i) labels[i] = (i32)(rng() % (u64)K);
            form = SPMV_SB;
        } else {
            Driver D;
            D.A = A;
            D.method = method;
            D.fixed_depth = depth;
            D.part_bytes = opts->part_bytes;
            D.fit_rule = opts->fit_rule;
            D.eps = opts->imbalance > 0 ? opts->imbalance : 0.10;
            D.seed = opts->seed;
            D.threads = opts->threads > 0 ? opts->threads : hardware_threads();
            // row-column-net models: segments of up to `seg` nonzeros of a row
            // keep the vertex count near 4M on large matrices
            const i32 seg = method == SPMV_PART_CN
                                ? 1
                                : (i32)std::min<i64>(8, std::max<i64>(1, (nnz + 3999999) / 4000000));
            HG H = build_model(A, method, seg, &D.seg_of);
            Driver::Job root;
            if (method == SPMV_PART_CN) {
                // columns with a single nonzero are single-pin nets
                std::vector<i32> colcnt((size_t)n, 0);
                for (i64 p = 0; p < nnz; ++p) colcnt[A->colidx[p]]++;
                i64 ne = 0, single = 0;
                for (i32 j = 0; j < n; ++j) {
                    ne += colcnt[j] > 0;
                    single += colcnt[j] == 1;
                }
                D.cost = ne;
                root.single_cols = single;
                D.single_r.assign((size_t)m, 0);
                D.single_c.assign((size_t)m, 0);
                for (i32 i = 0; i < m; ++i)
                    for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
                        if (colcnt[A->colidx[p]] == 1) D.single_c[i]++;
            } else {
                i64 ner = 0, nec = 0, sr = 0, sc = 0;
                std::vector<i32> colcnt((size_t)n, 0);
                for (i64 p = 0; p < nnz; ++p) colcnt[A->colidx[p]]++;
                for (i32 j = 0; j < n; ++j) {
                    nec += colcnt[j] > 0;
                    sc += colcnt[j] == 1;
                }
                D.cost = 0;
                D.row_cut.assign((size_t)m, 0);
                D.single_r.assign((size_t)H.nv, 0);
                D.single_c.assign((size_t)H.nv, 0);
                for (i32 i = 0; i < m; ++i) {
                    const i32 a = A->rowptr[i], b = A->rowptr[i + 1];
                    ner += b > a;
                    if (b > a && D.seg_of[a] == D.seg_of[b - 1]) {
                        D.single_r[D.seg_of[a]]++;     // the whole row is one vertex
                        ++sr;
                    }
                    for (i32 p = a; p < b; ++p)
                        if (colcnt[A->colidx[p]] == 1) D.single_c[D.seg_of[p]]++;
                }
                D.cost = (method == SPMV_PART_RCN) ? ner + nec : nec;
                root.single_rows = sr;
                root.single_cols = sc;
            }
            const i32 nvert = H.nv;
            root.H = std::move(H);
            D.run(std::move(root));
            // leaves -> part ids
            std::vector<std::pair<u64, size_t>> keys;
            for (size_t l = 0; l < D.leaves.size(); ++l) {
                const Leaf &L = D.leaves[l];
                const u64 aligned = L.depth ? (L.path << (64 - L.depth)) : 0;
                keys.emplace_back(aligned, l);
            }
            std::sort(keys.begin(), keys.end());
            std::vector<i32> vpart;
            vpart.assign((size_t)nvert, -1);
            if (depth >= 0) {
                K = 1 << depth;
                for (auto &k : keys) {
                    const Leaf &L = D.leaves[k.second];
                    const i32 id = (i32)(L.depth ? (L.path << (depth - L.depth)) : 0);
                    for (i32 v : L.vids) vpart[v] = id;
                }
            } else {
                K = (i32)keys.size();
                for (size_t r = 0; r < keys.size(); ++r)
                    for (i32 v : D.leaves[keys[r].second].vids) vpart[v] = (i32)r;
            }
            cost = D.cost.load();
            cost_rows = D.cost_rows.load();
            if (method == SPMV_PART_CN) {
                labels.swap(vpart);
                form = SPMV_SB;
                cost_cols = cost;
                cost_rows = 0;
            } else if (method == SPMV_PART_RCN) {
                // every nonzero takes the part of its row segment
                labels.resize((size_t)nnz);
                for (i64 p = 0; p < nnz; ++p) labels[p] = vpart[D.seg_of[p]];
                form = SPMV_SPLIT;
                // rows' share: lambda(r_i) sums, computed from the labels
                std::vector<i32> seen((size_t)K, -1);
                i64 lr = 0;
                for (i32 i = 0; i < m; ++i)
                    for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
                        if (seen[labels[p]] != i) {
                            seen[labels[p]] = i;
                            ++lr;
                        }
                cost_rows = lr;
                cost_cols = cost - lr;
            } else {
                // eRCN: row label = part of its (uncut) nonzeros, K = border
                form = SPMV_DB;
                labels.assign((size_t)m, -1);
                for (i32 i = 0; i < m; ++i) {
                    if (D.row_cut[i]) {
                        labels[i] = K;
                        continue;
                    }
                    if (A->rowptr[i + 1] > A->rowptr[i]) labels[i] = vpart[D.seg_of[A->rowptr[i]]];
                    else labels[i] = (i32)((i64)i * K / std::max<i32>(m, 1));
                }
                cost_cols = cost - cost_rows;
            }
        }
        // derived form
        out->row_perm = (i32 *)std::malloc(sizeof(i32) * (size_t)std::max(m, 1));
        out->col_perm = (i32 *)std::malloc(sizeof(i32) * (size_t)std::max(n, 1));
        out->row_part_ptr = (i32 *)std::malloc(sizeof(i32) * (size_t)(K + 2));
        out->col_part_ptr = (i32 *)std::malloc(sizeof(i32) * (size_t)(K + 2));
        out->labels = (i32 *)std::malloc(sizeof(i32) * std::max<size_t>(labels.size(), 1));
        if (!out->row_perm || !out->col_perm || !out->row_part_ptr || !out->col_part_ptr ||
            !out->labels) {
            spmv_partition_free(out);
            set_error("out of host memory");
            return SPMV_E_NOMEM;
        }
        std::copy(labels.begin(), labels.end(), out->labels);
        st = form_from_labels(A, form, K, labels.data(), out->row_perm, out->col_perm,
                              out->row_part_ptr, out->col_part_ptr);
        if (st != SPMV_OK) {
            spmv_partition_free(out);
            return st;
        }
        if (method == SPMV_PART_RANDOM) {
            // bound of eq. (4) for the random labels
            std::vector<i32> first((size_t)n, -1);
            std::vector<uint8_t> multi((size_t)n, 0);
            std::vector<i32> seen((size_t)n, -1);
            i64 lam = 0;
            for (i32 k = 0; k < K; ++k)
                for (i32 ii = out->row_part_ptr[k]; ii < out->row_part_ptr[k + 1]; ++ii) {
                    const i32 i = out->row_perm[ii];
                    for (i32 p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
                        if (seen[A->colidx[p]] != k) {
                            seen[A->colidx[p]] = k;
                            ++lam;
                        }
                }
            cost = cost_cols = lam;
        }
        out->form = form;
        out->K = K;
        out->n_labels = (i32)labels.size();
        out->cost = cost;
        out->cost_cols = cost_cols;
        out->cost_rows = cost_rows;
        out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return SPMV_OK;
    } catch (const std::bad_alloc &) {
        spmv_partition_free(out);
        set_error("out of host memory");
        return SPMV_E_NOMEM;
    } catch (...) {
        spmv_partition_free(out);
        set_error("internal error in the partitioner");
        return SPMV_E_INTERNAL;
    }
}

extern "C" void spmv_partition_free(spmv_partition_out *out)
{
    if (!out) return;
    std::free(out->labels);
    std::free(out->row_perm);
    std::free(out->col_perm);
    std::free(out->row_part_ptr);
    std::free(out->col_part_ptr);
    out->labels = out->row_perm = out->col_perm = out->row_part_ptr = out->col_part_ptr = nullptr;
}
