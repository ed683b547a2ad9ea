"""The comparison reorderings of Sec. 5.1 (sBFS, sRCM, the separated
block-diagonal order of sHP_RN): the oracle's restatement pinned by a
hand-worked fixture, brute-force level structures and the block structure
itself; the library's orders equal the oracle's; the row-net partition
yields that order."""
import json
import os

import numpy as np
import pytest

import oracle.order as OO
import synth

S = pytest.importorskip("paper_1203_2739_gb300")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "orders_small.json")


def _from_rows(m, n, rows):
    r = np.concatenate([np.full(len(x), i) for i, x in enumerate(rows)] + [np.zeros(0)])
    c = np.concatenate([np.array(x, dtype=np.int64) for x in rows] + [np.zeros(0)])
    return synth.coo_to_csr(m, n, r.astype(np.int64), c.astype(np.int64), np.ones(r.size))


def test_golden_orders():
    g = json.load(open(GOLDEN))
    gg = g["graph"]
    rp, ci, _ = _from_rows(gg["m"], gg["n"], gg["rows"])
    for name, fn in (("bfs", OO.bfs_order), ("rcm", OO.rcm_order)):
        r, c = fn(gg["m"], gg["n"], rp, ci)
        assert r.tolist() == gg[name]["row_perm"] and c.tolist() == gg[name]["col_perm"], name
    s = g["sbd"]
    rp, ci, _ = _from_rows(s["m"], s["n"], s["rows"])
    r, c = OO.sbd_order(s["m"], s["n"], rp, ci, s["K"], s["col_labels"])
    assert r.tolist() == s["row_perm"] and c.tolist() == s["col_perm"]


def _bipartite_dist(m, n, rp, ci, start):
    """Distances from `start` in the bipartite graph by repeated relaxation
    (no queue: an independent way to the same numbers)."""
    INF = 1 << 30
    d = [INF] * (m + n)
    d[start] = 0
    edges = [(i, m + int(ci[p])) for i in range(m) for p in range(int(rp[i]), int(rp[i + 1]))]
    changed = True
    while changed:
        changed = False
        for a, b in edges:
            if d[a] + 1 < d[b]:
                d[b] = d[a] + 1
                changed = True
            if d[b] + 1 < d[a]:
                d[a] = d[b] + 1
                changed = True
    return d


@pytest.mark.parametrize("seed", range(5))
def test_bfs_visits_by_distance(seed):
    """The breadth-first order lists each component's vertices by
    nondecreasing distance from its start (the first vertex of the component
    in the order), components in order of their lowest vertex."""
    m, n = 30, 25
    rp, ci, _ = synth.random_sparse(m, n, 0.06, seed, empty_rows=0.1)
    r, c = OO.bfs_order(m, n, rp, ci)
    assert sorted(r.tolist()) == list(range(m)) and sorted(c.tolist()) == list(range(n))
    pos = {}
    for k, v in enumerate(r.tolist()):
        pos[v] = ("r", k)
    # rebuild the vertex sequence: merge by the BFS rule is not needed; check
    # per component that rows and columns each appear by distance
    seen = set()
    for s in range(m + n):
        if s in seen:
            continue
        d = _bipartite_dist(m, n, rp, ci, s)
        comp = [v for v in range(m + n) if d[v] < (1 << 30)]
        seen.update(comp)
        rows_in = [v for v in r.tolist() if v in comp]
        cols_in = [m + v for v in c.tolist() if (m + v) in comp]
        assert [d[v] for v in rows_in] == sorted(d[v] for v in rows_in)
        assert [d[v] for v in cols_in] == sorted(d[v] for v in cols_in)


@pytest.mark.parametrize("seed", range(4))
def test_rcm_recovers_a_scrambled_bidiagonal(seed):
    """The bipartite graph of a bidiagonal matrix is a path; whatever the
    row and column permutation, reverse Cuthill-McKee walks it from an end,
    so the reordered matrix is bidiagonal again (bandwidth 1)."""
    n = 40
    r = np.r_[np.arange(n), np.arange(n - 1)]
    c = np.r_[np.arange(n), np.arange(1, n)]
    pr, pc = synth.random_perm(n, seed), synth.random_perm(n, seed + 7)
    rp, ci, _ = synth.coo_to_csr(n, n, np.argsort(pr)[r], np.argsort(pc)[c], np.ones(r.size))
    rperm, cperm = OO.rcm_order(n, n, rp, ci)
    ri, cinv = np.argsort(rperm), np.argsort(cperm)
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.abs(cinv[ci] - ri[rows]).max() <= 1


@pytest.mark.parametrize("seed", range(5))
def test_sbd_block_structure(seed):
    """In the separated block-diagonal order, the rows of leaf block k use
    only columns of leaf k, and a separator's rows use columns of both halves
    of its bisection and none outside it; blocks and separators follow the
    in-order walk of the bisection tree."""
    m, n, K = 60, 40, 8
    rp, ci, _ = synth.random_sparse(m, n, 0.05, seed, empty_rows=0.1)
    lab = synth.random_labels(n, K, seed + 1)
    rperm, cperm = OO.sbd_order(m, n, rp, ci, K, lab)
    assert [lab[j] for j in cperm] == sorted(lab.tolist())
    last = -1
    for i in rperm.tolist():
        parts = sorted({int(lab[ci[p]]) for p in range(rp[i], rp[i + 1])})
        if not parts:
            key = 2 * K
        elif len(parts) == 1:
            key = 2 * parts[0]
        else:
            # the smallest aligned interval holding both ends; its midpoint
            size = 2
            while parts[0] // size != parts[-1] // size:
                size *= 2
            lo = parts[0] // size * size
            mid = lo + size // 2
            assert parts[0] < mid <= parts[-1]
            key = 2 * mid - 1
        assert key >= last
        last = key


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(40, 40), (37, 51), (60, 23)])
def test_library_orders_equal_the_oracle(seed, shape):
    m, n = shape
    rp, ci, _ = synth.random_sparse(m, n, 0.05, seed, empty_rows=0.15)
    for meth, fn in ((S.SPMV_ORDER_BFS, OO.bfs_order), (S.SPMV_ORDER_RCM, OO.rcm_order)):
        got = S.spmv_reorder(m, n, rp, ci, meth)
        want = fn(m, n, rp, ci)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), meth
    K = 8
    lab = synth.random_labels(n, K, seed + 3)
    got = S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_SBD, K, lab)
    want = OO.sbd_order(m, n, rp, ci, K, lab)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_row_net_partition_gives_the_sbd_order():
    rp, ci, _ = synth.mesh5(48, seed=2)
    m = n = len(rp) - 1
    out = S.spmv_partition(m, n, rp, ci, S.SPMV_PART_RN, K=16, seed=0)
    assert out["form"] == S.SPMV_NATURAL and out["K"] == 16 and out["labels"].size == n
    rperm, cperm = OO.sbd_order(m, n, rp, ci, 16, out["labels"])
    assert np.array_equal(out["row_perm"], rperm) and np.array_equal(out["col_perm"], cperm)
    # cost: the sum over rows of the number of column parts they touch
    lam = sum(len({int(out["labels"][ci[p]]) for p in range(rp[i], rp[i + 1])})
              for i in range(m))
    assert out["cost"] == lam
    with pytest.raises(S.SpmvError):
        S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_SBD, 12, out["labels"])


# ------------------------------------------------ nested border order ---
def test_golden_nested_border_order():
    s = json.load(open(GOLDEN))["nested"]
    rp, ci, _ = _from_rows(s["m"], s["n"], s["rows"])
    r, c = OO.nested_order(s["m"], s["n"], rp, ci, s["K"], s["row_labels"])
    assert r.tolist() == s["row_perm"] and c.tolist() == s["col_perm"]
    got = S.spmv_reorder(s["m"], s["n"], rp, ci, S.SPMV_ORDER_NESTED, s["K"], s["row_labels"])
    assert got[0].tolist() == s["row_perm"] and got[1].tolist() == s["col_perm"]


def _transpose(m, n, rp, ci):
    r = np.repeat(np.arange(m), np.diff(rp))
    return synth.coo_to_csr(n, m, ci.astype(np.int64), r.astype(np.int64), np.ones(r.size))


@pytest.mark.parametrize("seed", range(4))
def test_nested_order_is_the_sbd_order_of_the_transpose(seed):
    """Without a row border the nested order of A from row parts is the
    separated block-diagonal order of A^T from the same labels on its
    columns, rows and columns exchanged (the pinned sbd_order)."""
    m, n, K = 45, 38, 8
    rp, ci, _ = synth.random_sparse(m, n, 0.06, seed, empty_rows=0.1)
    lab = synth.random_labels(m, K, seed + 7)
    tp, tc, _ = _transpose(m, n, rp, ci)
    r, c = OO.nested_order(m, n, rp, ci, K, lab)
    tr, tcol = OO.sbd_order(n, m, tp, tc, K, lab)
    assert np.array_equal(r, tcol) and np.array_equal(c, tr)


@pytest.mark.parametrize("seed", range(4))
def test_nested_border_sits_between_the_halves(seed):
    """Brute force on the permuted matrix: every column whose rows span parts
    a < b comes after every column of the parts left of the bisection that
    split them and before every column of the parts right of it; R_B rows
    and the columns only R_B touches come last."""
    m, n, K = 60, 50, 8
    rp, ci, _ = synth.random_sparse(m, n, 0.05, seed, empty_rows=0.1)
    lab = synth.random_labels(m, K, seed + 9, border_frac=0.1)
    r, c = OO.nested_order(m, n, rp, ci, K, lab)
    assert [lab[i] for i in r] == sorted(lab)
    pos = np.empty(n, dtype=np.int64)
    pos[c] = np.arange(n)
    spans = {}
    for i in range(m):
        if lab[i] == K:
            continue
        for p in range(rp[i], rp[i + 1]):
            spans.setdefault(int(ci[p]), set()).add(int(lab[i]))
    untouched = [j for j in range(n) if j not in spans]
    assert sorted(pos[untouched].tolist()) == list(range(n - len(untouched), n))
    for j, parts in spans.items():
        a, b = min(parts), max(parts)
        if a == b:
            continue
        size = 2
        while a // size != b // size:
            size *= 2
        lo = a // size * size
        mid = lo + size // 2
        for k, ps in spans.items():
            if len(ps) == 1:
                (q,) = ps
                if lo <= q < mid:
                    assert pos[k] < pos[j]
                elif mid <= q < lo + size:
                    assert pos[k] > pos[j]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(40, 40), (37, 51), (60, 23)])
def test_library_nested_order_equals_the_oracle(seed, shape):
    m, n = shape
    rp, ci, _ = synth.random_sparse(m, n, 0.05, seed, empty_rows=0.15)
    for K, frac in ((8, 0.0), (16, 0.15), (1, 0.2)):
        lab = synth.random_labels(m, K, seed + 5, border_frac=frac)
        got = S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_NESTED, K, lab)
        want = OO.nested_order(m, n, rp, ci, K, lab)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    with pytest.raises(S.SpmvError):
        S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_NESTED, 12, synth.random_labels(m, 12, 1))
    with pytest.raises(S.SpmvError):
        bad = synth.random_labels(m, 8, 2)
        bad[0] = 9
        S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_NESTED, 8, bad)


def test_nested_fixture_catches_planted_mistakes():
    """The nested fixture separates the oracle from plausible wrong readings:
    counting R_B's rows in a column's parts, placing a cut column by its
    lowest part instead of its bisection, and leaving untouched columns in
    index order among the others."""
    s = json.load(open(GOLDEN))["nested"]
    rp, ci, _ = _from_rows(s["m"], s["n"], s["rows"])
    m, n, K, lab = s["m"], s["n"], s["K"], s["row_labels"]

    def parts_of(j, with_border):
        return [lab[i] for i in range(m) for p in range(rp[i], rp[i + 1])
                if ci[p] == j and (with_border or lab[i] < K)]

    def order(key):
        return sorted(range(n), key=lambda j: (key(j), j))

    def with_border(j):
        # R_B's rows counted as a part K; the split leaf from the highest
        # differing bit, as a bitwise implementation would compute it
        ps = parts_of(j, True)
        if not ps:
            return 2 * K
        a, b = min(ps), max(ps)
        if a == b:
            return 2 * a
        hb = (a ^ b).bit_length() - 1
        return 2 * ((b >> hb) << hb) - 1

    def lowest_part(j):
        ps = parts_of(j, False)
        return 2 * K if not ps else 2 * min(ps)

    def untouched_inline(j):
        ps = parts_of(j, False)
        if not ps:
            return -1
        a, b = min(ps), max(ps)
        return 2 * a if a == b else OO._between(a, b, K)

    for wrong in (with_border, lowest_part, untouched_inline):
        assert order(wrong) != s["col_perm"], wrong.__name__
