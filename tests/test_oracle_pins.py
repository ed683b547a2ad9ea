"""Pins of the CPU oracle against facts that do not come from the oracle:
brute force on tiny inputs, closed forms, exact integer arithmetic, and
hand-worked fixtures in tests/golden (each citing the passage it follows)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _small_from_rows(g):
    m, n = g["m"], g["n"]
    rows = [np.full(len(r), i) for i, r in enumerate(g["rows"])]
    r = np.concatenate(rows)
    c = np.concatenate([np.array(x) for x in g["rows"]])
    v = np.arange(1, r.size + 1, dtype=np.float64)
    return (m, n) + synth.coo_to_csr(m, n, r, c, v)


def _dense(m, n, rp, ci, v):
    return synth.csr_to_dense(m, n, rp, ci, v)


# ------------------------------------------------------------------ SpMV ---

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(1, 1), (7, 13), (33, 17), (64, 64), (5, 64)])
def test_spmv_equals_dense_matvec_exactly(seed, shape):
    """Brute force: with small integers every FP64 sum is exact, so the CSR
    definition must equal the dense product bit for bit (Sec. 2.1)."""
    m, n = shape
    rp, ci, v = synth.random_sparse(m, n, 0.3, seed, integer=True, empty_rows=0.2)
    A = _dense(m, n, rp, ci, v)
    x = synth.integer_x(n, seed + 1)
    y, a = oracle.spmv(m, n, rp, ci, v, x)
    assert np.array_equal(y, A @ x)
    assert np.array_equal(a, np.abs(A) @ np.abs(x))
    X = synth.integer_x(n, seed + 2, nrhs=3)
    Y, _ = oracle.spmv(m, n, rp, ci, v, X)
    assert np.array_equal(Y, A @ X)


@pytest.mark.parametrize("seed", range(4))
def test_plain_loop_equals_dense_matvec_exactly(seed):
    """The timed plain CSR loop (Sec. 2.1) is the dense product by brute force
    with exact integer data, on one thread and on every host thread; and it
    is a running left-to-right sum (1e16 + 1 - 1e16 gives 0, where the
    compensated checker gives 1)."""
    m, n = 300, 211
    rp, ci, v = synth.random_sparse(m, n, 0.1, seed, integer=True, empty_rows=0.2)
    A = _dense(m, n, rp, ci, v)
    x = synth.integer_x(n, seed + 1)
    rp64 = np.ascontiguousarray(rp, dtype=np.int64)
    for threads in (1, oracle.plain_max_threads()):
        y = oracle.spmv_plain(m, rp64, np.ascontiguousarray(ci, dtype=np.int32), v, x, threads)
        assert np.array_equal(y, A @ x)
    y = oracle.spmv_plain(1, np.array([0, 3], dtype=np.int64), np.array([0, 1, 2], np.int32),
                          np.array([1e16, 1.0, -1e16]), np.ones(3))
    assert y[0] == 0.0


def test_spmv_sums_are_compensated():
    """The oracle's row sums carry a running error term (Neumaier), so
    cancellation that a plain left-to-right FP64 sum gets wrong comes out
    exact: 1e16 + 1 - 1e16 = 1 (plain: 0), and the sum of 10^5 copies of 0.1
    after 1e8 matches the exactly rounded value."""
    rp = np.array([0, 3, 6], dtype=np.int64)
    ci = np.array([0, 1, 2, 0, 1, 2], dtype=np.int32)
    v = np.array([1e16, 1.0, -1e16, 1.0, 1e16, -1e16])
    y, a = oracle.spmv(2, 3, rp, ci, v, np.ones(3))
    assert y[0] == 1.0 and y[1] == 1.0
    assert a[0] == 2e16 + 1.0
    k = 100_000
    rp = np.array([0, k + 1], dtype=np.int64)
    ci = np.arange(k + 1, dtype=np.int32)
    v = np.r_[1e8, np.full(k, 0.1)]
    y, _ = oracle.spmv(1, k + 1, rp, ci, v, np.ones(k + 1))
    from fractions import Fraction
    exact = Fraction(1e8) + k * Fraction(0.1)
    assert y[0] == float(exact)


def test_spmv_laplacian_eigenvector_closed_form():
    """Dirichlet 3D Laplacian: v = sin(i pi a/(N+1)) sin(j pi b/(N+1))
    sin(k pi c/(N+1)) is an eigenvector with eigenvalue
    sum(2 - 2 cos(. pi/(N+1))); this holds in any symmetric permutation."""
    N = 8
    rp, ci, v = synth.laplacian3d(N, permute=False)
    n = N ** 3
    a = np.arange(1, N + 1)
    for (i, j, k) in [(1, 1, 1), (2, 5, 7), (8, 3, 1)]:
        vx = np.sin(i * np.pi * a / (N + 1))
        vy = np.sin(j * np.pi * a / (N + 1))
        vz = np.sin(k * np.pi * a / (N + 1))
        vec = (vz[:, None, None] * vy[None, :, None] * vx[None, None, :]).reshape(-1)
        lam = sum(2 - 2 * np.cos(t * np.pi / (N + 1)) for t in (i, j, k))
        y, _ = oracle.spmv(n, n, rp, ci, v, vec)
        assert np.max(np.abs(y - lam * vec)) < 1e-13 * lam
        perm = synth.random_perm(n, 3)
        prp, pci, pv = oracle.permute(n, n, rp, ci, v, perm, perm)
        yp, _ = oracle.spmv(n, n, prp, pci, pv, vec[perm])
        assert np.max(np.abs(yp - lam * vec[perm])) < 1e-13 * lam


def test_laplacian_row_sums():
    """A 1 = 6 - (number of in-grid neighbours) for the 7-point stencil."""
    N = 6
    rp, ci, v = synth.laplacian3d(N, permute=False)
    y, _ = oracle.spmv(N ** 3, N ** 3, rp, ci, v, np.ones(N ** 3))
    g = np.arange(N ** 3)
    gx, gy, gz = g % N, (g // N) % N, g // (N * N)
    boundary = sum(((t == 0).astype(int) + (t == N - 1).astype(int)) for t in (gx, gy, gz))
    assert np.array_equal(y, boundary.astype(np.float64))


# --------------------------------------------------------- permutations ---

@pytest.mark.parametrize("seed", range(5))
def test_permutation_invariant_exact(seed):
    """P_r^T (P_r A P_c)(P_c^T x) = A x bit-exactly with integer data (Sec. 3)."""
    m, n = 40, 29
    rp, ci, v = synth.random_sparse(m, n, 0.25, seed, integer=True)
    A = _dense(m, n, rp, ci, v)
    rperm, cperm = synth.random_perm(m, seed + 11), synth.random_perm(n, seed + 12)
    prp, pci, pv = oracle.permute(m, n, rp, ci, v, rperm, cperm)
    # the permuted matrix is the dense matrix indexed by the perms (brute force)
    assert np.array_equal(_dense(m, n, prp, pci, pv), A[rperm][:, cperm])
    assert all(np.all(np.diff(pci[prp[i]:prp[i + 1]]) > 0) for i in range(m))
    x = synth.integer_x(n, seed)
    yh, _ = oracle.spmv(m, n, prp, pci, pv, x[cperm])
    y = np.empty(m)
    y[rperm] = yh
    assert np.array_equal(y, A @ x)


def test_is_perm():
    assert oracle.is_perm(np.array([2, 0, 1]))
    assert not oracle.is_perm(np.array([0, 0, 1]))
    assert not oracle.is_perm(np.array([0, 3, 1]))
    assert not oracle.is_perm(np.array([-1, 0, 1]))


# ----------------------------------------------------------------- forms ---

def test_sb_form_golden():
    g = _golden("forms_small.json")
    m, n, rp, ci, v = _small_from_rows(g)
    s = g["sb"]
    rperm, cperm, rptr, cptr = oracle.form_rows(m, n, rp, ci, s["K"], s["labels"])
    assert rperm.tolist() == s["row_perm"]
    assert cperm.tolist() == s["col_perm"]
    assert rptr.tolist() == s["row_part_ptr"]
    assert cptr.tolist() == s["col_part_ptr"]
    lam, _ = oracle.lambda_rows(m, n, rp, ci, s["K"], s["labels"])
    assert lam.tolist() == s["lambda"]
    assert oracle.bound_sb(m, n, rp, ci, s["K"], s["labels"]) == s["bound_eq4"]
    bad, _ = oracle.check_structure(m, n, rp, ci, rperm, cperm, s["K"], rptr, cptr)
    assert bad == 0


def test_db_form_golden():
    g = _golden("forms_small.json")
    m, n, rp, ci, v = _small_from_rows(g)
    s = g["db"]
    rperm, cperm, rptr, cptr = oracle.form_rows(m, n, rp, ci, s["K"], s["labels"], border=True)
    assert rperm.tolist() == s["row_perm"]
    assert cperm.tolist() == s["col_perm"]
    assert rptr.tolist() == s["row_part_ptr"]
    assert cptr.tolist() == s["col_part_ptr"]
    lam, _ = oracle.lambda_rows(m, n, rp, ci, s["K"], s["labels"])
    assert lam.tolist() == s["lambda_prime"]
    assert oracle.bound_db(m, n, rp, ci, s["K"], s["labels"]) == s["bound_eq6"]
    bad, _ = oracle.check_structure(m, n, rp, ci, rperm, cperm, s["K"], rptr, cptr)
    assert bad == 0


@pytest.mark.parametrize("which", ["sb", "db"])
def test_border_order_golden(which):
    """The order of the coupling columns inside the border, hand-derived
    (tests/golden/forms_small.json, "border_order")."""
    g = _golden("forms_small.json")["border_order"]
    m, n, rp, ci, v = _small_from_rows(g)
    s = g[which]
    rperm, cperm, rptr, cptr = oracle.form_rows(m, n, rp, ci, s["K"], s["labels"],
                                                border=which == "db")
    assert rperm.tolist() == s["row_perm"] and rptr.tolist() == s["row_part_ptr"]
    assert cperm.tolist() == s["col_perm"] and cptr.tolist() == s["col_part_ptr"]


def test_split_golden():
    g = _golden("forms_small.json")
    m, n, rp, ci, v = _small_from_rows(g)
    s = g["split"]
    K = s["K"]
    lr, lc = oracle.lambda_split(m, n, rp, ci, K, s["nz_part"])
    assert lr.tolist() == s["lambda_r"] and lc.tolist() == s["lambda_c"]
    assert oracle.bound_split(m, n, rp, ci, K, s["nz_part"]) == (s["bound_x"], s["bound_y"])
    rperm, cperm, rptr, cptr = oracle.form_split(m, n, rp, ci, K, s["nz_part"])
    assert rperm.tolist() == s["row_perm"] and cperm.tolist() == s["col_perm"]
    assert rptr.tolist() == s["row_part_ptr"] and cptr.tolist() == s["col_part_ptr"]
    prp, prows, gptr, pos = oracle.split_parts(m, rp, K, s["nz_part"])
    assert prp.tolist() == s["part_row_ptr"] and prows.tolist() == s["part_rows"]
    assert gptr.tolist() == s["gcsr_ptr"] and pos.tolist() == s["nz_pos"]


def _brute_lambda(A, labels, K):
    m, n = A.shape
    return [len({labels[i] for i in range(m) if A[i, j] != 0 and 0 <= labels[i] < K})
            for j in range(n)]


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("border", [False, True])
def test_row_forms_bruteforce(seed, border):
    """Random labels: the derived form obeys eqs. (1)-(3)/(5) by brute force."""
    m, n, K = 37, 31, 4
    rp, ci, v = synth.random_sparse(m, n, 0.12, seed, integer=True, empty_rows=0.1)
    A = _dense(m, n, rp, ci, v)
    labels = synth.random_labels(m, K, seed + 5, border_frac=0.2 if border else 0.0)
    rperm, cperm, rptr, cptr = oracle.form_rows(m, n, rp, ci, K, labels, border=border)
    assert oracle.is_perm(rperm) and oracle.is_perm(cperm)
    lam = _brute_lambda(A, labels, K)
    # rows: grouped by label, increasing inside each group, border last
    for k in range(K + 1):
        block = rperm[rptr[k]:rptr[k + 1]].tolist()
        assert block == sorted(i for i in range(m) if labels[i] == k)
    # columns: C_k exactly the lambda=1 columns of part k, in index order
    for k in range(K):
        ck = cperm[cptr[k]:cptr[k + 1]].tolist()
        expect = [j for j in range(n) if lam[j] == 1 and
                  any(A[i, j] != 0 and labels[i] == k for i in range(m))]
        assert ck == expect
    cb = cperm[cptr[K]:cptr[K + 1]].tolist()
    # the border: coupling columns by the part holding most of their
    # nonzeros (lower part on ties), then index; untouched columns last
    def majority(j):
        cnt = [sum(1 for i in range(m) if A[i, j] != 0 and labels[i] == k) for k in range(K)]
        return max(range(K), key=lambda k: (cnt[k], -k))
    assert cb == sorted((j for j in range(n) if lam[j] >= 2), key=lambda j: (majority(j), j)) \
        + [j for j in range(n) if lam[j] == 0]
    # structure rule by brute force on the permuted dense matrix
    Ah = A[rperm][:, cperm]
    for k in range(K):
        blk = Ah[rptr[k]:rptr[k + 1]]
        allowed = np.zeros(n, bool)
        allowed[cptr[k]:cptr[k + 1]] = True
        allowed[cptr[K]:] = True
        assert not np.any(blk[:, ~allowed])
    bad, _ = oracle.check_structure(m, n, rp, ci, rperm, cperm, K, rptr, cptr)
    assert bad == 0
    bound = oracle.bound_db(m, n, rp, ci, K, labels) if border else \
        oracle.bound_sb(m, n, rp, ci, K, labels)
    extra = sum(int(np.count_nonzero(A[i])) for i in range(m) if labels[i] == K)
    assert bound == sum(lam) + extra


def test_structure_validator_catches_a_planted_violation():
    g = _golden("forms_small.json")
    m, n, rp, ci, v = _small_from_rows(g)
    s = g["sb"]
    rperm, cperm, rptr, cptr = oracle.form_rows(m, n, rp, ci, s["K"], s["labels"])
    bad_cperm = cperm.copy()
    # move column 2 (in C_0) into C_1's place and column 1 (in C_1) into C_0's
    a, b = list(bad_cperm).index(2), list(bad_cperm).index(1)
    bad_cperm[a], bad_cperm[b] = bad_cperm[b], bad_cperm[a]
    bad, first = oracle.check_structure(m, n, rp, ci, rperm, bad_cperm, s["K"], rptr, cptr)
    assert bad > 0 and first[0] >= 0


@pytest.mark.parametrize("seed", range(6))
def test_split_bruteforce(seed):
    """Sum of the A^k equals A exactly and the parts are nonzero-disjoint
    (Sec. 4); lambda counts and first-touch order by brute force."""
    m, n, K = 30, 26, 5
    rp, ci, v = synth.random_sparse(m, n, 0.15, seed, integer=True, empty_rows=0.1)
    A = _dense(m, n, rp, ci, v)
    nnz = int(rp[-1])
    part = synth.random_labels(nnz, K, seed + 9)
    prp, prows, gptr, pos = oracle.split_parts(m, rp, K, part)
    assert sorted(pos.tolist()) == list(range(nnz))
    rows_of = np.repeat(np.arange(m), np.diff(rp))
    S = np.zeros_like(A)
    x = synth.integer_x(n, seed)
    y = np.zeros(m)
    for k in range(K):
        Ak = np.zeros_like(A)
        rows_k = prows[prp[k]:prp[k + 1]]
        assert np.all(np.diff(rows_k) > 0)
        for t in range(prp[k], prp[k + 1]):
            for q in range(gptr[t], gptr[t + 1]):
                p = pos[q]
                assert part[p] == k and rows_of[p] == prows[t]
                Ak[rows_of[p], ci[p]] = v[p]
        assert np.array_equal(np.nonzero(Ak.any(axis=1))[0], rows_k)
        S += Ak
        y = y + Ak @ x
    assert np.array_equal(S, A)
    assert np.array_equal(y, A @ x)
    lr, lc = oracle.lambda_split(m, n, rp, ci, K, part)
    brute_r = [len({part[p] for p in range(rp[i], rp[i + 1])}) for i in range(m)]
    brute_c = [len({part[p] for p in range(nnz) if ci[p] == j}) for j in range(n)]
    assert lr.tolist() == brute_r and lc.tolist() == brute_c
    rperm, cperm, rptr, cptr = oracle.form_split(m, n, rp, ci, K, part)
    first_r = [min([part[p] for p in range(rp[i], rp[i + 1])], default=K) for i in range(m)]
    assert rperm.tolist() == sorted(range(m), key=lambda i: (first_r[i], i))
    first_c = [min([part[p] for p in range(nnz) if ci[p] == j], default=K) for j in range(n)]
    assert cperm.tolist() == sorted(range(n), key=lambda j: (first_c[j], j))


# -------------------------------------------------------------- fitting ---

def test_csr_sizes_reproduce_table1_range():
    g = _golden("table1_csr_sizes.json")
    for c in g["cases"]:
        size = oracle.part_bytes(c["rows"], c["nnz"], 0, xb=0, yb=0)
        assert round(size / 1e6) == c["mb"], c


def test_fits_is_strict():
    assert oracle.fits(99, 100) and not oracle.fits(100, 100)
    assert oracle.part_bytes(2, 3, 4) == 3 * 12 + 3 * 4 + 4 * 8 + 2 * 8
    assert oracle.part_bytes(2, 3, 4, gcsr=True) == oracle.part_bytes(2, 3, 4) + 8


# ------------------------------------------------------- cache simulator ---

def test_lru_golden_traces():
    g = _golden("lru_traces.json")
    for t in g["traces"]:
        el = np.array(t["elements"])
        out = oracle.cachesim_trace(np.zeros(el.size), el, t["lines"] * t["line_bytes"],
                                    t["line_bytes"])
        assert out[0] == t["misses"], t


def _textbook_lru(arrays, indices, lines, line_bytes):
    """Fully associative LRU over (array, line) keys with an ordered dict:
    a hit moves the line to the back, a miss evicts the front when full."""
    from collections import OrderedDict
    cache, misses = OrderedDict(), np.zeros(6, dtype=np.int64)
    for a, i in zip(arrays, indices):
        key = (int(a), int(i) * 8 // line_bytes)
        if key in cache:
            cache.move_to_end(key)
            continue
        misses[a] += 1
        cache[key] = True
        if len(cache) > lines:
            cache.popitem(last=False)
    return misses


@pytest.mark.parametrize("seed", range(6))
def test_lru_matches_a_textbook_lru_on_random_traces(seed):
    """The simulator's hashed, linked-list LRU against an ordered-dict LRU
    on random traces of several arrays, for several capacities and lines."""
    rng = np.random.default_rng(seed)
    n = 3000
    arrays = rng.integers(0, 6, n).astype(np.int32)
    # a skewed index mix: some reuse at every distance
    indices = np.where(rng.random(n) < 0.5, rng.integers(0, 40, n),
                       rng.integers(0, 2000, n)).astype(np.int64)
    for line_bytes in (8, 64):
        for lines in (1, 2, 7, 64, 500):
            got = oracle.cachesim_trace(arrays, indices, lines * line_bytes, line_bytes)
            want = _textbook_lru(arrays, indices, lines, line_bytes)
            assert np.array_equal(got, want), (line_bytes, lines)


@pytest.mark.parametrize("seed", range(3))
def test_lru_compulsory_misses_when_everything_fits(seed):
    rp, ci, v = synth.random_sparse(50, 60, 0.1, seed)
    out = oracle.cachesim_csr(50, rp, ci, cache_bytes=1 << 20, line_bytes=8)
    nnz = int(rp[-1])
    assert out["x"] == len(set(ci.tolist()))
    assert out["y"] == 50
    assert out["val"] == nnz
    assert out["col"] == (nnz + 1) // 2 if nnz else True
    assert out["rowptr"] == 26          # 51 four-byte entries over 8-byte lines


def _gcsr_trace(part_rows, gptr, gcol, drop_y=False):
    """The access order of the multiple SpMxV over GCSR parts (Sec. 4, GCSR
    Sec. 5.2), written out: per stored row t its row-list entry, its two row
    starts, per nonzero its column index, value and x entry, then its y
    entry; (array id, element, element bytes) with the simulator's array ids
    (0 rowptr, 1 col, 2 val, 3 x, 4 y, 5 rowlist)."""
    tr = []
    for t in range(len(part_rows)):
        tr += [(5, t, 4), (0, t, 4), (0, t + 1, 4)]
        for q in range(int(gptr[t]), int(gptr[t + 1])):
            tr += [(1, q, 4), (2, q, 8), (3, int(gcol[q]), 8)]
        if not drop_y:
            tr.append((4, int(part_rows[t]), 8))
    return tr


def _textbook_replay(trace, lines, line_bytes):
    from collections import OrderedDict
    cache, misses = OrderedDict(), np.zeros(6, dtype=np.int64)
    for a, i, es in trace:
        key = (a, i * es // line_bytes)
        if key in cache:
            cache.move_to_end(key)
            continue
        misses[a] += 1
        cache[key] = True
        if len(cache) > lines:
            cache.popitem(last=False)
    return misses


def test_gcsr_lru_golden_trace():
    """A hand-worked GCSR replay (tests/golden/lru_traces.json)."""
    g = _golden("lru_traces.json")["gcsr"]
    for c in g["cases"]:
        out = oracle.cachesim_gcsr(g["part_rows"], g["gcsr_ptr"], g["gcsr_col"],
                                   c["lines"] * c["line_bytes"], c["line_bytes"])
        got = [out[k] for k in oracle.ARRAYS]
        assert got == c["misses"], c


@pytest.mark.parametrize("seed", range(4))
def test_gcsr_lru_compulsory_misses_when_everything_fits(seed):
    """With a cache larger than everything the replay touches, each array
    misses once per distinct line: row list ceil(4T/L), row starts
    ceil(4(T+1)/L), columns ceil(4 nnz/L), values ceil(8 nnz/L), x and y the
    distinct lines of the columns and rows touched."""
    m, n, K = 70, 90, 4
    rp, ci, v = synth.random_sparse(m, n, 0.08, seed)
    nnz = int(rp[-1])
    part = synth.random_labels(nnz, K, seed + 3)
    prp, prows, gptr, pos = oracle.split_parts(m, rp, K, part)
    gcol = ci[pos]
    T = len(prows)
    for L in (8, 64):
        out = oracle.cachesim_gcsr(prows, gptr, gcol, 1 << 22, L)
        assert out["rowlist"] == -(-4 * T // L)
        assert out["rowptr"] == -(-4 * (T + 1) // L)
        assert out["col"] == -(-4 * nnz // L)
        assert out["val"] == -(-8 * nnz // L)
        assert out["x"] == len({8 * int(c) // L for c in gcol})
        assert out["y"] == len({8 * int(i) // L for i in prows})


@pytest.mark.parametrize("seed", range(4))
def test_gcsr_lru_matches_the_written_out_access_order(seed):
    """The C replay against the access order of Sec. 4 written out in Python
    and an ordered-dict LRU, for several capacities and line sizes; the same
    comparison tells a replay that drops the y accesses apart."""
    m, n, K = 60, 50, 5
    rp, ci, v = synth.random_sparse(m, n, 0.1, seed)
    nnz = int(rp[-1])
    part = synth.random_labels(nnz, K, seed + 1)
    prp, prows, gptr, pos = oracle.split_parts(m, rp, K, part)
    gcol = ci[pos]
    tr = _gcsr_trace(prows, gptr, gcol)
    no_y = _gcsr_trace(prows, gptr, gcol, drop_y=True)
    for L in (8, 64):
        for lines in (1, 3, 16, 200):
            out = oracle.cachesim_gcsr(prows, gptr, gcol, lines * L, L)
            got = np.array([out[k] for k in oracle.ARRAYS])
            assert np.array_equal(got, _textbook_replay(tr, lines, L)), (L, lines)
            assert not np.array_equal(got, _textbook_replay(no_y, lines, L)), (L, lines)


def _sb_parts_sizes(m, n, rp, ci, K, labels):
    sizes = []
    for k in range(K):
        rows = [i for i in range(m) if labels[i] == k]
        nnz = sum(int(rp[i + 1] - rp[i]) for i in rows)
        cols = len({int(c) for i in rows for c in ci[rp[i]:rp[i + 1]]})
        sizes.append(oracle.part_bytes(len(rows), nnz, cols))
    return sizes


@pytest.mark.parametrize("seed", range(4))
def test_theorem1_bound_holds_in_simulator(seed):
    """Eq. (4): if every R_k fits, x misses <= sum_j lambda(c_j)."""
    m, n, K = 120, 100, 6
    rp, ci, v = synth.random_sparse(m, n, 0.05, seed)
    labels = synth.random_labels(m, K, seed)
    rperm, cperm, rptr, cptr = oracle.form_rows(m, n, rp, ci, K, labels)
    prp, pci, _ = oracle.permute(m, n, rp, ci, v, rperm, cperm)
    cache = max(_sb_parts_sizes(m, n, rp, ci, K, labels)) + 64
    miss = oracle.cachesim_csr(m, prp, pci, cache, 8)
    bound = oracle.bound_sb(m, n, rp, ci, K, labels)
    assert miss["x"] <= bound
    # the bound is not vacuous: a single part (K=1) would allow only n misses
    assert bound > len(set(ci.tolist()))


@pytest.mark.parametrize("seed", range(4))
def test_theorem2_bound_holds_in_simulator(seed):
    """Eq. (6): if every R_k of A'_SB fits, x misses <= sum lambda' + nnz(R_B)."""
    m, n, K = 120, 100, 6
    rp, ci, v = synth.random_sparse(m, n, 0.05, seed)
    labels = synth.random_labels(m, K, seed, border_frac=0.15)
    rperm, cperm, rptr, cptr = oracle.form_rows(m, n, rp, ci, K, labels, border=True)
    prp, pci, _ = oracle.permute(m, n, rp, ci, v, rperm, cperm)
    cache = max(_sb_parts_sizes(m, n, rp, ci, K, labels)) + 64
    miss = oracle.cachesim_csr(m, prp, pci, cache, 8)
    assert miss["x"] <= oracle.bound_db(m, n, rp, ci, K, labels)


@pytest.mark.parametrize("seed", range(4))
def test_theorem3_bounds_hold_in_simulator(seed):
    """Theorem 3: (a) x misses <= sum lambda(c_j) when each A^k fits;
    (b) y misses <= sum lambda(r_i) with any cache size."""
    m, n, K = 90, 80, 5
    rp, ci, v = synth.random_sparse(m, n, 0.06, seed)
    nnz = int(rp[-1])
    part = synth.random_labels(nnz, K, seed + 1)
    prp, prows, gptr, pos = oracle.split_parts(m, rp, K, part)
    gcol = ci[pos]
    sizes = []
    for k in range(K):
        t0, t1 = prp[k], prp[k + 1]
        sizes.append(oracle.part_bytes(int(t1 - t0), int(gptr[t1] - gptr[t0]),
                                       len(set(gcol[gptr[t0]:gptr[t1]].tolist())), gcsr=True))
    bx, by = oracle.bound_split(m, n, rp, ci, K, part)
    miss = oracle.cachesim_gcsr(prows, gptr, gcol, max(sizes) + 64, 8)
    assert miss["x"] <= bx and miss["y"] <= by
    tiny = oracle.cachesim_gcsr(prows, gptr, gcol, 8 * 4, 8)
    assert tiny["y"] <= by


# -------------------------------------------------------------------- CG ---

def test_cg_solves_spd_system():
    N = 6
    rp, ci, v = synth.laplacian3d(N, permute=True, seed=1)
    n = N ** 3
    A = _dense(n, n, rp, ci, v)
    xs = synth.uniform_x(n, 0)
    b = A @ xs
    x, it, rel = oracle.cg(n, rp, ci, v, b, tol=1e-12)
    assert rel <= 1e-12
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    assert np.max(np.abs(x - xs)) < 1e-9


# ------------------------------------------------------------ generators ---

def test_generator_closed_form_sizes():
    rp, ci, v = synth.mesh5(16, seed=0)
    assert rp[-1] == 5 * 16 * 16 - 4 * 16
    rp, ci, v = synth.laplacian3d(8)
    assert rp[-1] == 7 * 8 ** 3 - 6 * 8 ** 2
    rp, ci, v = synth.rmat(scale=10, deg=16, seed=0)
    assert rp[-1] == 16 * 1024
    for rpi, cii in [(rp, ci)]:
        for i in range(len(rpi) - 1):
            assert np.all(np.diff(cii[rpi[i]:rpi[i + 1]]) > 0)
    rp, ci, v = synth.blocks(nb=4, bs=64, fill=0.05, border_frac=0.05, seed=0, permute=False)
    per = int(round(0.05 * 64 * 64))
    assert rp[-1] == 4 * per + int(round(0.05 * per * 4))


def test_zipf_row_degrees():
    rp, ci, v = synth.zipf_matrix(m=2048, n=2048, seed=0)
    deg = np.diff(rp)
    assert deg.max() <= 512 and deg.min() >= 1
    assert 6.5 < deg.mean() < 9.5


# ------------------------------------------------ selector MLP (extension) ---
def _mlp_params(rng, nin, nh, nc, scale=0.5):
    return [rng.normal(0, scale, (nh, nin)), rng.normal(0, scale, nh),
            rng.normal(0, scale, (nh, nh)), rng.normal(0, scale, nh),
            rng.normal(0, scale, (nc, nh)), rng.normal(0, scale, nc)]


def test_mlp_gradients_match_finite_differences():
    # central differences of the loss pin every gradient, independently of
    # the chain-rule code under test
    rng = np.random.default_rng(5)
    nin, nh, nc, batch = 3, 4, 3, 5
    X = rng.normal(0, 1, (batch, nin))
    y = rng.integers(0, nc, batch)
    params = _mlp_params(rng, nin, nh, nc)
    _, _, grads = oracle.mlp_loss_grad(X, y, params)
    h = 1e-6
    for p, g in zip(params, grads):
        flat, gflat = p.reshape(-1), g.reshape(-1)
        for k in range(flat.size):
            old = flat[k]
            flat[k] = old + h
            lp = oracle.mlp_loss_grad(X, y, params, grads=False)[0]
            flat[k] = old - h
            lm = oracle.mlp_loss_grad(X, y, params, grads=False)[0]
            flat[k] = old
            assert abs((lp - lm) / (2 * h) - gflat[k]) <= 1e-7 * max(1.0, abs(gflat[k]))


def test_mlp_loss_closed_forms():
    rng = np.random.default_rng(6)
    nin, nh, nc, batch = 4, 5, 7, 6
    X = rng.normal(0, 1, (batch, nin))
    y = rng.integers(0, nc, batch)
    zero = [np.zeros_like(p) for p in _mlp_params(rng, nin, nh, nc)]
    loss, logits, grads = oracle.mlp_loss_grad(X, y, zero)
    # all logits zero: softmax uniform, loss log(nc); only b3 gets a gradient
    assert abs(loss - np.log(nc)) < 1e-14 and not np.any(logits)
    onehot = np.zeros((batch, nc))
    onehot[np.arange(batch), y] = 1.0
    assert np.allclose(grads[5], (1.0 / nc - onehot).mean(axis=0), atol=1e-15)
    assert not np.any(grads[0]) and not np.any(grads[4])
    # a network that only passes b3: logits = b3 for every sample
    b3 = rng.normal(0, 1, nc)
    loss, logits, _ = oracle.mlp_loss_grad(X, y, zero[:5] + [b3])
    lse = np.log(np.exp(b3).sum())
    assert abs(loss - np.mean(lse - b3[y])) < 1e-13
    assert np.allclose(logits, np.tile(b3, (batch, 1)))
