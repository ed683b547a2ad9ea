"""The oracle's restatement of ICSR (Sec. 2.1), pinned by a hand-worked
example, the round trip to CSR, and the product against a dense
brute-force one on matrices with many empty rows (the case ICSR serves in
the multiple-SpMxV framework, Sec. 4)."""
import json
import os

import numpy as np
import pytest

import oracle.icsr as IC
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "icsr_small.json")


def _csr(m, n, rows):
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], dtype=np.int64)
    return rp, ci


def test_golden_example():
    g = json.load(open(GOLDEN))
    rp, ci = _csr(g["m"], g["n"], g["rows"])
    cd, rj = IC.icsr_encode(g["m"], g["n"], rp, ci)
    assert cd.tolist() == g["col_diff"] and rj.tolist() == g["row_jump"]
    y = IC.icsr_spmv(g["m"], g["n"], cd, rj, g["vals"], g["x"])
    assert y.tolist() == g["y"]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(30, 30), (17, 90), (80, 5)])
def test_round_trip_and_product(seed, shape):
    m, n = shape
    rp, ci, v = synth.random_sparse(m, n, 0.08, seed, empty_rows=0.4)
    cd, rj = IC.icsr_encode(m, n, rp, ci)
    # one increment per nonzero, one jump per nonzero row
    assert cd.size == rp[-1] and rj.size == int(np.count_nonzero(np.diff(rp)))
    rp2, ci2 = IC.icsr_decode(m, n, cd, rj)
    assert np.array_equal(rp2, rp) and np.array_equal(ci2, ci)
    x = synth.integer_x(n, seed + 10)
    dense = synth.csr_to_dense(m, n, rp, ci, v)
    assert np.array_equal(IC.icsr_spmv(m, n, cd, rj, v, x), dense @ x)
    # sorted unique columns: increments inside a row are >= 1; the first of
    # a later row is col - previous col + n, in [1, 2n - 1]
    first = np.zeros(int(rp[-1]), dtype=bool)
    first[rp[:-1][np.diff(rp) > 0]] = True
    first[rp[:-1][np.diff(rp) > 0][0]] = False
    assert np.all(cd[~first][1:] >= 1)
    assert np.all((cd[first] >= 1) & (cd[first] <= 2 * n - 1))


def test_empty_and_single_row():
    assert IC.icsr_spmv(4, 3, [], [], [], [1, 2, 3]).tolist() == [0, 0, 0, 0]
    cd, rj = IC.icsr_encode(3, 5, [0, 0, 0, 3], [0, 2, 4])
    assert cd.tolist() == [0, 2, 2] and rj.tolist() == [2]


def test_fixture_catches_planted_mistakes():
    """The hand-worked fixture separates the oracle from plausible wrong
    readings: no extra n at a row change (the loop cannot see row ends),
    absolute row indices in rowJump instead of increments, and a running
    column that restarts at every row."""
    g = json.load(open(GOLDEN))
    rp, ci = _csr(g["m"], g["n"], g["rows"])
    cd, rj = IC.icsr_encode(g["m"], g["n"], rp, ci)

    def no_signal(m, n, rowptr, colidx):
        c = np.asarray(colidx, dtype=np.int64)
        return np.diff(np.r_[0, c]), IC.icsr_encode(m, n, rowptr, colidx)[1]

    def absolute_rows(m, n, rowptr, colidx):
        d, _ = IC.icsr_encode(m, n, rowptr, colidx)
        return d, np.flatnonzero(np.diff(np.asarray(rowptr)))

    def restart_per_row(m, n, rowptr, colidx):
        return np.asarray(colidx, dtype=np.int64), IC.icsr_encode(m, n, rowptr, colidx)[1]

    for wrong in (no_signal, absolute_rows, restart_per_row):
        wd, wj = wrong(g["m"], g["n"], rp, ci)
        assert (wd.tolist(), wj.tolist()) != (g["col_diff"], g["row_jump"]), wrong.__name__
    y = IC.icsr_spmv(g["m"], g["n"], cd, rj, g["vals"], g["x"])
    assert y.tolist() == g["y"]
