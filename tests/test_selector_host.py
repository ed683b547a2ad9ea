"""Host side of the learned selector: the matrix features against a direct
numpy computation of their definitions (include/spmv.h, spmv_features)."""
import numpy as np
import pytest

import synth

S = pytest.importorskip("paper_1203_2739_gb300")


def _features_numpy(m, n, rp, ci):
    rp = rp.astype(np.int64)
    deg = np.diff(rp).astype(np.float64)
    rows = np.repeat(np.arange(m), np.diff(rp))
    cdeg = np.bincount(ci, minlength=n).astype(np.float64)
    nnz = len(ci)
    di = rows * n / m
    dist = np.abs(ci - di)
    blk = np.minimum(15, rows * 16 // m)
    owners = {}
    for j, b in zip(ci, blk):
        owners.setdefault(int(j), set()).add(int(b))
    cut = sum(1 for v in owners.values() if len(v) > 1)
    rmean, cmean = deg.mean(), nnz / n
    return np.array([
        np.log2(1 + m), np.log2(1 + n), np.log2(1 + nnz), rmean, deg.std() / rmean,
        np.log2(1 + deg.max()), deg.max() / rmean, cdeg.std() / cmean, np.log2(1 + cdeg.max()),
        cdeg.max() / cmean, dist.sum() / nnz / n, (dist < max(1, n // 64)).sum() / nnz,
        cut / len(owners), (deg == 0).mean(), deg[deg > 64].sum() / nnz,
        np.log2(1 + nnz * 12.0) - 27.0], dtype=np.float64)


@pytest.mark.parametrize("which", ["zipf", "mesh", "rect"])
def test_features_match_their_definitions(which):
    if which == "zipf":
        m = n = 2048
        rp, ci, _ = synth.zipf_matrix(m, n, seed=1)
    elif which == "mesh":
        m = n = 40 * 40
        rp, ci, _ = synth.mesh5(40, seed=2)
    else:
        m, n = 300, 700
        rp, ci, _ = synth.random_sparse(m, n, 0.05, 3, empty_rows=0.1)
    got = S.spmv_features(m, n, rp, ci)
    want = _features_numpy(m, n, rp, ci)
    assert got.shape == (S.SPMV_SEL_FEATURES,)
    assert np.allclose(got, want, rtol=2e-6, atol=1e-6), np.c_[got, want]


def test_features_see_a_reordering():
    # the same mesh in grid order and randomly permuted: equal degree
    # statistics, very different locality
    rp, ci, _ = synth.mesh5(64, permute=False)
    rq, cq, _ = synth.mesh5(64, seed=4, permute=True)
    a = S.spmv_features(4096, 4096, rp, ci)
    b = S.spmv_features(4096, 4096, rq, cq)
    assert np.allclose(a[:10], b[:10], rtol=1e-6)
    assert a[10] < 0.05 * b[10]                 # mean distance from the diagonal
    assert a[11] > 2 * b[11]                    # near-diagonal share
    assert a[12] < 0.5 and b[12] == 1.0         # columns cut by 16 row blocks
