"""Parity at the sizes and in the launch shapes the benchmark times: the
three 1,048,576-row matrices of the FP64 sweep (5-point mesh 1024^2, R-MAT
degree 16, 64 blocks of 16384^2 with a 5% border), each in natural order and
in SB (K = 1024), DB (K = 1024) and split (K = 16) forms, the tiled forms in
every tile shape the autotuner chooses from.  The forms come from cheap
labels (contiguous row ranges, a border of every 16th row, nonzeros labelled
by row range and column range) rather than from the bisection: that changes
which rows share a tile, not the code that runs.  The oracle recomputes a
random sample of rows one by one from the original CSR; every output entry
must be written."""
import numpy as np
import pytest

import bench
import oracle
import synth
from tests._util import TOL, err_ratio, run_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S = None
K_ROWS = 1024       # SB / DB parts, as the sweep
K_SPLIT = 16

MATRICES = {
    "mesh5_1024": lambda: synth.mesh5(1024, seed=0),
    "rmat20_d16": lambda: synth.rmat(20, 16, seed=0),
    "blocks64_0.2pct": lambda: synth.blocks(seed=0),
}
# the tile shape of each (matrix, form): SB, DB, split; the autotuner's
# shapes and the staged 256-thread shape, staged and unstaged
SHAPES = {
    "mesh5_1024": ("cta256", "cta256s", "cta1024"),
    "rmat20_d16": ("cta256w", "cta256x8", "cta256s"),
    "blocks64_0.2pct": ("cta1024", "cta256", "cta256x8"),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global S
    import paper_1203_2739_gb300 as lib
    S = lib
    torch.cuda.set_device(0)
    yield


def _sample_reference(m, n, rp, ci, v, x, rows):
    """y and |A||x| of the sampled rows, from the oracle on those rows of the
    original CSR."""
    lens = (rp[rows + 1] - rp[rows]).astype(np.int64)
    srp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(lens, out=srp[1:])
    idx = np.repeat(rp[rows].astype(np.int64) - srp[:-1], lens) + np.arange(srp[-1])
    return oracle.spmv(rows.size, n, srp, ci[idx], v[idx], x)


def _forms(m, n, rp, ci):
    """(name, spmv_plan_create keyword arguments) of the three tiled forms."""
    rows = (np.arange(m, dtype=np.int64) * K_ROWS // m).astype(np.int32)
    out = []
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, K_ROWS, rows)
    out.append(("sb", dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SB, K=K_ROWS,
                           row_part_ptr=rpp, col_part_ptr=cpp)))
    db = rows.copy()
    db[::16] = K_ROWS
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_DB, K_ROWS, db)
    out.append(("db", dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_DB, K=K_ROWS,
                           row_part_ptr=rpp, col_part_ptr=cpp)))
    # A^k: nonzeros in row range a and column range b of a 4 x 4 grid
    r_of = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
    nz = ((r_of * 4 // m) * 4 + ci.astype(np.int64) * 4 // n).astype(np.int32)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, K_SPLIT, nz)
    out.append(("split", dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SPLIT, K=K_SPLIT,
                              row_part_ptr=rpp, col_part_ptr=cpp, nz_part=nz)))
    return out


@pytest.mark.parametrize("name", list(MATRICES))
def test_full_size_forms_and_shapes(name):
    rp, ci, v = MATRICES[name]()
    m = n = len(rp) - 1
    nnz = int(rp[-1])
    x = synth.uniform_x(n, 1)
    rng = np.random.default_rng(17)
    rows = np.unique(np.r_[0, m - 1, rng.integers(0, m, 4096)])
    y_ref, absax = _sample_reference(m, n, rp, ci, v, x, rows)
    shapes = bench.tile_shapes(S, S.SPMV_F64, 1, nnz)
    shapes["cta256s"] = dict(dtype=S.SPMV_F64, nrhs=1, flags=S.SPMV_FLAG_STAGE)
    plans = [("natural", S.spmv_plan_create(m, n, rp, ci, v))]
    for (form, kw), shape in zip(_forms(m, n, rp, ci), SHAPES[name]):
        plans.append(("%s/%s" % (form, shape), S.spmv_plan_create(m, n, rp, ci, v,
                                                                   **shapes[shape], **kw)))
    for label, plan in plans:
        y = run_plan(S, plan, x)
        assert not np.any(np.isnan(y)), label
        r = err_ratio(y[rows], y_ref, absax)
        assert r <= TOL[0], (label, r)
        S.spmv_plan_destroy(plan)
