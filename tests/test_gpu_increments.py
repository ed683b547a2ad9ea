"""GPU parity of the column-increment storage (SPMV_FLAG_COL_DELTA): the
chunks of tiles that stage nothing keep 16-bit increments of the column
index along each row, the colDiff array of ICSR (Sec. 2.1) kept per lane,
read two slots per 32-bit load.  Every case is compared with the FP64
oracle: bit for bit on integer data, within the precision's bound on
real-valued data."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import TOL, err_ratio, run_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S = None
DELTA = 64


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global S
    import paper_1203_2739_gb300 as lib
    S = lib
    assert S.SPMV_FLAG_COL_DELTA == DELTA
    torch.cuda.set_device(0)
    yield


def _check(plan, m, n, rp, ci, v, x, exact):
    y = run_plan(S, plan, x)
    y_ref, absax = oracle.spmv(m, n, rp, ci, v, x)
    if exact:
        assert np.array_equal(y, y_ref)
    else:
        r = err_ratio(y, y_ref, absax)
        assert r <= TOL[plan.info["dtype"]], r


def _forms(m, n, rp, ci, seed):
    """Natural order through the tiles, SB and DB from random row labels,
    a split from random nonzero labels."""
    out = [dict(flags=S.SPMV_FLAG_TILED_NATURAL)]
    for form, frac in ((S.SPMV_SB, 0.0), (S.SPMV_DB, 0.1)):
        lab = synth.random_labels(m, 8, seed, border_frac=frac)
        rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, form, 8, lab)
        out.append(dict(row_perm=rperm, col_perm=cperm, form=form, K=8, row_part_ptr=rpp,
                        col_part_ptr=cpp))
    nzl = synth.random_labels(int(rp[-1]), 16, seed + 1)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, 16, nzl)
    out.append(dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SPLIT, K=16, row_part_ptr=rpp,
                    col_part_ptr=cpp, nz_part=nzl))
    return out


def _plan(m, n, rp, ci, v, kw, **opts):
    kw = dict(kw)
    kw["flags"] = kw.get("flags", 0) | opts.pop("flags", 0) | DELTA
    return S.spmv_plan_create(m, n, rp, ci, v, **kw, **opts)


@pytest.fixture(scope="module")
def mesh():
    rp, ci, v = synth.mesh5(200, seed=3)
    m = n = len(rp) - 1
    return m, n, rp, ci, v


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("nrhs", [1, 2, 4, 8])
def test_every_form_exact(mesh, dtype, nrhs):
    """Batches of 8 (r = 1), 4 (r = 2) and 2 (r >= 4) slots, every form."""
    m, n, rp, ci, _ = mesh
    vi = synth.integer_values(int(rp[-1]), 41)
    x = synth.integer_x(n, 42, nrhs=nrhs) if nrhs > 1 else synth.integer_x(n, 42)
    for kw in _forms(m, n, rp, ci, 43):
        plan = _plan(m, n, rp, ci, vi, kw, dtype=dtype, nrhs=nrhs)
        assert plan.info["delta_nnz"] > 0
        _check(plan, m, n, rp, ci, vi, x, exact=True)


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_real_values_within_bound(mesh, dtype):
    m, n, rp, ci, v = mesh
    x = synth.uniform_x(n, 45)
    for kw in _forms(m, n, rp, ci, 46):
        _check(_plan(m, n, rp, ci, v, kw, dtype=dtype), m, n, rp, ci, v, x, exact=False)


def _ragged(seed, m=3000, n=5000, maxlen=40):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, maxlen + 1, size=m)
    rp = np.zeros(m + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate([np.sort(rng.choice(n, size=k, replace=False)) for k in lens]
                        ).astype(np.int32)
    return m, n, rp, ci


@pytest.mark.parametrize("cta", [256, 512, 1024])
@pytest.mark.parametrize("warp_rows", [0, 16])
def test_chunks_of_every_length_exact(cta, warp_rows):
    """Row lengths 0..40 give chunks of odd and even length (the odd last
    slot is stored plainly), empty lanes, and (warp_rows = 16) warp rows that
    keep 32-bit indices in the same tile."""
    m, n, rp, ci = _ragged(47)
    vi = synth.integer_values(int(rp[-1]), 48)
    x = synth.integer_x(n, 49)
    plan = _plan(m, n, rp, ci, vi, dict(flags=S.SPMV_FLAG_TILED_NATURAL), cta_threads=cta,
                 warp_rows=warp_rows)
    assert plan.info["delta_nnz"] > 0
    _check(plan, m, n, rp, ci, vi, x, exact=True)


def test_wide_rows_keep_32_bit_chunks_exact():
    """Chunks whose increments exceed 16 bits are stored with 32-bit indices
    beside increment chunks of the same tiles."""
    rng = np.random.default_rng(50)
    m, n = 4096, 400000
    lens = rng.integers(2, 9, size=m)
    rows = []
    for i, k in enumerate(lens):
        if i % 3 == 0:
            rows.append(np.sort(rng.choice(n, size=k, replace=False)))
        else:
            c0 = rng.integers(0, n - 2000)
            rows.append(np.sort(c0 + rng.choice(2000, size=k, replace=False)))
    rp = np.zeros(m + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate(rows).astype(np.int32)
    vi = synth.integer_values(int(rp[-1]), 51)
    order = np.argsort(ci[rp[:-1]], kind="stable").astype(np.int32)
    plan = _plan(m, n, rp, ci, vi, dict(flags=S.SPMV_FLAG_TILED_NATURAL, row_perm=order))
    assert 0 < plan.info["delta_nnz"] < int(rp[-1])
    _check(plan, m, n, rp, ci, vi, synth.integer_x(n, 52), exact=True)


@pytest.mark.parametrize("flags", [4, 8])
def test_persistent_launches_exact(mesh, flags):
    """The SM-affine and persistent kernels run the same tile code."""
    m, n, rp, ci, _ = mesh
    vi = synth.integer_values(int(rp[-1]), 53)
    plan = _plan(m, n, rp, ci, vi, _forms(m, n, rp, ci, 54)[1], flags=flags, tile_nnz=4096)
    assert plan.info["delta_nnz"] > 0
    for seed in (55, 56):
        _check(plan, m, n, rp, ci, vi, synth.integer_x(n, seed), exact=True)


def test_same_product_as_32_bit_indices(mesh):
    """Increments change the index stream, not the arithmetic: with the same
    tiles and row order the FP64 product is bit-identical to the 32-bit
    plan's on real-valued data."""
    m, n, rp, ci, v = mesh
    x = synth.uniform_x(n, 58)
    for kw in _forms(m, n, rp, ci, 59):
        plain = S.spmv_plan_create(m, n, rp, ci, v, **kw)
        inc = _plan(m, n, rp, ci, v, kw)
        assert inc.info["n_tiles"] == plain.info["n_tiles"]
        assert np.array_equal(run_plan(S, inc, x), run_plan(S, plain, x))


def test_degenerate_matrices():
    """No nonzeros, one nonzero, and a tall matrix with three columns (every
    increment 0, 1 or 2) under the increment flag, in the natural and split
    forms."""
    m, n = 37, 11
    rp = np.zeros(m + 1, dtype=np.int32)
    ci = np.zeros(0, dtype=np.int32)
    v = np.zeros(0)
    plan = _plan(m, n, rp, ci, v, dict(flags=S.SPMV_FLAG_TILED_NATURAL))
    assert np.array_equal(run_plan(S, plan, synth.uniform_x(n, 0)), np.zeros(m))
    plan = _plan(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]),
                 dict(flags=S.SPMV_FLAG_TILED_NATURAL))
    assert run_plan(S, plan, np.array([2.0]))[0] == 6.0
    m, n = 10000, 3
    rng = np.random.default_rng(60)
    rows = [np.sort(rng.choice(n, size=rng.integers(0, 4), replace=False)) for _ in range(m)]
    rp = np.zeros(m + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate(rows).astype(np.int32)
    vi = synth.integer_values(int(rp[-1]), 61)
    x = synth.integer_x(n, 62)
    nzl = synth.random_labels(int(rp[-1]), 4, 63)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, 4, nzl)
    for kw in (dict(flags=S.SPMV_FLAG_TILED_NATURAL),
               dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SPLIT, K=4,
                    row_part_ptr=rpp, col_part_ptr=cpp, nz_part=nzl)):
        plan = _plan(m, n, rp, ci, vi, kw)
        assert plan.info["delta_nnz"] == int(rp[-1])
        _check(plan, m, n, rp, ci, vi, x, exact=True)
