"""GPU parity of every form, precision and right-hand-side count against the
CPU oracle, through the C ABI.  Integer data make every sum exact, so those
cases are bit-exact; floating data are held to |y - y_ref| <= tol (|A||x|)."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import TOL, err_ratio, run_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global S
    import paper_1203_2739_gb300 as lib
    S = lib
    torch.cuda.set_device(0)
    yield


def _check(plan, m, n, rp, ci, v, x, exact=False, tol=None):
    y = run_plan(S, plan, x)
    y_ref, absax = oracle.spmv(m, n, rp, ci, v, x)
    if exact:
        assert np.array_equal(y, y_ref)
    else:
        r = err_ratio(y, y_ref, absax)
        assert r <= (tol if tol is not None else TOL[plan.info["dtype"]]), r
    return y


def _sb_plan(m, n, rp, ci, v, K, seed, border=False, **kw):
    lab = synth.random_labels(m, K, seed, border_frac=0.1 if border else 0.0)
    form = S.SPMV_DB if border else S.SPMV_SB
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, form, K, lab)
    return S.spmv_plan_create(m, n, rp, ci, v, row_perm=rperm, col_perm=cperm, form=form, K=K,
                              row_part_ptr=rpp, col_part_ptr=cpp, **kw)


def _split_plan(m, n, rp, ci, v, K, seed, **kw):
    nzl = synth.random_labels(int(rp[-1]), K, seed)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, K, nzl)
    return S.spmv_plan_create(m, n, rp, ci, v, row_perm=rperm, col_perm=cperm,
                              form=S.SPMV_SPLIT, K=K, row_part_ptr=rpp, col_part_ptr=cpp,
                              nz_part=nzl, **kw)


@pytest.fixture(scope="module")
def zipf():
    m = n = 16384
    rp, ci, v = synth.zipf_matrix(m, n, seed=0)
    return m, n, rp, ci, v


# ------------------------------------------------------- natural (K1) ---
@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("nrhs", [1, 8])
def test_natural_zipf(zipf, dtype, nrhs):
    m, n, rp, ci, v = zipf
    plan = S.spmv_plan_create(m, n, rp, ci, v, dtype=dtype, nrhs=nrhs)
    x = synth.uniform_x(n, 1, nrhs=nrhs)
    _check(plan, m, n, rp, ci, v, x)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_natural_lanes_exact(zipf, lanes):
    m, n, rp, ci, _ = zipf
    vi = synth.integer_values(int(rp[-1]), 5)
    plan = S.spmv_plan_create(m, n, rp, ci, vi, lanes=lanes, long_row=64)
    assert plan.info["lanes"] == lanes
    _check(plan, m, n, rp, ci, vi, synth.integer_x(n, 2), exact=True)


# -------------------------------------------------------------- SB / DB ---
@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("nrhs", [1, 2, 4, 8])
def test_sb_zipf(zipf, dtype, nrhs):
    m, n, rp, ci, v = zipf
    plan = _sb_plan(m, n, rp, ci, v, 8, 3, dtype=dtype, nrhs=nrhs)
    _check(plan, m, n, rp, ci, v, synth.uniform_x(n, 4, nrhs=nrhs))


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_db_zipf(zipf, dtype):
    m, n, rp, ci, v = zipf
    plan = _sb_plan(m, n, rp, ci, v, 8, 5, border=True, dtype=dtype)
    _check(plan, m, n, rp, ci, v, synth.uniform_x(n, 6))


def _contiguous_labels(m, K):
    return (np.arange(m, dtype=np.int64) * K // max(m, 1)).astype(np.int32)


@pytest.mark.parametrize("K", [1, 4, 64])
def test_sb_mesh_exact_and_staged(K):
    rp, ci, _ = synth.mesh5(96, seed=0, permute=False)
    m = n = 96 * 96
    vi = synth.integer_values(int(rp[-1]), 1)
    lab = _contiguous_labels(m, K)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, K, lab)
    plan = S.spmv_plan_create(m, n, rp, ci, vi, row_perm=rperm, col_perm=cperm, form=S.SPMV_SB,
                              K=K, row_part_ptr=rpp, col_part_ptr=cpp, tile_cols=1024,
                              flags=S.SPMV_FLAG_STAGE)
    assert plan.info["n_staged_tiles"] > 0
    for dtype in (0, 1, 2):
        p = S.spmv_plan_create(m, n, rp, ci, vi, row_perm=rperm, col_perm=cperm,
                               form=S.SPMV_SB, K=K, row_part_ptr=rpp, col_part_ptr=cpp,
                               tile_cols=1024, dtype=dtype, flags=S.SPMV_FLAG_STAGE)
        _check(p, m, n, rp, ci, vi, synth.integer_x(n, 3), exact=True)
        # default 256-thread CTAs stage nothing
        p = S.spmv_plan_create(m, n, rp, ci, vi, row_perm=rperm, col_perm=cperm,
                               form=S.SPMV_SB, K=K, row_part_ptr=rpp, col_part_ptr=cpp,
                               dtype=dtype)
        assert p.info["n_staged_tiles"] == 0
        _check(p, m, n, rp, ci, vi, synth.integer_x(n, 3), exact=True)


# ----------------------------------------------------------------- split ---
@pytest.mark.parametrize("K", [1, 4, 16, 64])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_split_zipf(zipf, K, dtype):
    m, n, rp, ci, v = zipf
    plan = _split_plan(m, n, rp, ci, v, K, 7, dtype=dtype)
    if K > 1:
        assert plan.info["partial_slots"] > 0 and plan.info["launches_per_exec"] == 2
    _check(plan, m, n, rp, ci, v, synth.uniform_x(n, 8))


@pytest.mark.parametrize("nrhs", [1, 8])
def test_split_exact(zipf, nrhs):
    m, n, rp, ci, _ = zipf
    vi = synth.integer_values(int(rp[-1]), 9)
    plan = _split_plan(m, n, rp, ci, vi, 16, 10, nrhs=nrhs, tile_cols=512)
    _check(plan, m, n, rp, ci, vi, synth.integer_x(n, 11, nrhs=nrhs), exact=True)


# ---------------------------------------------------- kernel variants ---
@pytest.mark.parametrize("flags", [1, 2, 3, 4, 5, 6, 8, 9, 10])
def test_flag_variants(zipf, flags):
    m, n, rp, ci, v = zipf
    if flags & 2:
        plan = S.spmv_plan_create(m, n, rp, ci, v, flags=flags)
    else:
        plan = _sb_plan(m, n, rp, ci, v, 8, 12, flags=flags)
    if flags & 1:
        assert plan.info["n_staged_tiles"] == 0
    _check(plan, m, n, rp, ci, v, synth.uniform_x(n, 13))


# ------------------------------------------ staged runs (bulk copies) ---
def _mesh_sb(nx, K, seed=0):
    rp, ci, _ = synth.mesh5(nx, seed=seed)
    m = n = len(rp) - 1
    part = S.spmv_partition(m, n, rp, ci, S.SPMV_PART_CN, K=K, seed=seed)
    kw = dict(row_perm=part["row_perm"], col_perm=part["col_perm"], form=part["form"],
              K=part["K"], row_part_ptr=part["row_part_ptr"], col_part_ptr=part["col_part_ptr"])
    return m, n, rp, ci, kw


@pytest.mark.parametrize("nx", [64, 63])          # n even, n odd (the last run ends unaligned)
@pytest.mark.parametrize("dtype,nrhs", [(0, 1), (1, 1), (2, 1), (0, 2), (1, 8)])
def test_staged_runs_exact(nx, dtype, nrhs):
    m, n, rp, ci, kw = _mesh_sb(nx, 16)
    vi = synth.integer_values(int(rp[-1]), 21)
    plan = S.spmv_plan_create(m, n, rp, ci, vi, dtype=dtype, nrhs=nrhs, tile_nnz=2048,
                              flags=S.SPMV_FLAG_STAGE, **kw)
    assert plan.info["n_staged_tiles"] > 0
    assert plan.info["smem_bytes"] % 16 == 0
    x = synth.integer_x(n, 22, nrhs=nrhs)
    _check(plan, m, n, rp, ci, vi, x, exact=True)


@pytest.mark.parametrize("flags", [4, 8])
def test_staged_runs_persistent_repeat(flags):
    # the persistent kernels reuse one mbarrier across tiles (its phase
    # alternates) and reset their claim counters for the next launch
    m, n, rp, ci, kw = _mesh_sb(96, 64)
    vi = synth.integer_values(int(rp[-1]), 23)
    plan = S.spmv_plan_create(m, n, rp, ci, vi, tile_nnz=2048, flags=flags | S.SPMV_FLAG_STAGE,
                              **kw)
    assert plan.info["n_staged_tiles"] > 1
    for seed in (24, 25, 26):
        _check(plan, m, n, rp, ci, vi, synth.integer_x(n, seed), exact=True)


@pytest.mark.parametrize("cta", [512, 1024])
@pytest.mark.parametrize("nrhs", [1, 8])
@pytest.mark.parametrize("dtype", [0, 2])
def test_wide_ctas_exact(zipf, dtype, nrhs, cta):
    # 512-thread (two per SM) and 1024-thread (one per SM) CTAs per tile with
    # large staging windows
    m, n, rp, ci, _ = zipf
    vi = synth.integer_values(int(rp[-1]), 31)
    x = synth.integer_x(n, 32, nrhs=nrhs)
    for plan in (_sb_plan(m, n, rp, ci, vi, 8, 33, dtype=dtype, nrhs=nrhs, cta_threads=cta),
                 _split_plan(m, n, rp, ci, vi, 16, 34, dtype=dtype, nrhs=nrhs, cta_threads=cta,
                             tile_nnz=8192),
                 S.spmv_plan_create(m, n, rp, ci, vi, dtype=dtype, nrhs=nrhs, cta_threads=cta,
                                    flags=S.SPMV_FLAG_TILED_NATURAL, long_row=200)):
        _check(plan, m, n, rp, ci, vi, x, exact=True)


@pytest.mark.parametrize("cta", [256, 512, 1024])
@pytest.mark.parametrize("dtype,nrhs", [(0, 1), (1, 1), (2, 1), (0, 2), (1, 8)])
def test_two_runs_and_mixed_prefix_exact(cta, dtype, nrhs):
    """Tiles that stage the home columns and a window of the border (two
    bulk copies) and still gather some entries: each chunk's leading slots
    load from both memories, the rest from shared memory only.  The host
    emulation of the same plan confirms the image has those features."""
    m, n, rp, ci, kw = _mesh_sb(95, 32)
    vi = synth.integer_values(int(rp[-1]), 37)
    x = synth.integer_x(n, 38, nrhs=nrhs)
    opts = dict(dtype=dtype, nrhs=nrhs, cta_threads=cta, tile_nnz=6000,
                flags=S.SPMV_FLAG_STAGE if cta == 256 else 0)
    _, st = S.spmv_plan_emulate(m, n, rp, ci, vi, np.asarray(x, dtype=np.float64), **opts,
                                **kw)
    assert st["mixed_slots"] > 0 and st["staged_tiles"] > 0
    if nrhs == 1:
        assert st["two_run_tiles"] > 0
    assert 0 < st["gathered_nnz"] < int(rp[-1])
    plan = S.spmv_plan_create(m, n, rp, ci, vi, **opts, **kw)
    _check(plan, m, n, rp, ci, vi, x, exact=True)


def test_wide_ctas_staged_mesh():
    m, n, rp, ci, kw = _mesh_sb(96, 16)
    vi = synth.integer_values(int(rp[-1]), 35)
    plan = S.spmv_plan_create(m, n, rp, ci, vi, cta_threads=1024, tile_nnz=16384, **kw)
    assert plan.info["n_staged_tiles"] > 0
    _check(plan, m, n, rp, ci, vi, synth.integer_x(n, 36), exact=True)


@pytest.mark.parametrize("warp_rows", [8, 128, 600])
def test_warp_row_threshold_exact(zipf, warp_rows):
    m, n, rp, ci, _ = zipf
    vi = synth.integer_values(int(rp[-1]), 44)
    for plan in (_sb_plan(m, n, rp, ci, vi, 8, 45, warp_rows=warp_rows),
                 _split_plan(m, n, rp, ci, vi, 16, 46, warp_rows=warp_rows, nrhs=2)):
        x = synth.integer_x(n, 47, nrhs=plan.info["nrhs"])
        _check(plan, m, n, rp, ci, vi, x if plan.info["nrhs"] > 1 else x.reshape(-1),
               exact=True)


def test_autotune_keeps_a_correct_plan(zipf):
    m, n, rp, ci, _ = zipf
    vi = synth.integer_values(int(rp[-1]), 41)
    lab = synth.random_labels(m, 8, 42)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, 8, lab)
    cands = [dict(), dict(cta_threads=1024), dict(flags=S.SPMV_FLAG_STAGE, tile_nnz=4096)]
    plan, best, ms = S.spmv_plan_autotune(m, n, rp, ci, vi, cands, reps=3, row_perm=rperm,
                                          col_perm=cperm, form=S.SPMV_SB, K=8,
                                          row_part_ptr=rpp, col_part_ptr=cpp)
    assert 0 <= best < len(cands) and ms > 0
    _check(plan, m, n, rp, ci, vi, synth.integer_x(n, 43), exact=True)


def test_misaligned_x_rejected(zipf):
    m, n, rp, ci, v = zipf
    plan = _sb_plan(m, n, rp, ci, v, 8, 12)
    buf = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    y = torch.zeros(m, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SpmvError, match="aligned"):
        S.spmv_exec(plan, buf[1:], y)
    S.spmv_plan_check(plan)


@pytest.mark.parametrize("tile_cols,tile_nnz,long_row", [(64, 256, 32), (4096, 2048, 100),
                                                         (65535 // 8, 100000, 5000)])
def test_tiling_parameters_exact(zipf, tile_cols, tile_nnz, long_row):
    m, n, rp, ci, _ = zipf
    vi = synth.integer_values(int(rp[-1]), 14)
    plan = _sb_plan(m, n, rp, ci, vi, 8, 15, tile_cols=tile_cols, tile_nnz=tile_nnz,
                    long_row=long_row, dtype=1)
    _check(plan, m, n, rp, ci, vi, synth.integer_x(n, 16), exact=True)
    plan = _split_plan(m, n, rp, ci, vi, 4, 17, tile_cols=tile_cols, tile_nnz=tile_nnz,
                       long_row=long_row)
    _check(plan, m, n, rp, ci, vi, synth.integer_x(n, 18), exact=True)


# --------------------------------------------------------------- edges ---
def test_empty_and_degenerate_matrices():
    # no nonzeros: y must be all zero in every form
    m, n = 37, 11
    rp = np.zeros(m + 1, dtype=np.int32)
    ci = np.zeros(0, dtype=np.int32)
    v = np.zeros(0)
    x = synth.uniform_x(n, 0)
    for plan in (S.spmv_plan_create(m, n, rp, ci, v),
                 S.spmv_plan_create(m, n, rp, ci, v, flags=2),
                 _sb_plan(m, n, rp, ci, v, 3, 0),
                 _split_plan(m, n, rp, ci, v, 3, 0)):
        assert np.array_equal(run_plan(S, plan, x), np.zeros(m))
    # one row, one column
    rp = np.array([0, 1], dtype=np.int32)
    ci = np.array([0], dtype=np.int32)
    plan = S.spmv_plan_create(1, 1, rp, ci, np.array([3.0]))
    assert run_plan(S, plan, np.array([2.0]))[0] == 6.0
    # zero rows
    plan = S.spmv_plan_create(0, 5, np.zeros(1, np.int32), ci[:0], v)
    assert plan.info["launches_per_exec"] == 0


def test_single_dense_long_row_and_rectangular():
    # one row touching every column (chunked), plus short rows; m != n
    m, n = 50, 20000
    rows = [np.zeros(n, dtype=np.int64)] + [np.full(3, i) for i in range(1, m)]
    cols = [np.arange(n)] + [np.array([i, i + 7, i + 900]) for i in range(1, m)]
    r, c = np.concatenate(rows), np.concatenate(cols)
    vi = synth.integer_values(r.size, 3)
    rp, ci, vi = synth.coo_to_csr(m, n, r, c, vi)
    x = synth.integer_x(n, 4)
    for plan in (S.spmv_plan_create(m, n, rp, ci, vi),
                 S.spmv_plan_create(m, n, rp, ci, vi, flags=2),
                 _sb_plan(m, n, rp, ci, vi, 2, 1),
                 _sb_plan(m, n, rp, ci, vi, 2, 1, border=True),
                 _split_plan(m, n, rp, ci, vi, 4, 2)):
        if plan.info["form"] != 0 or plan.info["launches_per_exec"] != 1:
            assert plan.info["n_chunk_tiles"] > 0
        _check(plan, m, n, rp, ci, vi, x, exact=True)


def test_permute_roundtrip_and_host_exec(zipf):
    m, n, rp, ci, v = zipf
    plan = _sb_plan(m, n, rp, ci, v, 8, 19)
    x = torch.from_numpy(synth.uniform_x(n, 20)).cuda()
    xh = torch.empty_like(x)
    S.spmv_permute_x(plan, x, xh)
    back = torch.empty_like(x)
    # x_hat[j'] = x[col_perm[j']] is a pure gather: check against numpy indexing
    lab = synth.random_labels(m, 8, 19)
    rperm, cperm, _, _ = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, 8, lab)
    assert np.array_equal(xh.cpu().numpy(), x.cpu().numpy()[cperm])
    yh = torch.empty(m, dtype=torch.float64, device="cuda")
    S.spmv_exec(plan, xh, yh)
    yh_host = np.empty(m)
    S.spmv_exec_host(plan, xh.cpu().numpy(), yh_host)
    torch.cuda.synchronize()
    assert np.array_equal(yh.cpu().numpy(), yh_host)
    pinned_x = xh.cpu().pin_memory()
    pinned_y = torch.empty(m, dtype=torch.float64).pin_memory()
    S.spmv_exec_host(plan, pinned_x, pinned_y)
    assert np.array_equal(pinned_y.numpy(), yh_host)
    y = torch.empty_like(yh)
    S.spmv_unpermute_y(plan, yh, y)
    torch.cuda.synchronize()
    expect = np.empty(m)
    expect[rperm] = yh.cpu().numpy()
    assert np.array_equal(y.cpu().numpy(), expect)
    del back


def test_repeated_exec_is_deterministic(zipf):
    m, n, rp, ci, v = zipf
    plan = _split_plan(m, n, rp, ci, v, 16, 21)
    x = synth.uniform_x(n, 22)
    y0 = run_plan(S, plan, x)
    for _ in range(3):
        assert np.array_equal(run_plan(S, plan, x), y0)


def test_side_stream(zipf):
    m, n, rp, ci, v = zipf
    plan = _sb_plan(m, n, rp, ci, v, 8, 23)
    s = torch.cuda.Stream()
    x = synth.uniform_x(n, 24)
    with torch.cuda.stream(s):
        y = run_plan(S, plan, x, stream=s)
    y_ref, absax = oracle.spmv(m, n, rp, ci, v, x)
    assert err_ratio(y, y_ref, absax) <= 1e-12
