"""Parity of the plans the benchmark times, at full size, against the oracle.

The FP64 sweep's three 1,048,576-row matrices (5-point mesh 1024^2, R-MAT
degree 16, 64 blocks of 16384^2 with a 5% border) are ordered and bisected
exactly as bench.py does (sBFS, sRCM, row-net K = 1024 for sHP_RN,
column-net K = 1024 and column-net until each part's x subvector is below
96 KB for SB, enhanced row-column-net K = 1024 for DB,
row-column-net K = 256 cut into the K = 4 / 16 / 64 / 256 splits),
and every tiled form of the sweep is built in every tile shape the
autotuner chooses from -- so whichever shape it keeps has been checked --
and compared row by row with the oracle on a random sample of rows (every
output entry must be written).  FP32 and BF16 run the SB, DB and K = 16
split forms.  The precision workload's 3D Laplacian 128^3 runs in its DB
form in all three precisions, and the L2-exceeding 6144^2 mesh in an SB
form of 32 x 32 grid tiles.

Partitions take minutes on the host; a directory named by the environment
variable SPMV_PARTITION_CACHE, when set, keeps and reuses them."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import bench
import oracle
import synth
from tests._util import TOL, err_ratio, run_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S = None
SWEEP = ("mesh5_1024", "rmat20_d16", "blocks64_0.2pct")
TILED_FORMS = ["tiled", "rtiled", "bfs", "rcm", "rn1024", "sb1024", "sbfit96", "db1024",
               "split4", "split16", "split64", "split256"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global S
    import paper_1203_2739_gb300 as lib
    S = lib
    torch.cuda.set_device(0)
    yield


@pytest.fixture(scope="module")
def sweep():
    """The sweep's matrices and their partitions, as bench.py makes them."""
    mats = bench.make_matrices("sweep")
    cache = os.environ.get("SPMV_PARTITION_CACHE") or None
    threads = max(1, (os.cpu_count() or 4) // 2)
    with cf.ThreadPoolExecutor(max_workers=len(mats)) as ex:
        futs = [ex.submit(bench.partition_jobs, S, rp, ci, TILED_FORMS, 0, threads, cache, name)
                for name, rp, ci, v in mats]
        parts = [f.result() for f in futs]
    return {name: (rp, ci, v, p) for (name, rp, ci, v), p in zip(mats, parts)}


def _sample(m, seed=17, count=4096):
    rng = np.random.default_rng(seed)
    return np.unique(np.r_[0, m - 1, rng.integers(0, m, count)])


def _build_all(m, n, rp, ci, v, kw, shapes):
    """One plan per shape, built on host threads at once (plan building is
    native code that runs outside the interpreter lock)."""
    fl = kw.get("flags", 0)
    base = {k: a for k, a in kw.items() if k != "flags"}

    def one(item):
        name, opt = item
        o = dict(opt)
        o["flags"] = o.get("flags", 0) | fl
        return name, S.spmv_plan_create(m, n, rp, ci, v, **o, **base)

    with cf.ThreadPoolExecutor(max_workers=len(shapes)) as ex:
        return list(ex.map(one, shapes.items()))


def _check_plans(label, plans, x, rows, y_ref, absax, tol):
    for shape, plan in plans:
        y = run_plan(S, plan, x)
        assert not np.any(np.isnan(y)), (label, shape, "unwritten entries")
        r = err_ratio(y[rows], y_ref, absax)
        assert r <= tol, (label, shape, r)
        S.spmv_plan_destroy(plan)


@pytest.mark.parametrize("name", SWEEP)
def test_sweep_plans_fp64_every_shape(sweep, name):
    """Every tiled form of the FP64 sweep, built as bench.py builds it, in
    every autotuner shape; and the plain CSR kernel in natural and random
    order."""
    rp, ci, v, parts = sweep[name]
    m = n = len(rp) - 1
    x = synth.uniform_x(n, 1)
    rows = _sample(m)
    y_ref, absax = oracle.spmv_rows(rp, ci, v, x, rows)
    for f in ("natural", "random"):
        kw, _ = bench.form_kwargs(S, f, rp, ci, parts)
        _check_plans("%s/%s" % (name, f), [("plain", S.spmv_plan_create(m, n, rp, ci, v, **kw))],
                     x, rows, y_ref, absax, TOL[0])
    shapes = bench.tile_shapes(S, S.SPMV_F64, 1, int(rp[-1]))
    for f in TILED_FORMS:
        kw, _ = bench.form_kwargs(S, f, rp, ci, parts)
        _check_plans("%s/%s" % (name, f), _build_all(m, n, rp, ci, v, kw, shapes), x, rows,
                     y_ref, absax, TOL[0])


@pytest.mark.parametrize("dtype", [1, 2])
@pytest.mark.parametrize("name", SWEEP)
def test_sweep_plans_reduced_precision(sweep, name, dtype):
    """FP32 and BF16 values (FP32 x, y and sums) in the SB, DB and K = 16
    split forms of the sweep, one-wave and eight-wave tiles, against the FP64
    oracle at the stated tolerances."""
    rp, ci, v, parts = sweep[name]
    m = n = len(rp) - 1
    x = synth.uniform_x(n, 2)
    rows = _sample(m, seed=18)
    y_ref, absax = oracle.spmv_rows(rp, ci, v, x, rows)
    shapes = bench.tile_shapes(S, dtype, 1, int(rp[-1]))
    shapes = {k: shapes[k] for k in ("cta256w", "cta256x8", "cta512")}
    for f in ("sb1024", "db1024", "split16"):
        kw, _ = bench.form_kwargs(S, f, rp, ci, parts)
        _check_plans("%s/%s/%d" % (name, f, dtype), _build_all(m, n, rp, ci, v, kw, shapes), x,
                     rows, y_ref, absax, TOL[dtype])


def test_laplacian_db_all_precisions():
    """The precision workload: the permuted 3D Laplacian 128^3 in its DB form
    (enhanced row-column-net bisection, K = 1024), FP64 / FP32 / BF16."""
    (name, rp, ci, v), = bench.make_matrices("precision")
    m = n = len(rp) - 1
    cache = os.environ.get("SPMV_PARTITION_CACHE") or None
    parts = bench.partition_jobs(S, rp, ci, ["db1024"], 0, max(1, os.cpu_count() or 4), cache,
                                 name)
    kw, _ = bench.form_kwargs(S, "db1024", rp, ci, parts)
    x = synth.uniform_x(n, 3)
    rows = _sample(m, seed=19)
    y_ref, absax = oracle.spmv_rows(rp, ci, v, x, rows)
    for dtype in (0, 1, 2):
        shapes = bench.tile_shapes(S, dtype, 1, int(rp[-1]))
        shapes = {k: shapes[k] for k in ("cta256", "cta256x8", "cta512", "cta1024")}
        _check_plans("%s/db1024/%d" % (name, dtype), _build_all(m, n, rp, ci, v, kw, shapes), x,
                     rows, y_ref, absax, TOL[dtype])


def test_scale_mesh_sb():
    """The L2-exceeding point: the permuted 5-point mesh 6144^2 (37.7M rows,
    x = 302 MB) in SB form with K = 1024 parts of 192 x 192 grid points, and
    in natural order through the plain kernel."""
    nx, tiles = 6144, 32
    rp, ci, v, pts = synth.mesh5(nx, seed=0, return_points=True)
    m = n = len(rp) - 1
    gx, gy = pts % nx, pts // nx
    labels = ((gy // (nx // tiles)) * tiles + gx // (nx // tiles)).astype(np.int32)
    K = tiles * tiles
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, K, labels)
    kw = dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SB, K=K, row_part_ptr=rpp,
              col_part_ptr=cpp)
    x = synth.uniform_x(n, 4)
    rows = _sample(m, seed=20)
    y_ref, absax = oracle.spmv_rows(rp, ci, v, x, rows)
    _check_plans("mesh6144/natural", [("plain", S.spmv_plan_create(m, n, rp, ci, v))], x, rows,
                 y_ref, absax, TOL[0])
    shapes = bench.tile_shapes(S, 0, 1, int(rp[-1]))
    shapes = {k: shapes[k] for k in ("cta256", "cta256x8", "cta1024")}
    _check_plans("mesh6144/sb", _build_all(m, n, rp, ci, v, kw, shapes), x, rows, y_ref, absax,
                 TOL[0])


NESTED_ICSR_FORMS = ["sbnest1024", "dbnest1024", "bfs_icsr", "sb1024_icsr", "sbnest1024_icsr",
                     "split16_icsr", "split256_icsr"]


@pytest.mark.parametrize("name", SWEEP)
def test_nested_border_and_increment_forms(sweep, name):
    """The nested border order (SB and DB partitions of the sweep, each
    bisection's cut columns between its halves) and the 16-bit column
    increments of unstaged chunks, on the sweep's full-size plans, in the
    unstaged shapes and the wide staged one; FP64, and BF16 for two of them."""
    rp, ci, v, parts = sweep[name]
    m = n = len(rp) - 1
    x = synth.uniform_x(n, 5)
    rows = _sample(m, seed=21)
    y_ref, absax = oracle.spmv_rows(rp, ci, v, x, rows)
    for dtype, forms in ((0, NESTED_ICSR_FORMS), (2, ["sbnest1024_icsr", "split16_icsr"])):
        shapes = bench.tile_shapes(S, dtype, 1, int(rp[-1]))
        shapes = {k: shapes[k] for k in ("cta256", "cta256w", "cta256x8", "cta1024")}
        for f in forms:
            kw, _ = bench.form_kwargs(S, f, rp, ci, parts)
            _check_plans("%s/%s/%d" % (name, f, dtype), _build_all(m, n, rp, ci, v, kw, shapes),
                         x, rows, y_ref, absax, TOL[dtype])
