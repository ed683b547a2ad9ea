"""The plan images the GPU runs, checked on the host: spmv_plan_emulate builds
the image spmv_plan_create would build and walks it as the kernels do (staged
windows, warp rows, 32-row chunks, chunk tiles of long rows, partial slots,
fix-ups), checking every index and that every row of y and every partial
slot is written exactly once.  With integer data every sum is exact, so the
result must equal the oracle's y = A x bit for bit (Sec. 3, Sec. 4), for
every form, tile shape, precision layout and right-hand-side count the
benchmark uses, at sizes where tiles, waves and chunk tiles all occur."""
import numpy as np
import pytest

import bench
import oracle
import synth

S = pytest.importorskip("paper_1203_2739_gb300")

SHAPE_NAMES = ["cta256", "cta256w", "cta256s", "cta512", "cta1024", "cta256x8"]


def _shapes(dtype, nrhs, nnz):
    """The autotuner's shapes and the staged 256-thread shape."""
    sh = bench.tile_shapes(S, dtype, nrhs, nnz)
    sh["cta256s"] = dict(dtype=dtype, nrhs=nrhs, flags=S.SPMV_FLAG_STAGE)
    return sh


def _integer(rp, ci, seed):
    return synth.integer_values(int(rp[-1]), seed)


def _reference(m, n, rp, ci, v, x):
    if x.ndim == 1:
        return oracle.spmv(m, n, rp, ci, v, x)[0]
    return np.stack([oracle.spmv(m, n, rp, ci, v, np.ascontiguousarray(x[:, c]))[0]
                     for c in range(x.shape[1])], axis=1)


def _contiguous(m, K):
    return (np.arange(m, dtype=np.int64) * K // max(m, 1)).astype(np.int32)


def _forms(m, n, rp, ci, K_rows, K_split, seed):
    """SB, DB (every 16th row in the border) and split forms from labels."""
    rows = _contiguous(m, K_rows)
    out = []
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, K_rows, rows)
    out.append(("sb", dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SB, K=K_rows,
                           row_part_ptr=rpp, col_part_ptr=cpp)))
    db = rows.copy()
    db[::16] = K_rows
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_DB, K_rows, db)
    out.append(("db", dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_DB, K=K_rows,
                           row_part_ptr=rpp, col_part_ptr=cpp)))
    nz = synth.random_labels(int(rp[-1]), K_split, seed)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, K_split, nz)
    out.append(("split", dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SPLIT, K=K_split,
                              row_part_ptr=rpp, col_part_ptr=cpp, nz_part=nz)))
    return out


def _check(m, n, rp, ci, v, x, y_ref, **kw):
    y, st = S.spmv_plan_emulate(m, n, rp, ci, v, x, **kw)
    assert np.array_equal(y, y_ref), {k: kw[k] for k in kw if k not in
                                      ("row_perm", "col_perm", "row_part_ptr", "col_part_ptr",
                                       "nz_part")}
    return st


MATRICES = {
    "zipf16k": lambda: synth.zipf_matrix(seed=0),
    "mesh160": lambda: synth.mesh5(160, seed=1),
    "rmat15": lambda: synth.rmat(15, 16, seed=2),
    "blocks16": lambda: synth.blocks(16, 2048, 34.0 / 2048, 0.05, seed=3),
}


@pytest.mark.parametrize("name", list(MATRICES))
def test_every_form_and_shape(name):
    rp, ci, _ = MATRICES[name]()
    m = n = len(rp) - 1
    v = _integer(rp, ci, 5)
    x = synth.integer_x(n, 6)
    y_ref = _reference(m, n, rp, ci, v, x)
    nnz = int(rp[-1])
    shapes = _shapes(S.SPMV_F64, 1, nnz)
    st = _check(m, n, rp, ci, v, x, y_ref)
    assert st["plain_csr"] == 1
    seen = {"chunk_tiles": 0, "staged_tiles": 0, "partial_slots": 0, "warp_rows": 0}
    forms = _forms(m, n, rp, ci, 64, 16, 7)
    if name in ("mesh160", "blocks16"):
        # a partitioner-made SB form: parts with local columns, which the
        # tiles stage
        part = S.spmv_partition(m, n, rp, ci, S.SPMV_PART_CN, K=16, seed=0)
        forms.append(("sb-cn", dict(row_perm=part["row_perm"], col_perm=part["col_perm"],
                                    form=part["form"], K=part["K"],
                                    row_part_ptr=part["row_part_ptr"],
                                    col_part_ptr=part["col_part_ptr"])))
    for shape in SHAPE_NAMES:
        st = _check(m, n, rp, ci, v, x, y_ref, flags=S.SPMV_FLAG_TILED_NATURAL |
                    shapes[shape].get("flags", 0),
                    **{k: a for k, a in shapes[shape].items() if k != "flags"})
        for form, kw in forms:
            st = _check(m, n, rp, ci, v, x, y_ref, **shapes[shape], **kw)
            assert st["plain_csr"] == 0 and st["tiles"] > 0
            for k in seen:
                seen[k] += st[k]
    # the shapes and forms together reach every part of the image: partial
    # slots (split rows), warp rows on the power-law matrices, staged
    # windows on the local ones
    assert seen["partial_slots"] > 0
    if name in ("zipf16k", "rmat15"):
        assert seen["warp_rows"] > 0
    if name == "mesh160":
        assert seen["staged_tiles"] > 0
    # rows over the long-row threshold become chunk tiles (R-MAT's hubs;
    # forced on the Zipf matrix with a low threshold)
    if name == "rmat15":
        assert seen["chunk_tiles"] > 0
    if name == "zipf16k":
        for form, kw in _forms(m, n, rp, ci, 64, 16, 7):
            st = _check(m, n, rp, ci, v, x, y_ref, long_row=100, **kw)
            # (the split's part rows are all shorter than 100)
            assert (st["chunk_tiles"] > 0) == (form != "split")


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("nrhs", [1, 2, 8])
def test_precision_layouts_and_right_hand_sides(dtype, nrhs):
    """The window capacity depends on the vector type and r, so each layout
    is checked; values are used in FP64 whatever the dtype."""
    rp, ci, _ = synth.mesh5(128, seed=4)
    m = n = len(rp) - 1
    v = _integer(rp, ci, 8)
    x = synth.integer_x(n, 9, nrhs=nrhs) if nrhs > 1 else synth.integer_x(n, 9)
    y_ref = _reference(m, n, rp, ci, v, x)
    shapes = _shapes(dtype, nrhs, int(rp[-1]))
    for shape in ("cta256", "cta256s", "cta512", "cta1024"):
        for form, kw in _forms(m, n, rp, ci, 32, 16, 10):
            _check(m, n, rp, ci, v, x, y_ref, **shapes[shape], **kw)


@pytest.mark.parametrize("n_sm", [1, 8, 152])
def test_sm_count_sets_tiles_not_results(n_sm):
    """Tiles are sized for one wave on n_sm SMs: far fewer SMs means far
    larger tiles, more rows cut into chunk tiles, the same product."""
    rp, ci, _ = synth.zipf_matrix(8192, 8192, seed=11)
    m = n = 8192
    v = _integer(rp, ci, 12)
    x = synth.integer_x(n, 13)
    y_ref = _reference(m, n, rp, ci, v, x)
    tiles = []
    for form, kw in _forms(m, n, rp, ci, 16, 4, 14):
        st = _check(m, n, rp, ci, v, x, y_ref, n_sm=n_sm, **kw)
        tiles.append(st["tiles"])
    assert min(tiles) > 0


def test_partitioner_forms_on_the_configured_small_matrix():
    """The forms the bisection produces (not only label-derived ones)."""
    m = n = 16384
    rp, ci, _ = synth.zipf_matrix(m, n, seed=0)
    v = _integer(rp, ci, 15)
    x = synth.integer_x(n, 16)
    y_ref = _reference(m, n, rp, ci, v, x)
    for method in (S.SPMV_PART_CN, S.SPMV_PART_ERCN, S.SPMV_PART_RCN):
        res = S.spmv_partition(m, n, rp, ci, method, K=8, seed=0)
        kw = dict(row_perm=res["row_perm"], col_perm=res["col_perm"], form=res["form"],
                  K=res["K"], row_part_ptr=res["row_part_ptr"],
                  col_part_ptr=res["col_part_ptr"])
        if res["form"] == S.SPMV_SPLIT:
            kw["nz_part"] = res["labels"]
        for shape in SHAPE_NAMES:
            _check(m, n, rp, ci, v, x, y_ref, **_shapes(0, 1, int(rp[-1]))[shape],
                   **kw)


def test_full_size_mesh_in_every_shape():
    """The 1024^2 mesh of the sweep at full size: SB and DB at K = 1024 and
    the split at K = 16, in every tile shape."""
    rp, ci, _ = synth.mesh5(1024, seed=0)
    m = n = len(rp) - 1
    v = _integer(rp, ci, 17)
    x = synth.integer_x(n, 18)
    y_ref = _reference(m, n, rp, ci, v, x)
    shapes = _shapes(0, 1, int(rp[-1]))
    forms = _forms(m, n, rp, ci, 1024, 16, 19)
    for shape in SHAPE_NAMES:
        for form, kw in forms:
            _check(m, n, rp, ci, v, x, y_ref, **shapes[shape], **kw)


def test_emulation_reports_validation_errors_like_plan_creation():
    rp, ci, _ = synth.random_sparse(20, 20, 0.2, 1)
    v = _integer(rp, ci, 2)
    with pytest.raises(S.SpmvError) as e:
        S.spmv_plan_emulate(20, 20, rp, ci, v, np.zeros(20), flags=1 << 10)
    assert e.value.status == S.SPMV_E_INVALID
    bad = np.arange(20, dtype=np.int32)
    bad[3] = 4
    with pytest.raises(S.SpmvError) as e:
        S.spmv_plan_emulate(20, 20, rp, ci, v, np.zeros(20), row_perm=bad, col_perm=None)
    assert e.value.status == S.SPMV_E_STRUCTURE


def _with_flags(kw, flags):
    out = dict(kw)
    out["flags"] = out.get("flags", 0) | flags
    return out


@pytest.mark.parametrize("name", list(MATRICES))
def test_column_increments_every_form_and_shape(name):
    """SPMV_FLAG_COL_DELTA: the chunks of tiles that stage nothing hold 16-bit
    column increments along each row (ICSR's colDiff, Sec. 2.1, per lane,
    slots in pairs).  The emulator decodes them as the kernel does, checks
    every running column (padding included) against n and every padding
    increment for 0, and the product must stay exact."""
    rp, ci, _ = MATRICES[name]()
    m = n = len(rp) - 1
    v = _integer(rp, ci, 21)
    x = synth.integer_x(n, 22)
    y_ref = _reference(m, n, rp, ci, v, x)
    nnz = int(rp[-1])
    shapes = _shapes(S.SPMV_F64, 1, nnz)
    total = 0
    for shape in SHAPE_NAMES:
        st = _check(m, n, rp, ci, v, x, y_ref,
                    **_with_flags(shapes[shape], S.SPMV_FLAG_TILED_NATURAL |
                                  S.SPMV_FLAG_COL_DELTA))
        total += st["delta_nnz"]
        for form, kw in _forms(m, n, rp, ci, 64, 16, 23):
            st = _check(m, n, rp, ci, v, x, y_ref,
                        **_with_flags(shapes[shape], S.SPMV_FLAG_COL_DELTA), **kw)
            assert 0 <= st["delta_nnz"] <= st["gathered_nnz"]
            total += st["delta_nnz"]
            # without the flag nothing is increment-coded
            st0 = _check(m, n, rp, ci, v, x, y_ref, **shapes[shape], **kw)
            assert st0["delta_nnz"] == 0
    assert total > 0


@pytest.mark.parametrize("nrhs", [1, 2, 4, 8])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_column_increments_layouts(dtype, nrhs):
    """Batches of 8, 4 and 2 slots (one per r) read the increments in pairs;
    rows of every length up to 40 give chunks of odd and even length."""
    rng = np.random.default_rng(24 + nrhs)
    m, n = 3000, 5000
    lens = rng.integers(0, 41, size=m)
    rp = np.zeros(m + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate([np.sort(rng.choice(n, size=k, replace=False)) for k in lens]
                        ).astype(np.int32)
    v = _integer(rp, ci, 25)
    x = synth.integer_x(n, 26, nrhs=nrhs) if nrhs > 1 else synth.integer_x(n, 26)
    y_ref = _reference(m, n, rp, ci, v, x)
    shapes = _shapes(dtype, nrhs, int(rp[-1]))
    for shape in ("cta256", "cta256w", "cta512", "cta1024"):
        st = _check(m, n, rp, ci, v, x, y_ref,
                    **_with_flags(shapes[shape], S.SPMV_FLAG_TILED_NATURAL |
                                  S.SPMV_FLAG_COL_DELTA))
        # n < 65536: every chunk of an unstaged tile fits 16 bits
        assert st["delta_nnz"] == st["gathered_nnz"] - _warp_row_nnz(rp, shapes[shape]), shape


def _warp_row_nnz(rp, shape):
    """Nonzeros of rows reduced by a whole warp (never increment-coded)."""
    lens = np.diff(rp)
    return int(lens[lens > shape.get("warp_rows", 64)].sum())


def test_column_increments_fall_back_on_wide_rows():
    """Rows whose successive columns lie more than 65535 apart keep 32-bit
    indices (their chunk's base is -1); the rest of the tile is still
    increment-coded, and the product is unchanged."""
    rng = np.random.default_rng(27)
    m, n = 4096, 400000
    lens = rng.integers(2, 9, size=m)
    rows = []
    for i, k in enumerate(lens):
        if i % 3 == 0:
            rows.append(np.sort(rng.choice(n, size=k, replace=False)))        # wide
        else:
            c0 = rng.integers(0, n - 2000)
            rows.append(np.sort(c0 + rng.choice(2000, size=k, replace=False)))  # narrow
    rp = np.zeros(m + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate(rows).astype(np.int32)
    v = _integer(rp, ci, 28)
    x = synth.integer_x(n, 29)
    y_ref = _reference(m, n, rp, ci, v, x)
    # rows sorted by length share chunks: a chunk mixes wide and narrow rows
    # and falls back; the base of 32 narrow rows spread over n does not fit
    # either, so order the rows by their first column first
    order = np.argsort(ci[rp[:-1]], kind="stable").astype(np.int32)
    st = _check(m, n, rp, ci, v, x, y_ref, row_perm=order,
                flags=S.SPMV_FLAG_TILED_NATURAL | S.SPMV_FLAG_COL_DELTA)
    assert 0 <= st["delta_nnz"] < st["gathered_nnz"]


@pytest.mark.parametrize("name", ["mesh160", "blocks16", "rmat15"])
def test_nested_border_forms_from_the_partitioner(name):
    """SB (column-net) and DB (enhanced row-column-net) partitions laid out
    with the nested border order, through the tiled kernel in the natural
    form, in every shape, with and without column increments."""
    rp, ci, _ = MATRICES[name]()
    m = n = len(rp) - 1
    v = _integer(rp, ci, 31)
    x = synth.integer_x(n, 32)
    y_ref = _reference(m, n, rp, ci, v, x)
    shapes = _shapes(S.SPMV_F64, 1, int(rp[-1]))
    for method in (S.SPMV_PART_CN, S.SPMV_PART_ERCN):
        part = S.spmv_partition(m, n, rp, ci, method, K=16, seed=0)
        rperm, cperm = S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_NESTED, 16, part["labels"])
        for shape in SHAPE_NAMES:
            for extra in (0, S.SPMV_FLAG_COL_DELTA):
                _check(m, n, rp, ci, v, x, y_ref, row_perm=rperm, col_perm=cperm,
                       **_with_flags(shapes[shape], S.SPMV_FLAG_TILED_NATURAL | extra))
