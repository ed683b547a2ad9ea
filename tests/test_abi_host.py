"""CPU tests of the C-ABI library: it loads, exports every symbol the header
declares, derives forms from labels bit-exactly like the oracle, and rejects
malformed input before touching the GPU."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_1203_2739_gb300 as S
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^[\w \*]*?\b(spmv_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    declared = _declared()
    assert {"spmv_plan_create", "spmv_exec", "spmv_plan_destroy", "spmv_partition"} <= declared
    for name in declared:
        assert hasattr(S.lib, name), name
    assert set(S.EXPORTS) == declared


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("shape", [(40, 40), (57, 31), (23, 70)])
def test_form_from_labels_matches_oracle(seed, shape):
    m, n = shape
    rp, ci, v = synth.random_sparse(m, n, 0.1, seed, empty_rows=0.1)
    K = 5
    lab = synth.random_labels(m, K, seed)
    got = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, K, lab)
    exp = oracle.form_rows(m, n, rp, ci, K, lab)
    for g, e in zip(got, exp):
        assert np.array_equal(g, e)
    lab = synth.random_labels(m, K, seed, border_frac=0.2)
    got = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_DB, K, lab)
    exp = oracle.form_rows(m, n, rp, ci, K, lab, border=True)
    for g, e in zip(got, exp):
        assert np.array_equal(g, e)
    nzl = synth.random_labels(int(rp[-1]), K, seed + 3)
    got = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, K, nzl)
    exp = oracle.form_split(m, n, rp, ci, K, nzl)
    for g, e in zip(got, exp):
        assert np.array_equal(g, e)


def test_form_from_labels_rejects_bad_labels():
    rp, ci, v = synth.random_sparse(10, 10, 0.3, 0)
    with pytest.raises(S.SpmvError) as e:
        S.spmv_form_from_labels(10, 10, rp, ci, S.SPMV_SB, 2, np.full(10, 2))
    assert e.value.status == S.SPMV_E_INVALID


def _plan_status(**kw):
    base = dict(m=6, n=6, rowptr=np.array([0, 2, 3, 3, 5, 6, 7]),
                colidx=np.array([0, 3, 1, 2, 4, 5, 0]), vals=np.ones(7))
    base.update(kw)
    try:
        S.spmv_plan_create(**base)
    except S.SpmvError as e:
        return e.status, str(e)
    return S.SPMV_OK, ""


def test_plan_create_validation_before_any_device_call():
    assert _plan_status(colidx=np.array([3, 0, 1, 2, 4, 5, 0]))[0] == S.SPMV_E_INVALID
    assert _plan_status(colidx=np.array([0, 6, 1, 2, 4, 5, 0]))[0] == S.SPMV_E_INVALID
    assert _plan_status(rowptr=np.array([0, 2, 1, 3, 5, 6, 7]))[0] == S.SPMV_E_INVALID
    st, msg = _plan_status(row_perm=np.array([0, 1, 1, 3, 4, 5]))
    assert st == S.SPMV_E_STRUCTURE and "row_perm" in msg
    assert _plan_status(nrhs=3)[0] == S.SPMV_E_UNSUPPORTED
    assert _plan_status(lanes=3)[0] == S.SPMV_E_INVALID
    assert _plan_status(dtype=7)[0] == S.SPMV_E_INVALID
    assert _plan_status(tile_cols=1 << 20)[0] == S.SPMV_E_UNSUPPORTED
    st, msg = _plan_status(warp_rows=-1)
    assert st == S.SPMV_E_INVALID and "warp_rows" in msg
    st, msg = _plan_status(cta_threads=384)
    assert st == S.SPMV_E_INVALID and "cta_threads" in msg
    st, msg = _plan_status(cta_threads=1024, flags=S.SPMV_FLAG_PERSISTENT | 2)
    assert st == S.SPMV_E_INVALID
    st, msg = _plan_status(flags=128)
    assert st == S.SPMV_E_INVALID and "flag" in msg
    st, msg = _plan_status(flags=S.SPMV_FLAG_SM_AFFINE | S.SPMV_FLAG_PERSISTENT)
    assert st == S.SPMV_E_INVALID and "flag" in msg.lower()
    # SB: row 0 (part 0) touches column 3, which is in C_1 -> structure error
    st, msg = _plan_status(form=S.SPMV_SB, K=2, row_part_ptr=np.array([0, 3, 6, 6]),
                           col_part_ptr=np.array([0, 3, 6, 6]))
    assert st == S.SPMV_E_STRUCTURE and "outside" in msg
    # SB with a non-empty row border
    st, _ = _plan_status(form=S.SPMV_SB, K=1, row_part_ptr=np.array([0, 5, 6]),
                         col_part_ptr=np.array([0, 6, 6]))
    assert st == S.SPMV_E_STRUCTURE
    st, _ = _plan_status(form=S.SPMV_SPLIT, K=2, nz_part=np.array([0, 1, 2, 0, 0, 0, 0]))
    assert st == S.SPMV_E_INVALID


def test_batched_plan_validation_before_any_device_call():
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    v = np.ones(2)
    mats = [(2, 2, rp, ci, v), (2, 2, rp, ci, v)]
    with pytest.raises(S.SpmvError) as e:
        S.spmv_plan_create_batched(mats, nz_parts=[np.array([0, 2]), np.array([0, 1])], K=2)
    assert e.value.status == S.SPMV_E_INVALID and "matrix 0" in str(e.value)
    bad = [(2, 2, rp, ci, v), (2, 2, np.array([0, 2, 1], dtype=np.int32), ci, v)]
    with pytest.raises(S.SpmvError) as e:
        S.spmv_plan_create_batched(bad)
    assert e.value.status == S.SPMV_E_INVALID and "matrix 1" in str(e.value)
    with pytest.raises(S.SpmvError) as e:
        S.spmv_plan_create_batched(mats, perms=[(np.array([0, 2]), None), None])
    assert e.value.status == S.SPMV_E_STRUCTURE

