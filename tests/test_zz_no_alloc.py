"""The entry point that allocates nothing (spmv_csr_exec_noalloc).

It is meant for callers that cannot allocate device memory when they need a
product -- code running inside a memory pool it does not own, a plugin handed
only its buffers, a step that must leave the allocator alone.  Its partial
sums live in a fixed scratch array compiled into the library.  Here its output
is checked, through the C ABI, against the CPU oracle's y and |A||x| with the
FP64 tolerance of the other tests, and against the planned entry point
(spmv_exec on a natural-order FP64 plan), on two calls in a row; after the
set-up call, the free device memory and torch's allocated bytes must not
change across calls.  This file is collected last, so that a run stopping at
its first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

import synth
from tests._util import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _matrix():
    # power-law rows, one row crossing many 4096-nonzero chunks, empty rows
    m = n = 16384
    rp, ci, v = synth.zipf_matrix(m, n, seed=4)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
    keep = ((rows % 97) != 5) & (rows != 7)     # some empty rows; row 7 rebuilt dense
    rows, cols, vals = rows[keep], ci[keep].astype(np.int64), v[keep]
    rows = np.concatenate([rows, np.full(n, 7)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, synth.uniform_x(n, 9)])
    return (m, n) + synth.coo_to_csr(m, n, rows, cols, vals)


def test_noalloc_matches_oracle_and_planned_entry_point_two_calls():
    import oracle
    import paper_1203_2739_gb300 as S
    torch.cuda.set_device(0)
    m, n, rp, ci, v = _matrix()
    assert int(np.diff(rp).max()) > 3 * 4096     # one row spans several chunks
    assert int((np.diff(rp) == 0).sum()) > 0     # and some rows are empty
    plan = S.spmv_plan_create(m, n, rp, ci, v)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    d_v = torch.from_numpy(v).cuda()
    xs = [synth.uniform_x(n, seed) for seed in (1, 2)]
    dx = [torch.from_numpy(x).cuda() for x in xs]
    y_plan = torch.empty(m, dtype=torch.float64, device="cuda")
    y_noalloc = torch.empty(m, dtype=torch.float64, device="cuda")
    # set-up call (m = 0): loads the entry point's module and kernels
    assert S.lib.spmv_csr_exec_noalloc(0, 0, 0, None, None, None, None, None, None) == S.SPMV_OK
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for call, (x, xd) in enumerate(zip(xs, dx)):
        y_noalloc.fill_(float("nan"))
        S.spmv_csr_exec_noalloc(m, n, d_rp, d_ci, d_v, xd, y_noalloc)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "call %d changed free device memory" % call
        assert torch.cuda.memory_allocated() == alloc0, "call %d allocated through torch" % call
        S.spmv_exec(plan, xd, y_plan)
        torch.cuda.synchronize()
        b = y_noalloc.cpu().numpy()
        assert not np.isnan(b).any(), "call %d left entries unwritten" % call
        y_ref, absax = oracle.spmv(m, n, rp, ci, v, x)
        tol = TOL[S.SPMV_F64] * absax
        err = np.abs(b - y_ref)
        assert np.all(err <= tol), (call, float((err / np.maximum(absax, 1e-300)).max()))
        # and the planned entry point, held to the same oracle
        assert np.all(np.abs(y_plan.cpu().numpy() - y_ref) <= tol), call
    S.spmv_plan_destroy(plan)


def test_noalloc_edges_and_limit():
    import paper_1203_2739_gb300 as S
    torch.cuda.set_device(0)
    # no nonzeros: y is all zeros
    m, n = 37, 5
    rp = torch.zeros(m + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    v = torch.zeros(0, dtype=torch.float64, device="cuda")
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    y = torch.full((m,), 3.0, dtype=torch.float64, device="cuda")
    S.spmv_csr_exec_noalloc(m, n, rp, ci, v, x, y)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0
    # more nonzeros than the scratch array covers: rejected before any launch
    st = S.lib.spmv_csr_exec_noalloc(10, 10, S.SPMV_NOALLOC_MAX_NNZ + 1, None, None, None, None,
                                     None, None)
    assert st == S.SPMV_E_UNSUPPORTED and "scratch" in S.spmv_last_error()
