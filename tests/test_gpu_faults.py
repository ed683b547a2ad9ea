"""Failure detection without a GPU fault: allocation failures injected on the
host through the plan's allocator hook are reported as SPMV_E_NOMEM, leave
nothing behind, and leave an existing plan usable; the status word of the
bounded device waits reads clean after normal work, and a wait made to run
out (a plan whose first wait on each staging copy polls zero times) is
reported as SPMV_E_TIMEOUT with the context still usable."""
import ctypes

import numpy as np
import pytest

import synth
from tests._util import run_plan

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


class _Allocator:
    """Device allocations through torch's caching allocator, failing from
    call number `fail_at` on (0: never fails)."""

    def __init__(self, fail_at=0):
        self.fail_at, self.calls, self.live = fail_at, 0, set()
        self.alloc_cb = S._ALLOC_T(self._alloc)
        self.free_cb = S._FREE_T(self._free)

    def _alloc(self, size, ctx):
        self.calls += 1
        if self.fail_at and self.calls >= self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(size))
        self.live.add(p)
        return p

    def _free(self, ptr, ctx):
        self.live.discard(ptr)
        torch.cuda.caching_allocator_delete(ptr)


def _create(rp, ci, v, m, n, alloc, **kw):
    A, keep = S._csr_struct(m, n, rp, ci, v)
    opts = S.spmv_opts(kw.get("dtype", 0), 1, 0, 0, 0, 0, kw.get("flags", 0), 0)
    opts.alloc, opts.release = alloc.alloc_cb, alloc.free_cb
    handle = ctypes.c_void_p()
    st = S.lib.spmv_plan_create(ctypes.byref(A), None, None, ctypes.byref(opts),
                                ctypes.byref(handle))
    return st, handle


def test_plan_creation_reports_allocation_failure():
    m = n = 4096
    rp, ci, v = synth.zipf_matrix(m, n, seed=3)
    for flags in (0, S.SPMV_FLAG_TILED_NATURAL):
        al = _Allocator(fail_at=1)
        st, h = _create(rp, ci, v, m, n, al, flags=flags)
        assert st == S.SPMV_E_NOMEM and not h.value
        assert b"allocation" in S.lib.spmv_last_error()
        assert not al.live


def test_host_io_allocation_failure_leaves_the_plan_usable():
    m = n = 4096
    rp, ci, v = synth.zipf_matrix(m, n, seed=4)
    al = _Allocator(fail_at=2)          # the plan's one allocation succeeds
    st, h = _create(rp, ci, v, m, n, al)
    assert st == S.SPMV_OK
    plan = S.Plan(h, None)
    plan.info = S.spmv_plan_get_info(plan)
    xh = np.zeros(n)
    yh = np.zeros(m)
    with pytest.raises(S.SpmvError) as e:
        S.spmv_exec_host(plan, xh, yh)
    assert e.value.status == S.SPMV_E_NOMEM
    # the device path still works and the status word is clean
    x = synth.integer_x(n, 5)
    y = run_plan(S, plan, x)
    import oracle
    y_ref, _ = oracle.spmv(m, n, rp, ci, v, x)
    assert np.allclose(y, y_ref, rtol=1e-12, atol=1e-9)
    S.spmv_plan_check(plan)
    S.spmv_plan_destroy(plan)
    assert not al.live


def test_bounded_wait_that_runs_out_reports_timeout():
    """The staged tiles of a plan built with SPMV_FLAG_TEST_WAIT_EXPIRES give
    up their first wait at once: they raise the status word, wait (bounded)
    for their copy and skip their rows.  spmv_plan_check reports
    SPMV_E_TIMEOUT; the device stays usable for the next plan."""
    import oracle
    nx = 64
    rp, ci, v = synth.mesh5(nx, seed=5)
    m = n = nx * nx
    lab = (np.arange(m) * 8 // m).astype(np.int32)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, 8, lab)
    kw = dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SB, K=8, row_part_ptr=rpp,
              col_part_ptr=cpp, tile_nnz=2048)
    bad = S.spmv_plan_create(m, n, rp, ci, v,
                             flags=S.SPMV_FLAG_STAGE | S.SPMV_FLAG_TEST_WAIT_EXPIRES, **kw)
    assert bad.info["n_staged_tiles"] > 0
    x = torch.from_numpy(synth.uniform_x(n, 6)).cuda()
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    S.spmv_exec(bad, x, y)
    with pytest.raises(S.SpmvError) as e:
        S.spmv_plan_check(bad)
    assert e.value.status == S.SPMV_E_TIMEOUT
    S.spmv_plan_destroy(bad)
    good = S.spmv_plan_create(m, n, rp, ci, v, flags=S.SPMV_FLAG_STAGE, **kw)
    xs = synth.uniform_x(n, 7)
    y = run_plan(S, good, xs)
    y_ref, absax = oracle.spmv(m, n, rp, ci, v, xs)
    assert np.all(np.abs(y - y_ref) <= 1e-12 * absax)
    S.spmv_plan_check(good)
    S.spmv_plan_destroy(good)
