"""Mixed-precision CG with FP64 iterative refinement (spmv_cg_ir) on a
symmetrically permuted 3D Laplacian, through the C ABI: the solver's FP64
residual must reach 1e-10, recomputed here by the CPU oracle, for FP64, FP32
and BF16 inner products, in natural order and in the SB / DB forms (whose
row and column permutations differ, so the solver moves products between
the two spaces)."""
import numpy as np
import pytest

import oracle
import synth

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


@pytest.fixture(scope="module")
def lap():
    rp, ci, v = synth.laplacian3d(16, seed=3)
    n = len(rp) - 1
    x_star = synth.uniform_x(n, 4)
    b, _ = oracle.spmv(n, n, rp, ci, v, x_star)
    return n, rp, ci, v, b, x_star


def _form(n, rp, ci, form):
    if form == "natural":
        return {}
    meth = {"sb": S.SPMV_PART_CN, "db": S.SPMV_PART_ERCN}[form]
    part = S.spmv_partition(n, n, rp, ci, meth, K=8, seed=1)
    assert not np.array_equal(part["row_perm"], part["col_perm"])
    return dict(row_perm=part["row_perm"], col_perm=part["col_perm"], form=part["form"],
                K=part["K"], row_part_ptr=part["row_part_ptr"], col_part_ptr=part["col_part_ptr"])


def _rel_residual(n, rp, ci, v, b, x):
    ax, _ = oracle.spmv(n, n, rp, ci, v, x)
    return float(np.linalg.norm(b - ax) / np.linalg.norm(b))


@pytest.mark.parametrize("form", ["natural", "sb", "db"])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_cg_ir_reaches_fp64_residual(lap, form, dtype):
    n, rp, ci, v, b, x_star = lap
    kw = _form(n, rp, ci, form)
    low = S.spmv_plan_create(n, n, rp, ci, v, dtype=dtype, **kw)
    f64 = S.spmv_plan_create(n, n, rp, ci, v, dtype=0, **kw)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = S.spmv_cg_ir(low, f64, bd, xd, tol=1e-10)
    x = xd.cpu().numpy()
    assert info["converged"], info
    assert info["rel_residual"] <= 1e-10
    # the oracle's own FP64 residual of the returned solution
    assert _rel_residual(n, rp, ci, v, b, x) <= 1.5e-10
    # and the solution against the one that generated b (kappa ~ 100 here)
    assert np.linalg.norm(x - x_star) / np.linalg.norm(x_star) <= 1e-7
    if dtype != 0:
        assert info["outer"] >= 2          # refinement did the last digits
    # the oracle's CG agrees
    xo, _, rel = oracle.cg(n, rp, ci, v, b, tol=1e-12)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-7


def test_cg_ir_initial_guess_and_repeat(lap):
    n, rp, ci, v, b, x_star = lap
    low = S.spmv_plan_create(n, n, rp, ci, v, dtype=1)
    f64 = S.spmv_plan_create(n, n, rp, ci, v, dtype=0)
    bd = torch.from_numpy(b).cuda()
    xd = torch.from_numpy(x_star).cuda().clone()
    info = S.spmv_cg_ir(low, f64, bd, xd, tol=1e-10)
    assert info["converged"] and info["outer"] == 0 and info["inner_total"] == 0
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    a = S.spmv_cg_ir(low, f64, bd, xd, tol=1e-10)
    x1 = xd.clone()
    xd.zero_()
    c = S.spmv_cg_ir(low, f64, bd, xd, tol=1e-10)
    assert a == c
    assert torch.equal(x1, xd)             # deterministic reductions


def test_cg_ir_rejects_bad_input(lap):
    n, rp, ci, v, b, _ = lap
    low = S.spmv_plan_create(n, n, rp, ci, v, dtype=1)
    f32 = S.spmv_plan_create(n, n, rp, ci, v, dtype=1)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SpmvError, match="SPMV_F64"):
        S.spmv_cg_ir(low, f32, bd, xd)
    # -A is negative definite: CG breaks down at once and says so
    neg_low = S.spmv_plan_create(n, n, rp, ci, -v, dtype=1)
    neg64 = S.spmv_plan_create(n, n, rp, ci, -v, dtype=0)
    with pytest.raises(S.SpmvError, match="positive definite"):
        S.spmv_cg_ir(neg_low, neg64, bd, xd)
    rp2, ci2, v2 = synth.laplacian3d(8, seed=0)
    other = S.spmv_plan_create(len(rp2) - 1, len(rp2) - 1, rp2, ci2, v2, dtype=0)
    with pytest.raises(S.SpmvError, match="same square matrix"):
        S.spmv_cg_ir(low, other, bd, xd)


def test_cg_ir_bf16_values_that_round():
    """A shifted graph Laplacian with random edge weights: BF16 rounds its
    values (unlike the 6 / -1 of the plain Laplacian), so the inner products
    use a perturbed matrix and the FP64 refinement has to make up for it.
    The FP64 residual still reaches 1e-10 (the oracle's own residual of the
    returned x agrees), with more refinement steps than FP32 needs."""
    rp, ci, v = synth.weighted_laplacian3d(16, seed=5)
    n = len(rp) - 1
    bf = v.astype(np.float32).view(np.uint32) & 0xFFFF0000
    assert np.mean(bf.view(np.float32).astype(np.float64) != v) > 0.9
    b, _ = oracle.spmv(n, n, rp, ci, v, synth.uniform_x(n, 6))
    bd = torch.from_numpy(b).cuda()
    f64 = S.spmv_plan_create(n, n, rp, ci, v, dtype=0)
    outer = {}
    for dtype in (1, 2):
        low = S.spmv_plan_create(n, n, rp, ci, v, dtype=dtype)
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = S.spmv_cg_ir(low, f64, bd, xd, tol=1e-10)
        assert info["converged"] and info["rel_residual"] <= 1e-10, (dtype, info)
        assert _rel_residual(n, rp, ci, v, b, xd.cpu().numpy()) <= 1.5e-10
        outer[dtype] = info["outer"]
    assert outer[2] > outer[1] >= 2, outer
