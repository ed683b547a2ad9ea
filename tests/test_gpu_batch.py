"""Batched plans (many matrices, one launch per exec) and a CUDA graph of 100
repeated split products, through the C ABI, against the oracle per matrix.
Integer data make every sum exact, so results are compared bit-exactly."""
import numpy as np
import pytest

import oracle
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


def _batch(seed):
    mats = []
    rp, ci, _ = synth.zipf_matrix(1000, 1200, seed=seed)
    mats.append((1000, 1200, rp, ci))
    rp, ci, _ = synth.random_sparse(300, 50, 0.2, seed + 1)
    mats.append((300, 50, rp, ci))
    mats.append((10, 7, np.zeros(11, dtype=np.int32), np.zeros(0, dtype=np.int32)))
    rp, ci, _ = synth.mesh5(40, seed=seed + 2)
    mats.append((1600, 1600, rp, ci))
    rp, ci, _ = synth.zipf_matrix(5000, 5000, seed=seed + 3)
    mats.append((5000, 5000, rp, ci))
    out = []
    for b, (m, n, rp, ci) in enumerate(mats):
        out.append((m, n, rp, ci, synth.integer_values(int(rp[-1]), seed + 10 + b)))
    return out


def _expected(mats, xs):
    ys = []
    for (m, n, rp, ci, v), x in zip(mats, xs):
        y, _ = oracle.spmv(m, n, rp, ci, v, x)
        ys.append(y)
    return np.concatenate(ys)


def _perms(mats, seed):
    out = []
    for b, (m, n, rp, ci, v) in enumerate(mats):
        out.append((synth.random_perm(m, seed + b), synth.random_perm(n, seed + 50 + b))
                   if b % 2 == 0 else None)
    return out


@pytest.mark.parametrize("dtype,nrhs", [(0, 1), (1, 1), (2, 8), (0, 8)])
@pytest.mark.parametrize("split", [False, True])
def test_batched_plan_exact(dtype, nrhs, split):
    mats = _batch(7)
    K = 16
    nz = [synth.random_labels(int(rp[-1]), K, 100 + b) for b, (m, n, rp, ci, v)
          in enumerate(mats)] if split else None
    plan = S.spmv_plan_create_batched([(m, n, rp, ci, v) for (m, n, rp, ci, v) in mats],
                                      perms=_perms(mats, 3), nz_parts=nz, K=K, dtype=dtype,
                                      nrhs=nrhs)
    M = sum(m for m, *_ in mats)
    N = sum(n for _, n, *_ in mats)
    assert plan.info["m"] == M and plan.info["n"] == N
    assert plan.info["launches_per_exec"] <= 2
    xs = [synth.integer_x(n, 200 + b, nrhs=nrhs) for b, (m, n, *_) in enumerate(mats)]
    y = run_plan(S, plan, np.concatenate(xs))
    assert np.array_equal(y, _expected(mats, xs))


def test_graph_of_repeated_split_products():
    mats = _batch(11)
    K = 16
    nz = [synth.random_labels(int(rp[-1]), K, 300 + b) for b, (m, n, rp, ci, v)
          in enumerate(mats)]
    plan = S.spmv_plan_create_batched([(m, n, rp, ci, v) for (m, n, rp, ci, v) in mats],
                                      nz_parts=nz, K=K, dtype=1)
    xs = [synth.integer_x(n, 400 + b) for b, (m, n, *_) in enumerate(mats)]
    x = torch.from_numpy(np.concatenate(xs)).float().cuda()
    ys = [torch.full((plan.info["m"],), float("nan"), device="cuda") for _ in range(100)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        S.spmv_exec(plan, x, ys[0])       # first call outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for i in range(100):
            S.spmv_exec(plan, x, ys[i])
    for t in ys:
        t.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    want = _expected(mats, xs)
    for t in ys:
        assert np.array_equal(t.double().cpu().numpy(), want)
    S.spmv_plan_check(plan)
