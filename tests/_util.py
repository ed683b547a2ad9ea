"""Helpers shared by the tests: running a plan through the C ABI on torch
tensors and measuring the error against the oracle."""
import numpy as np

# |y - y_ref|_i <= tol * (|A||x|)_i, per value precision
TOL = {0: 1e-12, 1: 1e-5, 2: 1e-2}


def run_plan(S, plan, x, stream=None):
    """Permute x in, spmv_exec, permute y out; x is (n,) or (n, r) float64."""
    import torch
    dt = torch.float64 if plan.info["dtype"] == S.SPMV_F64 else torch.float32
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dt).reshape(-1)
    m = plan.info["m"]
    r = plan.info["nrhs"]
    xh = torch.empty_like(xd)
    yh = torch.full((m * r,), float("nan"), dtype=dt, device="cuda")
    y = torch.full((m * r,), float("nan"), dtype=dt, device="cuda")
    S.spmv_permute_x(plan, xd, xh, stream)
    S.spmv_exec(plan, xh, yh, stream)
    S.spmv_unpermute_y(plan, yh, y, stream)
    S.spmv_plan_check(plan, stream)         # no bounded device wait gave up
    torch.cuda.synchronize()
    out = y.double().cpu().numpy()
    return out.reshape(m, r) if np.ndim(x) == 2 else out


def err_ratio(y, y_ref, absax):
    y, y_ref, absax = (np.asarray(a, dtype=np.float64).reshape(-1) for a in (y, y_ref, absax))
    assert not np.any(np.isnan(y)), "unwritten output entries"
    err = np.abs(y - y_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(absax > 0, err / absax, np.where(err > 0, np.inf, 0.0))
    return float(ratio.max()) if ratio.size else 0.0
