"""Benchmark of the repeated SpMV y <- A x over reordered and split matrices.

One step = one y <- A x on every (matrix, form) pair of the workload, each
plan reading its own x_hat and writing its own y_hat (device-resident inputs).
The default workload is the FP64 reordering sweep: three 1,048,576-row
matrices (5-point 1024^2 mesh, randomly permuted; R-MAT a,b,c = .57,.19,.19
with 16 nonzeros per row; 64 diagonal 16,384^2 blocks at 0.2% fill plus 5%
random off-block nonzeros, shuffled), each in natural order, a random
symmetric permutation, the 1D SB form (column-net partitioning), the 2D DB
form (enhanced row-column-net) and splits with K = 4, 16, 64, 256
(row-column-net).

Metric: compulsory-bytes SpMV throughput, GB/s = sum over the step of
[nnz*(8+4) + (m+1)*4 + n*8 + m*8] / time (Sec. 2.2 streaming model), with
GFLOP/s = 2 nnz / time and the roofline of the dominant kernel against the
measured HBM copy bandwidth.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload sweep|zipf16k|precision]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FORMS_SWEEP = ["natural", "random", "sb", "db", "split4", "split16", "split64", "split256"]


# ----------------------------------------------------------------- inputs --
def make_matrices(workload):
    if workload == "sweep":
        return [("mesh5_1024", synth.mesh5(1024, seed=0)),
                ("rmat20_d16", synth.rmat(20, 16, seed=0)),
                ("blocks64_0.2pct", synth.blocks(seed=0))]
    if workload == "zipf16k":
        return [("zipf16k", synth.zipf_matrix(seed=0))]
    if workload == "precision":
        return [("laplace3d_128", synth.laplacian3d(128, seed=0))]
    raise ValueError(workload)


def sizes(rp, n):
    return len(rp) - 1, n, int(rp[-1])


def compulsory_bytes(m, n, nnz, vb=8, xb=8, r=1):
    return nnz * (vb + 4) + (m + 1) * 4 + n * xb * r + m * xb * r


# ---------------------------------------------------------------- forms --
def build_forms(S, name, rp, ci, n, forms, seed=0, log=None):
    """Partition (host) for every requested form; returns {form: kwargs for
    spmv_plan_create} and partition timings."""
    m = len(rp) - 1
    out, ptime = {}, {}
    for f in forms:
        t0 = time.perf_counter()
        if f == "natural":
            out[f] = {}
        elif f == "tiled":
            # natural order through the tiled kernel
            out[f] = dict(flags=S.SPMV_FLAG_TILED_NATURAL)
        elif f == "random":
            p = synth.random_perm(m, 1000 + seed)
            q = p if m == n else synth.random_perm(n, 2000 + seed)
            out[f] = dict(row_perm=p, col_perm=q)
        elif f == "sbblock":
            # trivial SB: K contiguous row blocks (any row partition is an SB form)
            K = 64
            lab = (np.arange(m, dtype=np.int64) * K // m).astype(np.int32)
            rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, K, lab)
            out[f] = dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SB, K=K,
                          row_part_ptr=rpp, col_part_ptr=cpp)
        elif f == "splitblock":
            # trivial split: a 4 x 4 grid of row/column blocks
            q = 4
            rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
            lab = ((rows * q // m) * q + (ci.astype(np.int64) * q // n)).astype(np.int32)
            rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, q * q,
                                                             lab)
            out[f] = dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SPLIT, K=q * q,
                          row_part_ptr=rpp, col_part_ptr=cpp, nz_part=lab)
        elif f[:2] in ("sb", "db") and f not in ("sbblock",):
            method = S.SPMV_PART_CN if f.startswith("sb") else S.SPMV_PART_ERCN
            if len(f) > 2:      # fixed K: bisect to depth log2(K)
                res = S.spmv_partition(m, n, rp, ci, method, K=int(f[2:]), seed=seed)
            else:               # size rule: bisect until the x subvector fits
                res = S.spmv_partition(m, n, rp, ci, method, part_bytes=_part_bytes(f),
                                       fit_rule=S.SPMV_FIT_X, seed=seed)
            out[f] = dict(row_perm=res["row_perm"], col_perm=res["col_perm"], form=res["form"],
                          K=res["K"], row_part_ptr=res["row_part_ptr"],
                          col_part_ptr=res["col_part_ptr"])
            out[f]["_cost"] = res["cost"]
        elif f.startswith("split"):
            K = int(f[5:])
            res = _split_cache(S, rp, ci, m, n, K, seed)
            out[f] = dict(row_perm=res["row_perm"], col_perm=res["col_perm"],
                          form=S.SPMV_SPLIT, K=K, row_part_ptr=res["row_part_ptr"],
                          col_part_ptr=res["col_part_ptr"], nz_part=res["labels"])
            out[f]["_cost"] = res["cost"]
        ptime[f] = time.perf_counter() - t0
        if log:
            log("  %s/%s: partition %.1fs" % (name, f, ptime[f]))
    return out, ptime


_SPLIT_TREE = {}


def _split_cache(S, rp, ci, m, n, K, seed):
    """Row-column-net bisection to depth log2(256) once; K-way splits for
    smaller K are the levels of the same recursion tree (labels >> shift)."""
    key = (id(rp), seed)
    if key not in _SPLIT_TREE:
        _SPLIT_TREE[key] = S.spmv_partition(m, n, rp, ci, S.SPMV_PART_RCN, K=256, seed=seed)
    full = _SPLIT_TREE[key]
    shift = int(np.log2(256 // K))
    lab = (full["labels"] >> shift).astype(np.int32)
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, K, lab)
    return dict(labels=lab, row_perm=rperm, col_perm=cperm, row_part_ptr=rpp,
                col_part_ptr=cpp, cost=None)


def _part_bytes(form):
    # x-subvector budget per part: the default staging capacity of one tile
    return 48 * 1024


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------- measured peak --
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1203_2739_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(label):
    """DRAM bytes per launch recorded from an ncu capture of the current kernel
    sources (profiles/ncu_traffic.json); None when absent or stale."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    e = d.get("entries", {}).get(label)
    return None if e is None else e.get("dram_bytes_per_launch")


# ------------------------------------------------------------- reference --
def run_reference(args, rank, world):
    """The oracle timed on the host cores, on a bounded sample per step."""
    if rank != 0:
        return
    import oracle
    mats = make_matrices(args.workload)
    # one oracle SpMV of one matrix per step, cycling through the matrices
    prepared = []
    for name, (rp, ci, v) in mats:
        n = len(rp) - 1          # every workload matrix is square
        prepared.append((name, rp.astype(np.int64), ci, v, synth.uniform_x(n, 0), n))
    for w in range(args.warmup):
        name, rp, ci, v, xx, n = prepared[w % len(prepared)]
        oracle.spmv(len(rp) - 1, n, rp, ci, v, xx)
    tot_bytes, tot_flops, t = 0, 0, 0.0
    for s in range(args.steps):
        name, rp, ci, v, xx, n = prepared[s % len(prepared)]
        m = len(rp) - 1
        t0 = time.perf_counter()
        oracle.spmv(m, n, rp, ci, v, xx)
        t += time.perf_counter() - t0
        tot_bytes += compulsory_bytes(m, n, int(rp[-1]))
        tot_flops += 2 * int(rp[-1])
    gbs = tot_bytes / t / 1e9
    line = {
        "impl": "reference", "metric": "SpMV GB/s (compulsory bytes)", "value": round(gbs, 3),
        "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t / max(args.steps, 1), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload,
                   "sample": "one FP64 oracle SpMV (compensated sums, 1 thread) of one sweep "
                             "matrix per step, cycling mesh/R-MAT/blocks"},
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "%d oracle SpMVs over the workload's matrices" % args.steps},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gflops": round(tot_flops / t / 1e9, 3),
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(mats, budget_s=15.0):
    """Oracle SpMV on the host on a bounded sample (whole matrices, cycling)."""
    import oracle
    t_tot, b_tot, count = 0.0, 0, 0
    names = []
    while t_tot < budget_s and count < 3 * len(mats):
        name, (rp, ci, v), n = mats[count % len(mats)]
        m = len(rp) - 1
        x = synth.uniform_x(n, 0)
        rp64 = rp.astype(np.int64)
        t0 = time.perf_counter()
        oracle.spmv(m, n, rp64, ci, v, x)
        t_tot += time.perf_counter() - t0
        b_tot += compulsory_bytes(m, n, int(rp[-1]))
        count += 1
        names.append(name)
    return {"value": round(b_tot / t_tot / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "%d FP64 oracle SpMVs (natural order, compensated sums): %s"
                      % (count, ",".join(names))}


# ------------------------------------------------------------------- ours --
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1203_2739_gb300 as S
    from tests._util import err_ratio   # test helper only measures the error
    import oracle

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    log = (lambda s: print(s, file=sys.stderr, flush=True)) if rank == 0 else (lambda s: None)
    forms = args.forms.split(",") if args.forms else (
        FORMS_SWEEP if args.workload == "sweep" else ["natural", "sb"])
    t_setup = time.perf_counter()
    mats = []
    for name, (rp, ci, v) in make_matrices(args.workload):
        n = len(rp) - 1
        mats.append((name, (rp, ci, v), n))
        log("generated %s: m=%d nnz=%d" % (name, n, int(rp[-1])))

    dtype = {"f64": S.SPMV_F64, "f32": S.SPMV_F32, "bf16": S.SPMV_BF16}[args.dtype]
    entries = []   # (label, plan, x_hat, y_hat, bytes, flops, err)
    stream = torch.cuda.current_stream()
    part_times = {}
    for name, (rp, ci, v), n in mats:
        m = len(rp) - 1
        fk, pt = build_forms(S, name, rp, ci, n, forms, log=log)
        x = synth.uniform_x(n, 1)
        y_ref, absax = oracle.spmv(m, n, rp, ci, v, x)
        for f in forms:
            kw = {k: val for k, val in fk[f].items() if not k.startswith("_")}
            plan = S.spmv_plan_create(m, n, rp, ci, v, dtype=dtype, **kw)
            xt = torch.from_numpy(x).to(dev, dtype=torch.float64 if dtype == 0 else torch.float32)
            xh = torch.empty_like(xt)
            S.spmv_permute_x(plan, xt, xh)
            yh = torch.empty(m, dtype=xt.dtype, device=dev)
            S.spmv_exec(plan, xh, yh)
            y = torch.empty_like(yh)
            S.spmv_unpermute_y(plan, yh, y)
            torch.cuda.synchronize()
            err = err_ratio(y.double().cpu().numpy(), y_ref, absax)
            info = plan.info
            entries.append(dict(label="%s/%s" % (name, f), plan=plan, xh=xh, yh=yh,
                                bytes=compulsory_bytes(m, n, int(rp[-1]),
                                                       vb={0: 8, 1: 4, 2: 2}[dtype],
                                                       xb=8 if dtype == 0 else 4),
                                flops=2 * int(rp[-1]), err=err, info=info,
                                cost=fk[f].get("_cost"), ptime=pt[f]))
            log("  plan %s/%s: K=%d tiles=%d staged=%d lanes=%d err=%.2e" % (
                name, f, info["K"], info["n_tiles"], info["n_staged_tiles"], info["lanes"], err))
        del y_ref, absax
    setup_s = time.perf_counter() - t_setup

    def step(events=None):
        for i, e in enumerate(entries):
            if events is not None:
                events[i][0].record(stream)
            S.spmv_exec(e["plan"], e["xh"], e["yh"], stream)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in entries] for _ in range(args.steps)]
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    if dist:
        tt = torch.tensor([elapsed_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
        torch.distributed.barrier()
    per = np.array([[a.elapsed_time(b) for (a, b) in row] for row in ev])   # steps x entries
    mean_ms = per.mean(axis=0)

    # end to end through the host-buffer entry point (copies in the timed region)
    e2e = None
    if not args.no_e2e:
        hx = [e["xh"].cpu().pin_memory() for e in entries]
        hy = [torch.empty(e["yh"].numel(), dtype=e["yh"].dtype).pin_memory() for e in entries]
        for i, e in enumerate(entries):
            S.spmv_exec_host(e["plan"], hx[i], hy[i])
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 5))
        ta = time.perf_counter()
        for _ in range(e2e_steps):
            for i, e in enumerate(entries):
                S.spmv_exec_host(e["plan"], hx[i], hy[i])
        tb = time.perf_counter()
        step_bytes = sum(e["bytes"] for e in entries)
        e2e = {"value": round(step_bytes * e2e_steps / (tb - ta) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hx)),
               "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hy))}

    step_bytes = sum(e["bytes"] for e in entries)
    step_flops = sum(e["flops"] for e in entries)
    ms_per_step = elapsed_ms / args.steps
    value = world * step_bytes / (ms_per_step * 1e-3) / 1e9
    if rank != 0:
        return
    peak, peak_kind = measured_peak()
    dom = int(np.argmax(mean_ms))
    d = entries[dom]
    achieved = d["bytes"] / (mean_ms[dom] * 1e-3) / 1e9
    detail = {}
    for i, e in enumerate(entries):
        gbs = e["bytes"] / (mean_ms[i] * 1e-3) / 1e9
        detail[e["label"]] = {
            "us": round(1e3 * mean_ms[i], 2), "GBps": round(gbs, 1),
            "GFLOPs": round(e["flops"] / (mean_ms[i] * 1e-3) / 1e9, 1),
            "frac": round(gbs / peak, 3), "err": e["err"], "K": e["info"]["K"],
            "tiles": e["info"]["n_tiles"], "staged_tiles": e["info"]["n_staged_tiles"],
            "launches": e["info"]["launches_per_exec"],
            "moved_over_compulsory": round(e["info"]["moved_bytes"] / e["bytes"], 3),
            "partition_s": round(e["ptime"], 2), "cost": e["cost"]}
    # natural FP64 CSR vs the best form, per matrix
    best = {}
    for e_label, dd in detail.items():
        mat, form = e_label.split("/")
        if mat not in best or dd["us"] < best[mat][1]:
            best[mat] = (form, dd["us"])
    speedup = {mat: {"best_form": best[mat][0],
                     "speedup_vs_natural": round(detail[mat + "/natural"]["us"] / best[mat][1], 3)
                     if (mat + "/natural") in detail else None} for mat in best}
    line = {
        "metric": "SpMV GB/s (compulsory bytes; % of GB300 HBM roofline)",
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": args.workload, "matrices": [m[0] for m in mats], "forms": forms,
                   "unit_of_work": "one y<-Ax per (matrix, form) per step",
                   "l2": "inputs larger than L2: each step streams %.2f GB over %d plans"
                         % (step_bytes / 1e9, len(entries)),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "gflops": round(world * step_flops / (ms_per_step * 1e-3) / 1e9, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "kernel": d["label"], "traffic": ncu_traffic(d["label"])},
        "gpu_launches": int(args.steps * sum(e["info"]["launches_per_exec"] for e in entries)),
        "clocks": clk,
        "e2e": e2e,
        "max_err_ratio": max(e["err"] for e in entries),
        "speedup_vs_natural": speedup,
        "detail": detail,
        "setup_s": round(setup_s, 1),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(mats, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep", choices=["sweep", "zipf16k", "precision"])
    ap.add_argument("--forms", default="")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: warmup raised to 3", file=sys.stderr)
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
