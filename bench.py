"""Benchmark of the repeated SpMV y <- A x over reordered and split matrices.

One step = one y <- A x on every (matrix, form) pair of the workload, each
plan reading its own x_hat and writing its own y_hat (device-resident inputs).
The default workload is the FP64 reordering sweep: three 1,048,576-row
matrices (5-point 1024^2 mesh, randomly permuted; R-MAT a,b,c = .57,.19,.19
with 16 nonzeros per row; 64 diagonal 16,384^2 blocks at 0.2% fill plus 5%
random off-block nonzeros, shuffled), each in natural order and after a
random symmetric permutation (through the plain CSR kernel and through the
tiled kernel), in the paper's comparison orders (sBFS and sRCM on the
bipartite graph, sHP_RN: row-net bisection, K = 1024), in the 1D SB form
(column-net bisection, K = 1024: about one part per resident CTA of a
launch), the 2D DB form (enhanced row-column-net bisection, K = 1024) and as
splits with K = 4, 16, 64, 256 (row-column-net bisection; the smaller K are
levels of the same recursion tree).

Metric: compulsory-bytes SpMV throughput, GB/s = sum over the step of
[nnz*(vb+4) + (m+1)*4 + n*xb + m*xb] / time (Sec. 2.2 streaming model), with
GFLOP/s = 2 nnz / time and the roofline of the dominant kernel against the
measured HBM copy bandwidth.

Other workloads: precision (CG with FP64 refinement over FP64 / FP32 / BF16
products on a 3D Laplacian), batching (256 R-MAT matrices of 1,024-262,144
rows in one plan, natural vs split K = 16, plus 100 products replayed from a
CUDA graph), scale (a mesh whose x exceeds L2), zipf16k, selector.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload sweep|zipf16k|precision|batching|scale|selector]
                       [--forms a,b,...] [--dtype f64|f32|bf16] [--nrhs 1|2|4|8]
                       [--batch-count B] [--batch-max-rows M]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# natural and random orders run through both the plain CSR kernel and the
# tiled kernel ("tiled", "rtiled"), so that the gain of a reordering is
# measured against the same kernel in the original order
FORMS_SWEEP = ["natural", "random", "tiled", "rtiled", "bfs", "rcm", "rn1024", "sb1024", "sbfit96",
               "db1024", "split4", "split16", "split64", "split256"]
NATURAL_FORMS = ("natural", "random", "tiled", "rtiled")
MATRICES = {
    "sweep": [("mesh5_1024", lambda: synth.mesh5(1024, seed=0)),
              ("rmat20_d16", lambda: synth.rmat(20, 16, seed=0)),
              ("blocks64_0.2pct", lambda: synth.blocks(seed=0))],
    "zipf16k": [("zipf16k", lambda: synth.zipf_matrix(seed=0))],
    "precision": [("laplace3d_128", lambda: synth.laplacian3d(128, seed=0))],
    "scale": [("mesh5_6144", lambda: _mesh_with_points("mesh5_6144", 6144))],
    "batching": [("rmat_batch256", lambda: _batch_matrix("rmat_batch256"))],
}
# tile shape per "matrix/form" label taken instead of the autotuner's choice
# (--shape-map: a bench JSON line's detail, or a {label: shape} object), so
# that a profiled run launches the kernels a timed run chose
SHAPE_MAP = {}

def load_shape_map(path):
    """{matrix/form: tile shape} from a JSON object of that form or from a
    bench run's output (its last line's detail)."""
    with open(path) as fh:
        text = fh.read().strip()
    try:
        d = json.loads(text)
    except ValueError:
        d = json.loads(text.splitlines()[-1])
    if "detail" in d:
        d = {k: e["tile_shape"] for k, e in d["detail"].items() if e.get("tile_shape")}
    return d


# grid point of every row of the meshes generated with their points (the
# scale workload's SB form is cut from the grid)
MESH_POINTS = {}


def _mesh_with_points(name, nx):
    rp, ci, v, pts = synth.mesh5(nx, seed=0, return_points=True)
    MESH_POINTS[name] = (nx, pts)
    return rp, ci, v


# the batching workload: member count, largest member's rows, split K values
# to partition for, partition cache
BATCH = {"count": 256, "max_rows": 262144, "K": (16,), "cache": None}
BATCHES = {}
BATCH_LABELS = {}


def _batch_member(spec):
    """Worker (spawned process, no GPU): one member of the batch and its
    row-column-net splits (Sec. 4.1) for each K."""
    scale, deg, seed, Ks, cache = spec
    import paper_1203_2739_gb300 as S
    m, n, rp, ci, v = synth.rmat_batch_member(scale, deg, seed)
    labels = {}
    for K in Ks:
        path = (os.path.join(cache, "batch_s%d_d%d_seed%d_rcn%d.npy" % (scale, deg, seed, K))
                if cache else None)
        if path and os.path.exists(path):
            labels[K] = np.load(path)
            continue
        labels[K] = S.spmv_partition(m, n, rp, ci, S.SPMV_PART_RCN, K=K, seed=0,
                                     threads=1)["labels"]
        if path:
            os.makedirs(cache, exist_ok=True)
            np.save(path, labels[K])
    return (m, n, rp, ci, v), labels


def _batch_matrix(name):
    """The batch as one block-diagonal CSR (the natural-form baseline runs it
    as one matrix); the member matrices and their splits are kept for the
    batched plan.  Members are generated and partitioned on spawned host
    processes, largest first."""
    import multiprocessing as mp
    specs = synth.rmat_batch_specs(BATCH["count"], hi=BATCH["max_rows"], seed=0)
    order = sorted(range(len(specs)), key=lambda b: -(specs[b][1] << specs[b][0]))
    # at most 32 workers: each holds one member and its hypergraph (up to a
    # few GB for the largest)
    with mp.get_context("spawn").Pool(max(1, min(32, os.cpu_count() or 4))) as pool:
        res = pool.map(_batch_member, [specs[b] + (tuple(BATCH["K"]), BATCH["cache"])
                                       for b in order], chunksize=1)
    mats, labels = [None] * len(specs), [None] * len(specs)
    for b, (mat, lab) in zip(order, res):
        mats[b], labels[b] = mat, lab
    BATCHES[name], BATCH_LABELS[name] = mats, labels
    return synth.block_diagonal(mats)
WORKLOAD_TEXT = {
    "sweep": "FP64 reordering sweep: mesh 1024^2 (5-pt, permuted), R-MAT 2^20 deg 16, "
             "64 blocks of 16384^2 at 0.2% + 5% border (shuffled); natural, random (plain CSR "
             "and tiled kernel), sBFS, sRCM, sHP_RN K=1024, SB K=1024, SB by the fit rule "
             "(x subvector of each part < 96 KB), DB K=1024, "
             "split K=4/16/64/256",
    "zipf16k": "Zipf 16384^2 (rows P(d)~d^-1.7498 on [1,512], Zipf(1.2) columns), natural vs SB",
    "batching": "256 R-MAT matrices (rows log-uniform in [1024, 262144], power-of-two sizes, "
                "degree U[8,32]) in one plan: natural block-diagonal through the plain CSR and "
                "the tiled kernel vs batched split K=16 (row-column-net bisection of each "
                "matrix); FP32 with --dtype f32",
    "scale": "L2-exceeding point: 5-pt mesh 6144^2 (37.7M rows, 188.7M nnz, x = 302 MB), "
             "permuted; natural (plain CSR and tiled kernel) vs SB K=1024 cut from the grid "
             "(32 x 32 tiles)",
    "precision": "7-pt Dirichlet Laplacian 128^3, permuted; natural, random, DB K=1024 "
                 "SpMV in the chosen dtype; CG with FP64 iterative refinement to 1e-10 "
                 "with FP64 / FP32 / BF16 inner products",
}


def default_forms(workload):
    return (FORMS_SWEEP if workload == "sweep" else (
        ["natural", "random", "tiled", "db1024"] if workload == "precision"
        else ["natural", "tiled", "sbgrid1024"] if workload == "scale"
        else ["natural", "tiled", "batch_split16"] if workload == "batching"
        else ["natural", "tiled", "sb8", "split16"]))


def compulsory_bytes(m, n, nnz, vb=8, xb=8, r=1):
    return nnz * (vb + 4) + (m + 1) * 4 + n * xb * r + m * xb * r


def max_over_ranks(value, device):
    """The slowest rank's time: every rank runs the same replica of the step."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(world, step_bytes, ms_per_step):
    """GB/s of the whole job: every rank processed step_bytes per step."""
    return world * step_bytes / (ms_per_step * 1e-3) / 1e9


def make_matrices(workload, log=None, only=None):
    out = []
    for name, fn in MATRICES[workload]:
        if only and name not in only:
            continue
        t0 = time.perf_counter()
        rp, ci, v = fn()
        out.append((name, rp, ci, v))
        if log:
            log("generated %s: m=%d nnz=%d (%.1fs)" % (name, len(rp) - 1, int(rp[-1]),
                                                        time.perf_counter() - t0))
    return out


# ---------------------------------------------------------------- forms --
ICSR = "_icsr"


def base_form(f):
    """A form name without its storage suffix: "<form>_icsr" is <form> with
    the column indices of its unstaged chunks stored as 16-bit increments
    along each row (SPMV_FLAG_COL_DELTA; ICSR's colDiff, Sec. 2.1)."""
    return f[:-len(ICSR)] if f.endswith(ICSR) else f


def partition_jobs(S, rp, ci, forms, seed, threads, cache_dir=None, name=""):
    """Host partitions every requested form needs, run concurrently.  With
    cache_dir, results are kept there as .npz files keyed by matrix, model,
    K and seed, and reused (preprocessing is not part of the timed step)."""
    m = n = len(rp) - 1
    need = {}
    forms = [base_form(f) for f in forms]
    for f in forms:
        if f.startswith("sbgrid"):
            continue                    # cut from the mesh's grid, no bisection
        if f.startswith("sbnest") or f.startswith("dbnest"):
            # the SB / DB partition, its border in the nested order
            K = int(f[6:])
            need[("cn" if f[0] == "s" else "ercn", K)] = dict(
                method=S.SPMV_PART_CN if f[0] == "s" else S.SPMV_PART_ERCN, K=K)
            continue
        if f.startswith("sbfit"):
            # the paper's stop rule (Sec. 5.1) on the GPU's window: bisect
            # until each part's x subvector is below `kb` KB (SPMV_FIT_X)
            kb = int(f[5:])
            need[("cnfit", kb)] = dict(method=S.SPMV_PART_CN, K=0, part_bytes=kb * 1024,
                                       fit_rule=S.SPMV_FIT_X)
        elif f.startswith("sb"):
            need[("cn", int(f[2:]))] = dict(method=S.SPMV_PART_CN, K=int(f[2:]))
        elif f.startswith("db"):
            need[("ercn", int(f[2:]))] = dict(method=S.SPMV_PART_ERCN, K=int(f[2:]))
        elif f.startswith("split"):
            need[("rcn", 256)] = dict(method=S.SPMV_PART_RCN, K=256)
        elif f.startswith("rn"):
            need[("rn", int(f[2:]))] = dict(method=S.SPMV_PART_RN, K=int(f[2:]))
    res = {}
    # the breadth-first orders (sBFS, sRCM) take seconds: not cached
    for f in forms:
        if f in ("bfs", "rcm"):
            t0 = time.perf_counter()
            rperm, cperm = S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_BFS if f == "bfs"
                                          else S.SPMV_ORDER_RCM)
            res[(f, 0)] = dict(form=S.SPMV_NATURAL, K=1, row_perm=rperm, col_perm=cperm, cost=0,
                               cost_cols=0, cost_rows=0, seconds=time.perf_counter() - t0)

    def path(key):
        return os.path.join(cache_dir, "%s_%s_K%d_s%d.npz" % (name, key[0], key[1], seed))

    if cache_dir:
        for key in list(need):
            if os.path.exists(path(key)):
                res[key] = load_partition(S, path(key), m, n, rp, ci)
                del need[key]
    if not need:
        return res
    with cf.ThreadPoolExecutor(max_workers=len(need)) as ex:
        futs = {key: ex.submit(S.spmv_partition, m, n, rp, ci, seed=seed, threads=threads, **kw)
                for key, kw in need.items()}
        for key, fu in futs.items():
            res[key] = fu.result()
            if cache_dir:
                os.makedirs(cache_dir, exist_ok=True)
                save_partition(path(key), res[key])
    return res


def save_partition(path, r):
    """Keep a partition as its labels (the smallest integer type that holds
    them, compressed) and its scalars; the form is derived again on load."""
    lab = np.asarray(r["labels"])
    dt = np.uint8 if r["K"] < 256 else (np.uint16 if r["K"] < 65535 else np.int32)
    np.savez_compressed(path, labels=lab.astype(dt), form=r["form"], K=r["K"], cost=r["cost"],
                        cost_cols=r["cost_cols"], cost_rows=r["cost_rows"],
                        seconds=r["seconds"])


def load_partition(S, path, m, n, rp, ci):
    """A partition kept by save_partition, with its form rebuilt from the
    labels exactly as spmv_partition derives it (spmv_form_from_labels)."""
    with np.load(path) as z:
        r = {k: z[k].item() for k in z.files if k != "labels"}
        lab = np.ascontiguousarray(z["labels"], dtype=np.int32)
    if int(r["form"]) == S.SPMV_NATURAL:
        # a row-net partition: column labels, nested separated block-diagonal
        rperm, cperm = S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_SBD, int(r["K"]), lab)
        r.update(labels=lab, row_perm=rperm, col_perm=cperm)
        return r
    rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, int(r["form"]), int(r["K"]),
                                                     lab)
    r.update(labels=lab, row_perm=rperm, col_perm=cperm, row_part_ptr=rpp, col_part_ptr=cpp)
    return r


def batched_split_plan(S, name, K, dtype, threads, nrhs=1):
    """One plan over a batch of matrices, each split K ways by its own
    row-column-net bisection (Sec. 4.1)."""
    mats = BATCHES[name]
    known = BATCH_LABELS.get(name)
    if known and all(K in lab for lab in known):
        nz = [lab[K] for lab in known]
    else:
        def labels(mat):
            m, n, rp, ci, _ = mat
            return S.spmv_partition(m, n, rp, ci, S.SPMV_PART_RCN, K=K, seed=0,
                                    threads=1)["labels"]
        with cf.ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
            nz = list(ex.map(labels, mats))
    return S.spmv_plan_create_batched(mats, nz_parts=nz, K=K, dtype=dtype, nrhs=nrhs)


def form_kwargs(S, f, rp, ci, parts, seed=0, name=None):
    """spmv_plan_create arguments of a form, and the partition it came from."""
    if f.endswith(ICSR):
        b = base_form(f)
        if b in ("natural", "random") or b.startswith("batch"):
            raise ValueError("%s: the plain CSR kernel has no increment storage" % f)
        kw, pres = form_kwargs(S, b, rp, ci, parts, seed, name)
        kw["flags"] = kw.get("flags", 0) | S.SPMV_FLAG_COL_DELTA
        return kw, pres
    m = n = len(rp) - 1
    if f == "natural" or f.startswith("batch"):
        return {}, None
    if f == "tiled":
        return dict(flags=S.SPMV_FLAG_TILED_NATURAL), None
    if f in ("random", "rtiled"):
        p = synth.random_perm(m, 1000 + seed)
        kw = dict(row_perm=p, col_perm=p)
        if f == "rtiled":
            kw["flags"] = S.SPMV_FLAG_TILED_NATURAL
        return kw, None
    if f.startswith("sbgrid"):
        # SB form of a mesh from its grid: K square tiles of grid points (the
        # planted partition of the column-net model on a mesh)
        K = int(f[6:])
        t = int(round(np.sqrt(K)))
        nx, pts = MESH_POINTS[name]
        gx, gy = pts % nx, pts // nx
        lab = ((gy * t // nx) * t + gx * t // nx).astype(np.int32)
        rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SB, t * t, lab)
        return dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SB, K=t * t, row_part_ptr=rpp,
                    col_part_ptr=cpp), None
    if f in ("bfs", "rcm") or f.startswith("rn"):
        # the comparison orders of Sec. 5.1, natural form through the tiled
        # kernel
        r = parts[(f, 0) if f in ("bfs", "rcm") else ("rn", int(f[2:]))]
        return dict(row_perm=r["row_perm"], col_perm=r["col_perm"],
                    flags=S.SPMV_FLAG_TILED_NATURAL), r
    if f.startswith("sbnest") or f.startswith("dbnest"):
        # SB / DB with each bisection's cut columns between its halves
        # (SPMV_ORDER_NESTED), natural form through the tiled kernel
        r = parts[("cn" if f[0] == "s" else "ercn", int(f[6:]))]
        if "nested" not in r:
            r["nested"] = S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_NESTED, int(r["K"]),
                                         r["labels"])
        rperm, cperm = r["nested"]
        return dict(row_perm=rperm, col_perm=cperm, flags=S.SPMV_FLAG_TILED_NATURAL), r
    if f.startswith("sbfit"):
        r = parts[("cnfit", int(f[5:]))]
        return dict(row_perm=r["row_perm"], col_perm=r["col_perm"], form=r["form"], K=r["K"],
                    row_part_ptr=r["row_part_ptr"], col_part_ptr=r["col_part_ptr"]), r
    if f.startswith("sb") or f.startswith("db"):
        r = parts[("cn" if f.startswith("sb") else "ercn", int(f[2:]))]
        return dict(row_perm=r["row_perm"], col_perm=r["col_perm"], form=r["form"], K=r["K"],
                    row_part_ptr=r["row_part_ptr"], col_part_ptr=r["col_part_ptr"]), r
    if f.startswith("split"):
        # A^k = the nonzeros whose K=256 label lies in the k-th of K equal
        # label ranges (the K-way cut of the same recursion tree).  Rows and
        # columns are grouped by the first K=256 part touching them, so the
        # rows of each A^k keep the locality of the finer parts; the home
        # ranges of A^k are the unions of those of its finer parts.
        K = int(f[5:])
        full = parts[("rcn", 256)]
        if "fine_form" not in full:
            full["fine_form"] = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, 256,
                                                        full["labels"])
        rperm, cperm, rpp, cpp = full["fine_form"]
        step = 256 // K
        lab = (full["labels"] // step).astype(np.int32)
        sel = np.r_[np.arange(0, 257, step), 257]
        return dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SPLIT, K=K,
                    row_part_ptr=np.ascontiguousarray(rpp[sel]),
                    col_part_ptr=np.ascontiguousarray(cpp[sel]), nz_part=lab), full
    raise ValueError(f)


def tile_shapes(S, dtype, nrhs, nnz):
    """The launch shapes the autotuner chooses from for a tiled plan: one
    wave of 256-thread tiles (rows over 64, or over 128, nonzeros reduced by
    a warp), 512-thread tiles (two per SM, 48 KB shared-memory windows),
    wide 1024-thread tiles (one per SM, 96 KB windows), or eight waves of
    smaller tiles (launched in order, so that the x windows of the tiles
    running at once stay within L2 when x does not).  Staging in the
    256-thread tiles (SPMV_FLAG_STAGE) measured two to three times slower on
    the sweep and is left out."""
    return {"cta256": dict(dtype=dtype, nrhs=nrhs),
            "cta256w": dict(dtype=dtype, nrhs=nrhs, warp_rows=128),
            "cta512": dict(dtype=dtype, nrhs=nrhs, cta_threads=512),
            "cta1024": dict(dtype=dtype, nrhs=nrhs, cta_threads=1024),
            "cta256x8": dict(dtype=dtype, nrhs=nrhs, tile_nnz=max(1024, nnz // (8 * 912)))}


def err_ratio(y, y_ref, absax):
    """max_i |y - y_ref|_i / (|A||x|)_i (inf where |A||x| is 0 and y differs);
    NaN entries (unwritten output) fail."""
    y, y_ref, absax = (np.asarray(a, dtype=np.float64).reshape(-1) for a in (y, y_ref, absax))
    if np.any(np.isnan(y)):
        raise RuntimeError("unwritten output entries")
    err = np.abs(y - y_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(absax > 0, err / absax, np.where(err > 0, np.inf, 0.0))
    return float(ratio.max()) if ratio.size else 0.0


def library_reference(S, m, n, rp, ci, v, x64):
    """y = A x and |A||x| in FP64 from this library's natural-order CSR
    kernel on the original matrix: what the timed plans' outputs are held
    to (|y - y_ref|_i <= tol (|A||x|)_i).  The CPU oracle is test
    infrastructure and stays out of the timed arm; the independent parity
    of every form and shape at these sizes is checked by the GPU tests."""
    import torch
    r = 1 if x64.dim() == 1 else int(x64.shape[1])
    out = []
    for vals, xx in ((v, x64), (np.abs(v), x64.abs())):
        p = S.spmv_plan_create(m, n, rp, ci, vals, dtype=S.SPMV_F64, nrhs=r)
        y = torch.empty((m, r) if r > 1 else m, dtype=torch.float64, device=x64.device)
        S.spmv_exec(p, xx.contiguous(), y)
        if y.is_cuda:
            torch.cuda.synchronize()
        out.append(y.cpu().numpy())
        S.spmv_plan_destroy(p)
    return out[0], out[1]


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
                 "--format=csv,noheader,nounits", "-lms", "100"],
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


def kernel_name(info, dtype):
    """The kernel a plan's exec launches (the fix-up aside), as ncu names it."""
    vt, xt = {"f64": ("double", "double"), "f32": ("float", "float"),
              "bf16": ("__nv_bfloat16", "float")}[dtype]
    r = info["nrhs"]
    if info["n_tiles"] == 0:
        return "k_csr_vector<%d, %d, %s, %s>" % (info["lanes"], r, vt, xt)
    nt = info.get("cta_threads", 256) or 256
    return "k_tiles<%d, %s, %s, %d>" % (r, vt, xt, nt)


KERNEL_SOURCES = ("spmv_kernels.cuh", "spmv_kern_f64.cu", "spmv_kern_f32.cu", "spmv_kern_bf16.cu",
                  "spmv_device.h", "spmv_internal.h", "spmv_plan.cpp", "spmv_capi.cu")


def kernel_source_hash():
    """Hash of the sources of the SpMV kernels and of the plans they run
    (the layout of every tile), with comments and blank space removed, so
    that the record of an ncu capture survives edits to comments only."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1203_2739_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(f.encode())
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(label, kernel):
    """DRAM bytes per launch of `kernel` on plan `label` recorded from an ncu
    capture of the current kernel sources (profiles/ncu_traffic.json, keyed
    "label kernel"); None when absent or stale."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    e = d.get("entries", {}).get("%s %s" % (label, kernel))
    return None if e is None else e.get("dram_bytes_per_launch")


# ------------------------------------------------------------- reference --
def _plain_prepared(mats):
    """The matrices in the arrays the oracle's plain loop reads (no
    conversion inside a timed call) with x ~ U(-1, 1)."""
    return [(name, len(rp) - 1, np.ascontiguousarray(rp, dtype=np.int64),
             np.ascontiguousarray(ci, dtype=np.int32), np.ascontiguousarray(v, dtype=np.float64),
             synth.uniform_x(len(rp) - 1, 1)) for name, rp, ci, v in mats]


def plain_cpu_gbs(prepared, threads, budget_s, reps=5):
    """The oracle's plain FP64 CSR loop (Sec. 2.1) on the host, the paper's
    protocol (3 warm-up calls, then timed calls; Sec. 5.2) per matrix: `reps`
    repetitions of `calls` calls, the median repetition.  GB/s = compulsory
    bytes of one product of every matrix / the sum of the matrices' median
    times per call.  `calls` is sized so that the whole measurement takes
    about budget_s seconds."""
    import oracle
    t_call, b_tot = 0.0, 0
    per = []
    for name, m, rp, ci, v, x in prepared:
        y = np.empty(m, dtype=np.float64)
        t0 = time.perf_counter()
        for _ in range(3):
            oracle.spmv_plain(m, rp, ci, v, x, threads, out=y)
        est = (time.perf_counter() - t0) / 3
        calls = int(max(1, min(100, budget_s / (len(prepared) * reps * max(est, 1e-6)))))
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            for _ in range(calls):
                oracle.spmv_plain(m, rp, ci, v, x, threads, out=y)
            ts.append((time.perf_counter() - t0) / calls)
        t_call += float(np.median(ts))
        b_tot += compulsory_bytes(m, m, int(rp[-1]))
        per.append("%s %d x %d calls" % (name, reps, calls))
    return b_tot / t_call / 1e9, per


def cpu_threads():
    import oracle
    return max(1, min(os.cpu_count() or 1, oracle.plain_max_threads()))


def run_reference(args, rank, world):
    """The reference arm: the oracle's plain FP64 CSR loop (Sec. 2.1) on the
    host's cores (OpenMP), on the same (matrix, form) units as this library's
    step.  Every form computes the same product y = A x, which the oracle
    computes on the matrix in its original order; one step = one product per
    unit of the step."""
    if rank != 0:
        return
    import oracle
    mats = make_matrices(args.workload, None, args.matrices.split(",") if args.matrices else None)
    prepared = _plain_prepared(mats)
    forms = args.forms.split(",") if args.forms else default_forms(args.workload)
    threads = cpu_threads()
    units = [(p, f) for p in prepared for f in forms]
    for w in range(args.warmup):
        name, m, rp, ci, v, x = units[w % len(units)][0]
        oracle.spmv_plain(m, rp, ci, v, x, threads)
    ys = {p[0]: np.empty(p[1], dtype=np.float64) for p in prepared}
    step_bytes = sum(compulsory_bytes(p[1], p[1], int(p[2][-1])) for p, _ in units)
    step_flops = sum(2 * int(p[2][-1]) for p, _ in units)
    ts = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        for (name, m, rp, ci, v, x), _ in units:
            oracle.spmv_plain(m, rp, ci, v, x, threads, out=ys[name])
        ts.append(time.perf_counter() - t0)
    t = float(np.sum(ts))
    gbs = step_bytes * args.steps / t / 1e9
    sample = ("oracle's plain FP64 CSR loop, OpenMP over %d host threads (nproc %d): %d steps of "
              "%d products (one per (matrix, form) unit: %s x %s), each on the matrix in "
              "original order" % (threads, os.cpu_count() or 0, args.steps, len(units),
                                  "/".join(p[0] for p in prepared), ",".join(forms)))
    line = {
        "impl": "reference", "metric": "SpMV GB/s (compulsory bytes; % of GB300 HBM roofline)",
        "value": round(gbs, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * t / max(args.steps, 1), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload],
                   "matrices": [p[0] for p in prepared], "forms": forms,
                   "unit_of_work": "one y<-Ax per (matrix, form) per step; every form computes "
                                   "the same product, which the oracle computes in original "
                                   "order",
                   "nrhs": 1, "parallelism": "%d host threads" % threads},
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gflops": round(step_flops * args.steps / t / 1e9, 3),
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(mats, budget_s):
    """The oracle's plain FP64 CSR loop on the host (Sec. 2.1; the paper's
    protocol of warm-up calls and timed calls, median of 5 repetitions), on
    every matrix of the workload in its original order: single-threaded and
    with OpenMP over all host cores.  `value` is the all-cores figure."""
    prepared = _plain_prepared(mats)
    threads = cpu_threads()
    one, per1 = plain_cpu_gbs(prepared, 1, budget_s / 2)
    allc, per = plain_cpu_gbs(prepared, threads, budget_s / 2)
    return {"value": round(allc, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": "oracle's plain FP64 CSR loop (Sec. 2.1) on each matrix in original order, "
                      "3 warm-ups then 5 repetitions, median; OpenMP over %d threads: %s"
                      % (threads, "; ".join(per)),
            "single_thread": {"value": round(one, 3), "unit": "GB/s", "cores": 1,
                              "sample": "; ".join(per1)}}


# ------------------------------------------------------------------- ours --
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1203_2739_gb300 as S

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    log = (lambda s: print(s, file=sys.stderr, flush=True)) if rank == 0 else (lambda s: None)
    forms = args.forms.split(",") if args.forms else default_forms(args.workload)
    dtype = {"f64": S.SPMV_F64, "f32": S.SPMV_F32, "bf16": S.SPMV_BF16}[args.dtype]
    vb, xb = {0: (8, 8), 1: (4, 4), 2: (2, 4)}[dtype]
    tdt = torch.float64 if dtype == S.SPMV_F64 else torch.float32
    r = args.nrhs
    threads = max(1, (os.cpu_count() or 4) // 2)
    t_setup = time.perf_counter()
    mats = make_matrices(args.workload, log, args.matrices.split(",") if args.matrices else None)

    entries = []
    stream = torch.cuda.current_stream()
    # the host partitions of every matrix at once (their top bisections are
    # mostly serial, so the matrices overlap on the host's cores)
    need_forms = forms + (["db1024"] if args.workload == "precision" else [])
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=max(1, len(mats))) as ex:
        futs = [ex.submit(partition_jobs, S, rp, ci, need_forms, 0, threads,
                          args.partition_cache, name) for name, rp, ci, v in mats]
        all_parts = [f.result() for f in futs]
    log("  partitions of all matrices %.1fs" % (time.perf_counter() - t0))
    for (name, rp, ci, v), parts in zip(mats, all_parts):
        m = n = len(rp) - 1
        parts_kept = parts
        for key, pr in parts.items():
            log("  %s %s K=%d: partition %.1fs, cost %d (cols %d, rows %d)" % (
                name, key[0], pr["K"], pr["seconds"], pr["cost"], pr["cost_cols"],
                pr["cost_rows"]))
        # X is n x r row-major
        x = synth.uniform_x(n, 1) if r == 1 else synth.uniform_x(n * r, 1).reshape(n, r)
        x64 = torch.from_numpy(x).to(dev)
        y_ref, absax = library_reference(S, m, n, rp, ci, v, x64)
        xt = x64.to(dtype=tdt)
        for f in forms:
            kw, pres = form_kwargs(S, f, rp, ci, parts, name=name)
            t1 = time.perf_counter()
            chosen = None
            shapes = tile_shapes(S, dtype, r, int(rp[-1]))
            if f.startswith("batch_split"):
                plan = batched_split_plan(S, name, int(f[11:]), dtype, threads, nrhs=r)
            elif f in ("natural", "random") or args.no_autotune:
                plan = S.spmv_plan_create(m, n, rp, ci, v, dtype=dtype, nrhs=r, **kw)
            else:
                # the form's own flags (natural order through the tiled
                # kernel) join each shape's
                fl = kw.pop("flags", 0)
                shapes = {k: dict(c, flags=c.get("flags", 0) | fl) for k, c in shapes.items()}
                fixed = args.shape or SHAPE_MAP.get("%s/%s" % (name, f))
                if fixed:
                    plan = S.spmv_plan_create(m, n, rp, ci, v, **shapes[fixed], **kw)
                    chosen = fixed
                else:
                    names = list(shapes)
                    plan, ibest, _ = S.spmv_plan_autotune(m, n, rp, ci, v,
                                                          [shapes[k] for k in names], reps=9,
                                                          **kw)
                    chosen = names[ibest]
            xh = torch.empty_like(xt)
            S.spmv_permute_x(plan, xt, xh)
            yh = torch.empty((m, r) if r > 1 else m, dtype=tdt, device=dev)
            S.spmv_exec(plan, xh, yh)
            y = torch.empty_like(yh)
            S.spmv_unpermute_y(plan, yh, y)
            torch.cuda.synchronize()
            err = err_ratio(y.double().cpu().numpy(), y_ref, absax)
            info = plan.info
            entries.append(dict(label="%s/%s" % (name, f), plan=plan, xh=xh, yh=yh,
                                bytes=compulsory_bytes(m, n, int(rp[-1]), vb, xb, r),
                                flops=2 * int(rp[-1]) * r, err=err, info=info, tile_shape=chosen,
                                cost=None if pres is None else int(pres["cost"]),
                                part_s=None if pres is None else float(pres["seconds"])))
            log("  plan %s/%s: K=%d tiles=%d staged=%d shape=%s err=%.2e (%.1fs)" % (
                name, f, info["K"], info["n_tiles"], info["n_staged_tiles"], chosen, err,
                time.perf_counter() - t1))
        del y_ref, absax, x64
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
    time.sleep(0.25)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    if dist:
        elapsed_ms = max_over_ranks(elapsed_ms, dev)
    per = np.array([[a.elapsed_time(b) for (a, b) in row] for row in ev])   # steps x entries
    mean_ms = per.mean(axis=0)

    # end to end through the host-buffer entry point (copies in the timed region)
    e2e = None
    if not args.no_e2e:
        hx = [e["xh"].cpu().pin_memory() for e in entries]
        hy = [torch.empty(e["yh"].numel(), dtype=e["yh"].dtype).pin_memory() for e in entries]
        for i, e in enumerate(entries):
            S.spmv_exec_host(e["plan"], hx[i], hy[i])
        e2e_steps = max(1, min(args.steps, 20))
        ta = time.perf_counter()
        for _ in range(e2e_steps):
            for i, e in enumerate(entries):
                S.spmv_exec_host(e["plan"], hx[i], hy[i])
        tb = time.perf_counter()
        step_bytes = sum(e["bytes"] for e in entries)
        e2e = {"value": round(world * step_bytes * e2e_steps / (tb - ta) / 1e9, 2),
               "unit": "GB/s",
               "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hx)),
               "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hy))}

    step_bytes = sum(e["bytes"] for e in entries)
    step_flops = sum(e["flops"] for e in entries)
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_gbs(world, step_bytes, ms_per_step)
    if rank != 0:
        return
    peak, peak_kind = measured_peak()
    # the dominant kernel: the kernel instance with the largest share of the
    # step's device time (plans launching the same kernel grouped); its
    # achieved bandwidth is the algorithmic bytes of its launches over their
    # summed duration
    groups = {}
    for i, e in enumerate(entries):
        groups.setdefault(kernel_name(e["info"], args.dtype), []).append(i)
    dom_kernel = max(groups, key=lambda k: sum(mean_ms[i] for i in groups[k]))
    members = groups[dom_kernel]
    achieved = (sum(entries[i]["bytes"] for i in members)
                / (sum(mean_ms[i] for i in members) * 1e-3) / 1e9)
    share = sum(mean_ms[i] for i in members) / float(np.sum(mean_ms))
    # DRAM traffic per launch from an ncu capture of one of its plans (the
    # slowest one that has a record for the current kernel sources)
    by_time = sorted(members, key=lambda i: -mean_ms[i])
    d = next((entries[i] for i in by_time
              if ncu_traffic(entries[i]["label"], dom_kernel) is not None),
             entries[by_time[0]])
    detail = {}
    for i, e in enumerate(entries):
        gbs = e["bytes"] / (mean_ms[i] * 1e-3) / 1e9
        detail[e["label"]] = {
            "us": round(1e3 * mean_ms[i], 2), "GBps": round(gbs, 1),
            "GFLOPs": round(e["flops"] / (mean_ms[i] * 1e-3) / 1e9, 1),
            "frac": round(gbs / peak, 3), "err": e["err"], "K": e["info"]["K"],
            "tiles": e["info"]["n_tiles"], "staged_tiles": e["info"]["n_staged_tiles"],
            "launches": e["info"]["launches_per_exec"], "tile_shape": e["tile_shape"],
            "moved_over_compulsory": round(e["info"]["moved_bytes"] / e["bytes"], 3),
            "bound_cost": e["cost"]}
    speedup = reorder_gains(detail)
    # the paper's Table 3 analogue: partitioning time on the host, and the
    # number of products after which a form has paid for it against plain
    # CSR in natural order
    for e in entries:
        dd = detail[e["label"]]
        nat = detail.get(e["label"].split("/")[0] + "/natural")
        dd["partition_s"] = None if e["part_s"] is None else round(e["part_s"], 2)
        gain_us = None if nat is None else nat["us"] - dd["us"]
        dd["amortized_after_spmvs"] = (int(np.ceil(e["part_s"] * 1e6 / gain_us))
                                       if e["part_s"] is not None and gain_us and gain_us > 0
                                       else None)
    line = {
        "metric": "SpMV GB/s (compulsory bytes; % of GB300 HBM roofline)",
        "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload],
                   "matrices": [m[0] for m in mats], "forms": forms,
                   "unit_of_work": "one y<-Ax per (matrix, form) per step",
                   "nrhs": r,
                   "l2": "inputs larger than L2: each step streams %.2f GB over %d plans"
                         % (step_bytes / 1e9, len(entries)),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "gflops": round(world * step_flops / (ms_per_step * 1e-3) / 1e9, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "kernel": dom_kernel, "share_of_step": round(share, 3),
                     "plans": [entries[i]["label"] for i in members],
                     "traffic": ncu_traffic(d["label"], dom_kernel), "traffic_plan": d["label"]},
        "gpu_launches": int(args.steps * sum(e["info"]["launches_per_exec"] for e in entries)),
        "clocks": clk,
        "e2e": e2e,
        "max_err_ratio": max(e["err"] for e in entries),
        "err_basis": "max_i |y - y_ref|_i / (|A||x|)_i with y_ref and |A||x| from this "
                     "library's FP64 natural-order CSR product on the GPU; the CPU oracle "
                     "holds the same plans in the GPU tests",
        "speedup_vs_natural": speedup,
        "detail": detail,
        "setup_s": round(setup_s, 1),
    }
    if args.workload == "precision":
        line["cg_ir"] = precision_solves(S, mats[0], parts_kept, dev, log)
    if args.workload == "batching":
        # 100 repeated products of the fastest batched plan (tiled natural
        # or split) replayed from one CUDA graph
        cands = [i for i, e in enumerate(entries) if not e["label"].endswith("/natural")]
        if cands:
            line["graph"] = graph_replay(S, entries[min(cands, key=lambda i: mean_ms[i])],
                                         stream)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(mats, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)


def reorder_gains(detail):
    """Per matrix: the fastest form; its speedup over plain CSR in natural
    order and over the faster of the two natural-order kernels (plain CSR,
    tiled); and, the paper's comparison (Table 2: each method's time against
    the original order), each reordered or split form's gain over the same
    tiled kernel in natural order (and random order's, for contrast)."""
    out = {}
    mats = []
    for label in detail:
        mat = label.split("/")[0]
        if mat not in mats:
            mats.append(mat)
    for mat in mats:
        us = {label.split("/")[1]: dd["us"] for label, dd in detail.items()
              if label.split("/")[0] == mat}
        best_form = min(us, key=us.get)
        nat = [us[f] for f in ("natural", "tiled") if f in us]
        e = {"best_form": best_form,
             "speedup_vs_natural": round(us["natural"] / us[best_form], 3)
             if "natural" in us else None,
             "speedup_vs_best_natural_kernel": round(min(nat) / us[best_form], 3)
             if nat else None}
        if "tiled" in us:
            e["gain_over_tiled_natural"] = {
                f: round(us["tiled"] / t, 3) for f, t in us.items()
                if f not in ("natural", "random", "tiled")}
            # the paper's Table 2: each method's time over the original
            # order's, with the same kernel (lower is better)
            e["normalized_time"] = {f: round(t / us["tiled"], 3) for f, t in us.items()
                                    if f not in ("natural", "random", "tiled")}
        # 16-bit column increments against 32-bit indices, same form
        inc = {f: round(us[f] / us[f + ICSR], 3) for f in us if f + ICSR in us}
        if inc:
            e["icsr_gain"] = inc
        out[mat] = e
    norm = [e["normalized_time"] for e in out.values() if "normalized_time" in e]
    if norm:
        forms = [f for f in norm[0] if all(f in d for d in norm)]
        out["geomean_normalized_time"] = {
            f: round(float(np.exp(np.mean([np.log(d[f]) for d in norm]))), 3) for f in forms}
    return out


def graph_replay(S, e, stream, iters=100, reps=5):
    """100 repeated products of one plan captured in a CUDA graph; the time
    per product of a replay (median of reps replays)."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        S.spmv_exec(e["plan"], e["xh"], e["yh"])
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(iters):
            S.spmv_exec(e["plan"], e["xh"], e["yh"])
    ts = []
    with torch.cuda.stream(s):          # replay() launches on the current stream
        g.replay()
        torch.cuda.synchronize()
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            g.replay()
            b.record(s)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
    us = 1e3 * float(np.median(ts)) / iters
    return {"plan": e["label"], "iterations": iters, "us_per_product": round(us, 2),
            "GBps": round(e["bytes"] / (us * 1e-6) / 1e9, 1),
            "launches_per_product": e["info"]["launches_per_exec"]}


def precision_solves(S, mat, parts, dev, log):
    """The precision extension: A x = b on the matrix in its DB form (eRCN,
    K=1024) by CG with FP64 iterative refinement, inner products in FP64,
    FP32 and BF16 values; b = A x* for a seeded x*.  Reports time to a
    relative FP64 residual of 1e-10 and the error against x*."""
    import torch
    name, rp, ci, v = mat
    n = len(rp) - 1
    kw, _ = form_kwargs(S, "db1024", rp, ci, parts)
    x_star = synth.uniform_x(n, 7)
    b, _ = library_reference(S, n, n, rp, ci, v, torch.from_numpy(x_star).to(dev))
    bd = torch.from_numpy(b).to(dev)
    f64 = S.spmv_plan_create(n, n, rp, ci, v, dtype=S.SPMV_F64, **kw)
    out = {}
    for label, dt in (("f64", S.SPMV_F64), ("f32", S.SPMV_F32), ("bf16", S.SPMV_BF16)):
        low = f64 if dt == S.SPMV_F64 else S.spmv_plan_create(n, n, rp, ci, v, dtype=dt, **kw)
        xd = torch.zeros(n, dtype=torch.float64, device=dev)
        S.spmv_cg_ir(low, f64, bd, xd, tol=1e-10)          # warm
        xd.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = S.spmv_cg_ir(low, f64, bd, xd, tol=1e-10)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        x = xd.cpu().numpy()
        ax, _ = library_reference(S, n, n, rp, ci, v, xd)
        out[label] = {"seconds": round(secs, 4), "outer": info["outer"],
                      "inner_iterations": info["inner_total"],
                      "rel_residual_solver": info["rel_residual"],
                      "rel_residual_fp64": float(np.linalg.norm(b - ax) / np.linalg.norm(b)),
                      "rel_error_vs_x_star": float(np.linalg.norm(x - x_star)
                                                   / np.linalg.norm(x_star)),
                      "converged": info["converged"]}
        log("  CG-IR %s: %s" % (label, out[label]))
    return out


# ------------------------------------------------------------- selector --
def selector_matrix(i):
    """Seeded matrix i of the selector's data: mesh, R-MAT, blocks or Zipf
    families with 10^4 .. 3 x 10^5 rows (log-uniform), taking turns."""
    g = np.random.default_rng(1000 + i)
    fam = i % 4
    rows = int(np.exp(g.uniform(np.log(1e4), np.log(3e5))))
    if fam == 0:
        rp, ci, v = synth.mesh5(max(100, int(np.sqrt(rows))), seed=i)
    elif fam == 1:
        rp, ci, v = synth.rmat(int(np.clip(np.round(np.log2(rows)), 13, 18)),
                               int(g.integers(4, 17)), seed=i, chunk=1 << 18)
    elif fam == 2:
        nb = int(g.choice([8, 16, 32, 64]))
        bs = max(256, rows // nb)
        rp, ci, v = synth.blocks(nb, bs, float(g.uniform(8, 24)) / bs, 0.05, seed=i)
    else:
        rp, ci, v = synth.zipf_matrix(rows, rows, seed=i)
    return rp, ci, v


def _selector_partitions(spec):
    """Worker (spawned process, no GPU): the matrix and the partitions its
    classes need (kept in / read from `cache` when given)."""
    i, cache = spec
    import paper_1203_2739_gb300 as S
    rp, ci, v = selector_matrix(i)
    m = n = len(rp) - 1
    out = {}
    for meth, K in ((S.SPMV_PART_CN, 16), (S.SPMV_PART_CN, 256), (S.SPMV_PART_ERCN, 16),
                    (S.SPMV_PART_ERCN, 256), (S.SPMV_PART_RCN, 256)):
        path = os.path.join(cache, "sel%d_m%d_K%d.npz" % (i, meth, K)) if cache else None
        if path and os.path.exists(path):
            out[(meth, K)] = load_partition(S, path, m, n, rp, ci)
            continue
        out[(meth, K)] = S.spmv_partition(m, n, rp, ci, meth, K=K, seed=0, threads=1)
        if path:
            os.makedirs(cache, exist_ok=True)
            save_partition(path, out[(meth, K)])
    return i, out


def run_selector(args, pool_results):
    """Train the selector on autotuner timings of the first 3/4 of the
    matrices and evaluate it on the rest: regret against the exhaustive
    optimum, and throughput against plain CSR."""
    import torch
    import paper_1203_2739_gb300 as S
    import paper_1203_2739_gb300.selector as SEL
    log = lambda s: print(s, file=sys.stderr, flush=True)   # noqa: E731
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    N = len(pool_results)
    feats, times, nbytes = [], [], []
    t_setup = time.perf_counter()
    for i in range(N):
        rp, ci, v = selector_matrix(i)
        m = n = len(rp) - 1
        parts = pool_results[i]
        feats.append(S.spmv_features(m, n, rp, ci))
        x = torch.from_numpy(synth.uniform_x(n, 1)).to(dev)
        y = torch.empty(m, dtype=torch.float64, device=dev)

        def build(cls):
            fw, K, ct = cls
            if fw == "natural":
                kw = {}
            elif fw == "tiled":
                kw = dict(flags=S.SPMV_FLAG_TILED_NATURAL, warp_rows=128)
            elif fw in ("sb", "db"):
                r = parts[(S.SPMV_PART_CN if fw == "sb" else S.SPMV_PART_ERCN, K)]
                kw = dict(row_perm=r["row_perm"], col_perm=r["col_perm"], form=r["form"],
                          K=r["K"], row_part_ptr=r["row_part_ptr"],
                          col_part_ptr=r["col_part_ptr"], cta_threads=ct)
            else:
                full = parts[(S.SPMV_PART_RCN, 256)]
                lab = (full["labels"] // (256 // K)).astype(np.int32)
                rperm, cperm, rpp, cpp = S.spmv_form_from_labels(m, n, rp, ci, S.SPMV_SPLIT, K,
                                                                 lab)
                kw = dict(row_perm=rperm, col_perm=cperm, form=S.SPMV_SPLIT, K=K,
                          row_part_ptr=rpp, col_part_ptr=cpp, nz_part=lab, cta_threads=ct)
            return S.spmv_plan_create(m, n, rp, ci, v, **kw)

        # every class's plan built at once on host threads, then timed in
        # turns (each call after another class's) with the median kept
        with cf.ThreadPoolExecutor(max_workers=len(SEL.CLASSES)) as ex:
            plans = list(ex.map(build, SEL.CLASSES))
        reps = 15
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in plans] for _ in range(reps)]
        for plan in plans:
            S.spmv_exec(plan, x, y)
        for r_ in range(reps):
            for k, plan in enumerate(plans):
                ev[r_][k][0].record(stream)
                S.spmv_exec(plan, x, y)
                ev[r_][k][1].record(stream)
        torch.cuda.synchronize()
        times.append([float(np.median([ev[r_][k][0].elapsed_time(ev[r_][k][1])
                                       for r_ in range(reps)])) for k in range(len(plans))])
        del plans
        nbytes.append(compulsory_bytes(m, n, int(rp[-1])))
        if i % 16 == 15:
            log("  selector data: %d/%d matrices timed" % (i + 1, N))
    setup_s = time.perf_counter() - t_setup
    F, T = np.array(feats), np.array(times)
    best = T.argmin(axis=1)
    ntr = (3 * N) // 4
    sel = SEL.Selector(seed=0)
    t0 = time.perf_counter()
    hist = sel.fit(F[:ntr], best[:ntr], epochs=400, lr=3e-3, batch=32)
    train_s = time.perf_counter() - t0
    test = np.arange(ntr, N)
    pick, conf = sel.predict(F[test])
    regret = T[test, pick] / T[test, best[test]] - 1.0
    # fallback: below the confidence threshold, time every class (regret 0)
    thr = 0.5
    regret_fb = np.where(conf >= thr, regret, 0.0)
    t_pick = T[test, pick].sum()
    t_plain = T[test, 0].sum()
    t_best = T[test, best[test]].sum()
    bytes_test = float(np.sum(np.array(nbytes)[test]))
    line = {
        "metric": "SpMV GB/s (compulsory bytes) of the selector's choice on held-out matrices",
        "value": round(bytes_test / (t_pick * 1e-3) / 1e9, 2), "unit": "GB/s", "n_gpus": 1,
        "steps": 20, "warmup": 3, "ms_per_step": round(float(t_pick), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "learned selector: %d seeded matrices (mesh / R-MAT / blocks / "
                               "Zipf, 1e4-3e5 rows), %d classes (plain CSR; natural order through "
                               "the tiled kernel; SB, DB, split at K = 16, 256; 256- or "
                               "1024-thread tiles); trained on %d, "
                               "evaluated on %d" % (N, len(SEL.CLASSES), ntr, N - ntr),
                   "l2": "matrices smaller than L2: repeated products with L2 warm"},
        "selector": {
            "regret_mean": round(float(regret.mean()), 4),
            "regret_median": round(float(np.median(regret)), 4),
            "within_10pct": round(float((regret <= 0.10).mean()), 3),
            "regret_mean_with_fallback": round(float(regret_fb.mean()), 4),
            "fallback_share": round(float((conf < thr).mean()), 3),
            "top1_accuracy": round(float((pick == best[test]).mean()), 3),
            "speedup_vs_plain_csr": round(float(t_plain / t_pick), 3),
            "speedup_vs_plain_csr_exhaustive_choice": round(float(t_plain / t_best), 3),
            "speedup_vs_best_fixed_class": round(float(
                T[test].sum(axis=0).min() / t_pick), 3),
            "train_loss_first_last": [round(hist[0], 4), round(hist[-1], 4)],
            "train_seconds_gpu_kernels": round(train_s, 2),
            "data_seconds": round(setup_s, 1)},
        "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep", choices=sorted(MATRICES) + ["selector"])
    ap.add_argument("--selector-matrices", type=int, default=200)
    ap.add_argument("--scale-nx", type=int, default=6144,
                    help="grid side of the scale workload's mesh (x exceeds L2 from about 4096)")
    ap.add_argument("--forms", default="")
    ap.add_argument("--matrices", default="", help="subset of the workload's matrices (by name)")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="tiled forms with the default tile shape instead of the autotuned one")
    ap.add_argument("--shape", default="", choices=["", "cta256", "cta256w", "cta512", "cta1024",
                                                    "cta256x8"],
                    help="tiled forms with this tile shape instead of the autotuned one")
    ap.add_argument("--shape-map", default=None,
                    help="JSON file: a bench line (its detail's tile_shape per plan) or a "
                         "{matrix/form: shape} object; those plans skip the autotuner")
    ap.add_argument("--partition-cache", default=None,
                    help="directory to keep and reuse host partitions (untimed preprocessing)")
    ap.add_argument("--nrhs", type=int, default=1, choices=[1, 2, 4, 8],
                    help="right-hand sides per product (Y = A X, X row-major n x nrhs)")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="matrices in the batching workload")
    ap.add_argument("--batch-max-rows", type=int, default=262144,
                    help="largest member of the batching workload (rows, log-uniform from 1024)")
    args = ap.parse_args()
    if args.shape_map:
        SHAPE_MAP.update(load_shape_map(args.shape_map))
    if args.workload == "batching":
        name = "rmat_batch%d" % args.batch_count
        BATCH.update(count=args.batch_count, max_rows=args.batch_max_rows,
                     cache=args.partition_cache,
                     K=() if args.impl == "reference" else tuple(
                         int(f[11:]) for f in (args.forms or "batch_split16").split(",")
                         if f.startswith("batch_split")))
        MATRICES["batching"] = [(name, lambda: _batch_matrix(name))]
        WORKLOAD_TEXT["batching"] = WORKLOAD_TEXT["batching"].replace(
            "256 R-MAT", "%d R-MAT" % args.batch_count).replace(
            "262144]", "%d]" % args.batch_max_rows)
    if args.scale_nx != 6144:
        nx = args.scale_nx
        MATRICES["scale"] = [("mesh5_%d" % nx, lambda: _mesh_with_points("mesh5_%d" % nx, nx))]
        WORKLOAD_TEXT["scale"] = WORKLOAD_TEXT["scale"].replace(
            "mesh 6144^2 (37.7M rows, 188.7M nnz, x = 302 MB)", "mesh %d^2" % nx)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "selector" and args.impl == "reference":
        print(json.dumps({"impl": "reference",
                          "unavailable": "the selector workload measures choices among this "
                                         "library's own plans; it has no CPU reference arm"}))
        return
    if args.workload == "selector":
        # partitions on host processes started before any GPU work
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(max(1, (os.cpu_count() or 4))) as pool:
            res = dict(pool.map(_selector_partitions,
                                [(i, args.partition_cache) for i in range(args.selector_matrices)],
                                chunksize=1))
        run_selector(args, [res[i] for i in range(args.selector_matrices)])
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.warmup < 3:
        print("note: warmup raised to 3", file=sys.stderr)
        args.warmup = 3
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
