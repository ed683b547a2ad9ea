"""Host logic of bench.py: the compulsory-bytes unit, kernel naming for the
dominant-kernel roofline, the partition cache round trip and the split
forms cut from one recursion tree."""
import json
import os

import numpy as np
import pytest

import bench
import synth

S = pytest.importorskip("paper_1203_2739_gb300")


def test_compulsory_bytes_unit():
    # nnz*(vb+4) + (m+1)*4 + n*r*xb + m*r*xb
    assert bench.compulsory_bytes(10, 20, 100) == 100 * 12 + 11 * 4 + 20 * 8 + 10 * 8
    assert bench.compulsory_bytes(10, 20, 100, vb=2, xb=4, r=8) == \
        100 * 6 + 11 * 4 + 20 * 4 * 8 + 10 * 4 * 8


def test_kernel_names_follow_the_plan():
    info = dict(n_tiles=0, lanes=4, nrhs=1, cta_threads=0)
    assert bench.kernel_name(info, "f64") == "k_csr_vector<4, 1, double, double>"
    info = dict(n_tiles=10, lanes=32, nrhs=8, cta_threads=1024)
    assert bench.kernel_name(info, "bf16") == "k_tiles<8, __nv_bfloat16, float, 1024>"
    info["cta_threads"] = 256
    assert bench.kernel_name(info, "f32") == "k_tiles<8, float, float, 256>"
    info["cta_threads"] = 512
    assert bench.kernel_name(info, "f64") == "k_tiles<8, double, double, 512>"


def test_partition_cache_round_trip(tmp_path):
    m = n = 3000
    rp, ci, _ = synth.zipf_matrix(m, n, seed=5)
    a = bench.partition_jobs(S, rp, ci, ["sb8", "split16"], 0, 2, cache_dir=str(tmp_path),
                             name="z")
    files = sorted(os.listdir(tmp_path))
    assert files == ["z_cn_K8_s0.npz", "z_rcn_K256_s0.npz"]
    b = bench.partition_jobs(S, rp, ci, ["sb8", "split16"], 0, 2, cache_dir=str(tmp_path),
                             name="z")
    for key in a:
        for k, v in a[key].items():
            assert np.array_equal(np.asarray(v), np.asarray(b[key][k])), (key, k)


def test_split_forms_are_cuts_of_one_tree():
    m = n = 2000
    rp, ci, _ = synth.zipf_matrix(m, n, seed=6)
    parts = bench.partition_jobs(S, rp, ci, ["split4"], 0, 2)
    full = parts[("rcn", 256)]["labels"]
    for K in (4, 16, 64, 256):
        kw, _ = bench.form_kwargs(S, "split%d" % K, rp, ci, parts)
        assert kw["K"] == K
        assert np.array_equal(kw["nz_part"], full // (256 // K))
        # home ranges are those of the K=256 leaves, taken every 256/K
        assert kw["row_part_ptr"].size == K + 2 and kw["col_part_ptr"].size == K + 2
        assert kw["row_part_ptr"][-1] == m and kw["col_part_ptr"][-1] == n
        assert np.all(np.diff(kw["col_part_ptr"]) >= 0)


def test_batch_members_match_the_serial_generator_and_are_split(tmp_path):
    """The batching workload's members, generated and partitioned on spawned
    processes, are the matrices of synth.rmat_batch, each with a valid
    K = 16 row-column-net split; the partition cache returns the same
    labels."""
    saved = dict(bench.BATCH)
    try:
        bench.BATCH.update(count=6, max_rows=8192, K=(16,), cache=str(tmp_path))
        rp, ci, v = bench._batch_matrix("t")
        ref = synth.rmat_batch(6, lo=1024, hi=8192, seed=0)
        got = bench.BATCHES["t"]
        assert [g[0] for g in got] == [r[0] for r in ref]
        for g, r in zip(got, ref):
            for a, b in zip(g[2:], r[2:]):
                assert np.array_equal(a, b)
        brp, bci, bv = synth.block_diagonal(ref)
        assert np.array_equal(rp, brp) and np.array_equal(ci, bci) and np.array_equal(v, bv)
        labs = bench.BATCH_LABELS["t"]
        for (m, n, mrp, mci, _), lab in zip(got, labs):
            assert lab[16].shape == (int(mrp[-1]),)
            assert lab[16].min() >= 0 and lab[16].max() < 16
        assert len(os.listdir(tmp_path)) == 6
        bench._batch_matrix("t2")
        for a, b in zip(labs, bench.BATCH_LABELS["t2"]):
            assert np.array_equal(a[16], b[16])
    finally:
        bench.BATCH.clear()
        bench.BATCH.update(saved)


def test_tile_shapes_are_the_autotuner_candidates():
    sh = bench.tile_shapes(S, S.SPMV_F32, 8, 36_000_000)
    assert list(sh) == ["cta256", "cta256w", "cta512", "cta1024", "cta256x8"]
    assert all(c["dtype"] == S.SPMV_F32 and c["nrhs"] == 8 for c in sh.values())
    assert sh["cta256w"]["warp_rows"] == 128 and sh["cta1024"]["cta_threads"] == 1024
    assert sh["cta512"]["cta_threads"] == 512
    # eight waves of 152 SMs x 6 resident CTAs
    assert sh["cta256x8"]["tile_nnz"] == 36_000_000 // (8 * 912)
    assert bench.tile_shapes(S, 0, 1, 1000)["cta256x8"]["tile_nnz"] == 1024


class _FakeSmi:
    """Stands in for the nvidia-smi sampling process: canned CSV rows in
    the order of ClockSampler.FIELDS."""

    def __init__(self, text):
        self.text = text
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_sampler_reports_median_max_and_throttle_reasons():
    rows = [
        "1980, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    cs = bench.ClockSampler(0)
    cs.proc = _FakeSmi("\n".join(rows) + "\n")
    out = cs.stop()
    assert cs.proc.terminated
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    cs.proc = _FakeSmi("2070, 2070, 1.0, 0x8, Active, Not Active, Active, Not Active\n")
    assert cs.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    cs.proc = _FakeSmi("")
    assert cs.stop() is None
    assert bench.ClockSampler(0).stop() is None      # never started


def test_whole_job_throughput_counts_every_rank():
    # 2 ranks, 1 GB each per 1 ms step: 2000 GB/s for the job
    assert bench.whole_job_gbs(2, 1e9, 1.0) == pytest.approx(2000.0)
    assert bench.whole_job_gbs(1, 5e8, 0.5) == pytest.approx(1000.0)


def _copy_sources(tmp_path):
    import shutil
    src = os.path.join(bench.ROOT, "paper_1203_2739_gb300", "csrc")
    dst = tmp_path / "paper_1203_2739_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The DRAM traffic of an ncu capture is used only while the kernel and
    plan sources are those it was taken from; edits to comments alone keep
    it."""
    import json
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (tmp_path / "profiles").mkdir()
    rec = {"kernel_source_hash": h0,
           "entries": {"m/f k<1>": {"dram_bytes_per_launch": 123}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("m/f", "k<1>") == 123
    assert bench.ncu_traffic("m/g", "k<1>") is None
    k = dst / "spmv_kernels.cuh"
    k.write_text(k.read_text() + "\n// a comment only\n/* and a block\n comment */\n")
    assert bench.kernel_source_hash() == h0
    assert bench.ncu_traffic("m/f", "k<1>") == 123
    k.write_text(k.read_text() + "\nstatic int changed_code = 1;\n")
    assert bench.kernel_source_hash() != h0
    assert bench.ncu_traffic("m/f", "k<1>") is None


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    import json
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6697.2}))
    assert bench.measured_peak() == (6697.2, "measured")


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the CPU oracle (no GPU needed) and
    prints the contract's JSON line."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl",
                          "reference", "--workload", "zipf16k", "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 1
    assert d["metric"].startswith("SpMV GB/s") and d["unit"] == "GB/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD_TEXT["zipf16k"]
    assert d["config"]["matrices"] == ["zipf16k"]
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == bench.cpu_threads()
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["config"]["forms"] == bench.default_forms("zipf16k")
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    sel = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl",
                          "reference", "--workload", "selector"],
                         capture_output=True, text=True, timeout=300, check=True).stdout
    assert "unavailable" in json.loads(sel.strip().splitlines()[-1])


class _HostS:
    """A stand-in for the library on host tensors (natural form only), to
    run bench.library_reference without a GPU."""
    SPMV_F64 = 0

    def __init__(self):
        self.live = 0

    def spmv_plan_create(self, m, n, rp, ci, vals, dtype=0, nrhs=1):
        import scipy.sparse as sp
        self.live += 1
        return (sp.csr_matrix((np.asarray(vals, dtype=np.float64), ci, rp), shape=(m, n)), nrhs)

    def spmv_exec(self, plan, x, y):
        import torch
        A, r = plan
        assert x.is_contiguous() and x.numel() == A.shape[1] * r
        y.copy_(torch.from_numpy(np.asarray(A @ x.numpy()).reshape(y.shape)))

    def spmv_plan_destroy(self, plan):
        self.live -= 1


@pytest.mark.parametrize("nrhs", [1, 4])
def test_library_reference_is_y_and_abs_product(nrhs):
    import torch
    import oracle
    m, n = 300, 280
    rp, ci, v = synth.random_sparse(m, n, 0.05, 3, integer=False)
    x = synth.uniform_x(n * nrhs, 2).reshape(n, nrhs) if nrhs > 1 else synth.uniform_x(n, 2)
    fake = _HostS()
    y, absax = bench.library_reference(fake, m, n, rp, ci, v, torch.from_numpy(x))
    assert fake.live == 0
    for c in range(nrhs):
        xc = x if nrhs == 1 else np.ascontiguousarray(x[:, c])
        want, want_abs = oracle.spmv(m, n, rp, ci, v, xc)
        got = y if nrhs == 1 else y[:, c]
        got_abs = absax if nrhs == 1 else absax[:, c]
        assert np.allclose(got, want, rtol=1e-13, atol=1e-13)
        assert np.allclose(got_abs, want_abs, rtol=1e-13, atol=1e-13)


def test_cpu_baseline_is_plain_loop_single_and_all_cores():
    """The CPU baseline times the oracle's plain CSR loop on one thread and on
    every host core, median of 5 repetitions, and says how many it used."""
    mats = [("z", *synth.zipf_matrix(2048, 2048, seed=0))]
    d = bench.cpu_baseline_sample(mats, budget_s=0.5)
    assert d["kind"] == "oracle" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["cores"] == bench.cpu_threads() and d["nproc"] == os.cpu_count()
    assert d["single_thread"]["cores"] == 1 and d["single_thread"]["value"] > 0
    assert "5 x" in d["sample"] and "plain" in d["sample"]


def test_reorder_gains_use_the_same_kernel_in_natural_order():
    detail = {"a/natural": {"us": 10.0}, "a/tiled": {"us": 8.0}, "a/random": {"us": 20.0},
              "a/rtiled": {"us": 16.0}, "a/sb1024": {"us": 4.0}, "a/split4": {"us": 5.0}}
    g = bench.reorder_gains(detail)["a"]
    assert g["best_form"] == "sb1024"
    assert g["speedup_vs_natural"] == 2.5
    assert g["speedup_vs_best_natural_kernel"] == 2.0
    assert g["gain_over_tiled_natural"] == {"rtiled": 0.5, "sb1024": 2.0, "split4": 1.6}


def test_err_ratio_flags_unwritten_entries():
    assert bench.err_ratio([1.0, 2.0], [1.0, 2.5], [1.0, 1.0]) == 0.5
    with pytest.raises(RuntimeError):
        bench.err_ratio([float("nan")], [0.0], [1.0])


def test_shape_map_from_object_or_bench_line(tmp_path):
    obj = tmp_path / "m.json"
    obj.write_text('{\n "a/sb1024": "cta256w",\n "b/tiled": "cta512"\n}\n')
    assert bench.load_shape_map(str(obj)) == {"a/sb1024": "cta256w", "b/tiled": "cta512"}
    line = tmp_path / "b.json"
    line.write_text("log line\n" + json.dumps({"detail": {
        "a/sb1024": {"tile_shape": "cta1024"}, "a/natural": {"tile_shape": None}}}) + "\n")
    assert bench.load_shape_map(str(line)) == {"a/sb1024": "cta1024"}


def test_increment_and_nested_forms():
    """"<form>_icsr" is <form> with SPMV_FLAG_COL_DELTA; "sbnest<K>" and
    "dbnest<K>" reuse the CN / eRCN partition of "sb<K>" / "db<K>" with the
    nested border order through the tiled kernel."""
    m = n = 2500
    rp, ci, _ = synth.mesh5(50, seed=2)
    parts = bench.partition_jobs(S, rp, ci, ["sb8_icsr", "dbnest8", "split4_icsr"], 0, 2)
    assert set(parts) == {("cn", 8), ("ercn", 8), ("rcn", 256)}
    kw, _ = bench.form_kwargs(S, "sb8_icsr", rp, ci, parts)
    kw0, _ = bench.form_kwargs(S, "sb8", rp, ci, parts)
    assert kw["flags"] == S.SPMV_FLAG_COL_DELTA and kw0.get("flags", 0) == 0
    assert np.array_equal(kw["col_perm"], kw0["col_perm"])
    kw, _ = bench.form_kwargs(S, "split16_icsr", rp, ci, parts)
    assert kw["flags"] == S.SPMV_FLAG_COL_DELTA and kw["K"] == 16
    for f, key in (("sbnest8", ("cn", 8)), ("dbnest8_icsr", ("ercn", 8))):
        if key not in parts:
            parts.update(bench.partition_jobs(S, rp, ci, [f], 0, 2))
        kw, r = bench.form_kwargs(S, f, rp, ci, parts)
        want = S.spmv_reorder(m, n, rp, ci, S.SPMV_ORDER_NESTED, 8, r["labels"])
        assert np.array_equal(kw["row_perm"], want[0]) and np.array_equal(kw["col_perm"], want[1])
        assert kw["flags"] & S.SPMV_FLAG_TILED_NATURAL
        assert bool(kw["flags"] & S.SPMV_FLAG_COL_DELTA) == f.endswith("_icsr")
    with pytest.raises(ValueError):
        bench.form_kwargs(S, "natural_icsr", rp, ci, parts)
    g = bench.reorder_gains({"a/tiled": {"us": 8.0}, "a/sb8": {"us": 4.0},
                             "a/sb8_icsr": {"us": 3.2}})["a"]
    assert g["icsr_gain"] == {"sb8": 1.25}
