"""Host logic of bench.py: the compulsory-bytes unit, kernel naming for the
dominant-kernel roofline, the partition cache round trip and the split
forms cut from one recursion tree."""
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
