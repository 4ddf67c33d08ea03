"""Host-side arithmetic of bench.py, on the CPU: the algorithmic amount each
kernel's roofline counts, the achieved rate and fraction computed from it, and
the rule that a committed ncu traffic figure goes stale once its kernel's
source file changes."""
import hashlib
import json

import bench

DENSE = bench.WORKLOADS["dense"]
M, N, K = DENSE["m"], DENSE["n"], DENSE["k"]
PEAKS = dict(hbm_gbs=6780.7, bf16_tflops=1898.9, bf16_tflops_sustained=1698.5, source="measured",
             fp32_tflops=69.9, tf32_tflops=1027.5, fp64_tflops=1.10)


def test_residual_reads_A_once():
    bound, amount, unit, launches = bench.algorithmic("tc_residual_kernel", DENSE, K, 5, 2, [9, 9])
    assert (bound, unit, launches) == ("hbm", "GB/s", 1)
    assert amount == M * N * 4  # one FP32 read of A per exact error


def test_column_gather_counts_a_sector_per_element():
    # each of the m k scattered elements costs one 32-byte DRAM sector, plus its
    # write; pilot and follow-up gathers are two launches
    bound, amount, _, launches = bench.algorithmic("gather_cols_kernel", DENSE, K, 5, 4, [9, 9])
    assert bound == "hbm" and launches == 2
    assert amount == 2 * M * K * (32 + 4)


def test_kmeans_contraction_flops():
    # 2 (m + n) k k2 flops per iteration over both sides (Section 3.2), width padded to the 64-wide K chunk
    bound, amount, unit, launches = bench.algorithmic("tc_assign_kernel", DENSE, K, 5, 2, [9, 9])
    assert (bound, unit, launches) == ("tensor", "TFLOP/s", 10)
    assert amount == 5 * 2.0 * (M + N) * K * K


def test_jacobi_flops_follow_the_sweeps():
    # k (k - 1) / 2 column pairs per sweep, 18 k flops per pair; pilot and final cores
    _, amount, _, launches = bench.algorithmic("svd32_cluster_kernel", DENSE, K, 5, 2, [9, 10])
    assert launches == 2
    assert amount == 19 * (K * (K - 1) / 2) * 18.0 * K


def test_refinement_flops_follow_the_iterations():
    _, amount, _, _ = bench.algorithmic("refine_persistent_kernel", DENSE, K, 5, 2, [9, 9], svd_refine=(2, 2))
    assert amount == 4 * 6 * 2.0 * K ** 3


def test_unknown_kernel_has_no_roofline():
    assert bench.algorithmic("draw_kernel", DENSE, K, 5, 2, [9, 9]) is None
    r = bench.roofline_of("draw_kernel", 8, 0.3, DENSE, K, 5, 2, [9, 9], 1, PEAKS, "bf16", "dense")
    assert r["bound"] is None and r["frac"] is None


def test_roofline_rate_and_fraction():
    # 8 GiB streamed in 1.44608 ms: 5940 GB/s, 0.876 of the 6780.7 GB/s copy
    r = bench.roofline_of("tc_residual_kernel", 1, 1.44608, DENSE, K, 5, 2, [9, 9], 1, PEAKS, "bf16",
                          "no-such-workload")
    want = M * N * 4 / 1.44608e-3 / 1e9
    assert abs(r["achieved"] - want) < 1e-3 and abs(want - 5940.15) < 0.01
    assert abs(r["frac"] - want / 6780.7) < 1e-5
    assert r["peak"] == 6780.7 and r["traffic"] is None and r["avg_launch_ms"] == 1.44608


def test_tensor_roofline_takes_the_peak_of_its_dtype():
    args = ("tc_assign_kernel", 10, 2.0, DENSE, K, 5, 2, [9, 9], 1, PEAKS)
    assert bench.roofline_of(*args, "bf16", "x")["peak"] == 1698.5   # BF16 sustained
    assert bench.roofline_of(*args, "tf32", "x")["peak"] == 1027.5   # measured TF32


def test_alu_roofline_takes_fp64_for_the_refinement():
    r = bench.roofline_of("refine_persistent_kernel", 2, 1.0, DENSE, K, 5, 2, [9, 9], 1, PEAKS, "bf16", "x",
                          svd_refine=(2, 2))
    assert r["peak"] == 1.10
    r = bench.roofline_of("svd32_cluster_kernel", 2, 3.2, DENSE, K, 5, 2, [9, 9], 1, PEAKS, "bf16", "x")
    assert r["peak"] == 69.9 and r["sms_used"] == 16
    assert abs(r["frac_of_sms_used"] - r["achieved"] / (69.9 * 16 / 152)) < 1e-4


def test_traffic_figure_goes_stale_with_its_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    table = {"dense": {"x_kernel": dict(dram_bytes_per_launch=123, source="k.cu", captured_on="a test case",
                                        source_sha256=hashlib.sha256(b"kernel v1").hexdigest())}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("x_kernel", "dense")["bytes"] == 123
    assert bench.kernel_traffic("x_kernel", "rbf") is None
    assert bench.kernel_traffic("y_kernel", "dense") is None
    src.write_text("kernel v2")
    assert bench.kernel_traffic("x_kernel", "dense") is None


def _run_bench(args, env_extra=None):
    import os
    import subprocess
    import sys
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), *args], capture_output=True,
                          text=True, env=env, timeout=600)


def test_reference_arm_line_on_the_host():
    """The reference arm (the oracle on one host core) needs no GPU: one JSON
    line with the metric, the reference marker, its cpu_baseline and an e2e
    that copies nothing."""
    out = _run_bench(["--impl", "reference", "--workload", "plain", "--steps", "1", "--warmup", "0"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "sketches/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == dict(value=d["value"], unit="sketches/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert d["config"]["workload"] == "plain"
    # the plain workload's error as the oracle computes it on the whole matrix
    assert abs(cb["oracle_error"] - 0.1162543807549) < 1e-9


def test_reference_arm_other_ranks_exit_quietly():
    out = _run_bench(["--impl", "reference", "--workload", "plain", "--steps", "1", "--warmup", "0"],
                     {"RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0 and out.stdout.strip() == ""
