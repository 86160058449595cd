"""bench.py's host logic without a GPU: the reference arm's JSON line (the
FP64 oracle timed on the host cores), rank handling under torchrun, the
whole-job throughput over ranks, and the DRAM-traffic line read from the
committed ncu summary of the dominant kernel."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(args, env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=300)


def test_reference_arm_prints_one_contract_line():
    # a tiny cut of the workload (the line's keys do not depend on its size)
    r = _run(["--impl", "reference", "--n", "2000", "--views", "1", "--steps", "2", "--warmup", "3"])
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in d, k
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "Mpix/s" and d["vs_baseline"] is None
    assert d["config"]["workload"] == bench.WORKLOAD["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == dict(value=d["value"], unit=d["unit"], h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert d["gpu_launches"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    r = _run(["--impl", "reference", "--n", "2000", "--views", "1", "--steps", "1"],
             env_extra=dict(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1"))
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_job_throughput_counts_all_ranks_over_the_slowest():
    # one process: pixels x steps over the timed region
    v, ms = bench.job_throughput(1_000_000, 10, 20.0)
    assert ms == 20.0
    assert v == pytest.approx(1_000_000 * 10 / 0.020 / 1e6)


def test_traffic_line_follows_the_kernel_sources(monkeypatch):
    got, note = bench.profiled_traffic("render_backward_2d")
    text = open(os.path.join(ROOT, "profiles", bench.STAGE_PROFILE["render_backward_2d"])).read()
    assert "sources_sha1:" in text and "dram_bytes_per_launch_full_workload:" in text
    if got is not None:  # the committed summary was taken on the current sources
        assert got > 0 and "capture" in note
    else:
        assert "stale" in note
    # any change to the hashed sources makes the line stale, so it is not reported
    monkeypatch.setattr(bench, "KERNEL_SOURCES", bench.KERNEL_SOURCES + ("bench.py",))
    got2, note2 = bench.profiled_traffic("render_backward_2d")
    assert got2 is None and "stale" in note2
    assert bench.profiled_traffic("slice_project") == (None, "no ncu summary for this kernel")


def test_cpu_baseline_reports_one_core_and_all_cores():
    """The CPU baseline times the oracle single-threaded and split over all
    host cores in the same run, with the core count and the CPU model."""
    from paper_2310_10642_gb300 import inputs as I
    c = I.config(3, n=2000, n_views=2, scale=0.05)
    cb = bench.cpu_baseline_both(c["gaussians"], c["views"], budget_s=0.5)
    host = bench.host_cpu()
    assert cb["cores"] == host["cores"] >= 1 and isinstance(cb["cpu_model"], str) and cb["cpu_model"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and f"{host['cores']} thread" in cb["sample"]
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and "1 thread" in st["sample"]


def test_block_diagonal_pair_reproduces_the_spatial_rotation(oracle):
    """The quaternion pair the bench uses to render the No-4DRot scene
    through the 4D kernels gives, under the oracle's Eq. 8, exactly
    blockdiag(R3(q), 1) with R3 the textbook rotation of the unit quaternion."""
    import numpy as np
    q = np.random.default_rng(5).normal(size=(4, 300))
    a, b = bench.block_diagonal_pair(q)
    for g in range(300):
        w, x, y, z = q[:, g] / np.linalg.norm(q[:, g])
        R3 = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                       [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                       [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        want = np.eye(4)
        want[:3, :3] = R3
        np.testing.assert_allclose(oracle.rotation4(a[:, g], b[:, g]), want, atol=1e-13)
