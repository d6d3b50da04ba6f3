"""Host logic of bench.py (no GPU): the DRAM-traffic records are used only while the
kernel sources match, every workload has a name the records can refer to, the FP64 flop
counts and the rank aggregation are consistent."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class Args:
    n = None
    precision = None
    eq = "entropic"
    batch_count = 4096

    def __init__(self, workload):
        self.workload = workload


def test_traffic_records_match_the_sources_and_workloads():
    recs = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    names = {bench.workload(Args(w))["name"] for w in ("tgv3d", "shear2d", "batch", "turb3d")}
    for r in recs:
        assert r["workload"] in names
        assert os.path.exists(os.path.join(ROOT, r["profile"]))
        assert r["source_hash"] == bench.source_hash(), "kernel sources changed since the capture"
        # every record names the launch shape it was taken in
        keys = ("threads", "blocks") if r["kernel"] == "k_step_batch" else bench.LAUNCH_KEYS
        assert r["precision"] in ("F64", "F32", "F16S") and r["bulk_corr"] in (0, 1)
        assert all(isinstance(r["launch"].get(k), int) for k in keys), r
    w = bench.workload(Args("tgv3d"))
    tgv = [r for r in recs if r["workload"] == w["name"] and r["kernel"] == "k_step_tma" and r["precision"] == "F16S"]
    assert tgv
    for r in tgv:
        per_cell, note = bench.ncu_traffic("k_step_tma", w["name"], 1, launch=r["launch"])
        assert note and 90 < per_cell <= 108  # binary16 D3Q27: at most the algorithmic 108 B per cell


def test_traffic_needs_the_launch_shape_that_ran():
    w = bench.workload(Args("tgv3d"))
    other = {"threads": 96, "blocks": 7, "stages": 5, "rows": 3, "seg": 11, "smem_bytes": 12345}
    value, note = bench.ncu_traffic("k_step_tma", w["name"], 512 ** 3, launch=other)
    assert value is None and "launch shape" in note


def test_traffic_is_null_once_the_kernel_changed(monkeypatch):
    w = bench.workload(Args("tgv3d"))
    monkeypatch.setattr(bench, "source_hash", lambda: "0000000000000000")
    value, note = bench.ncu_traffic("k_step_tma", w["name"], 512 ** 3)
    assert value is None and "source changed" in note


def test_fp64_flop_counts():
    counts = [bench.fp64_flops_per_cell(eq, bulk) for eq in range(3) for bulk in range(2)]
    assert counts == [116, 122, 107, 112, 100, 105]
    counts3 = [bench.fp64_flops_per_cell(eq, bulk, D=3) for eq in range(3) for bulk in range(2)]
    assert counts3 == [309, 315, 310, 315, 284, 289]


def test_cpu_baseline_helpers():
    info = bench.cpu_info()
    assert info["model"] and info["logical_cpus"] >= 1 and info["usable_cpus"] >= 1
    from oracle import core
    from paper_2303_08163_gb300 import inputs
    rho, u = inputs.taylor_green_2d(32, u0=0.05)
    f = core.init(2, (32, 32, 1), 0, rho, u)
    g, steps, used = bench.time_oracle(2, (32, 32, 1), 0, 0, 0.8, f, 2, 0.05)
    assert g > 0 and steps >= 1 and used >= 1
    assert core.set_threads(1) == 1
    for wl in ("tgv3d", "shear2d", "batch", "turb3d", "tgv2d"):
        D, dims, eq, tau, rho, u, what = bench.cpu_sample(bench.workload(Args(wl)))
        n = 1
        for d in dims:
            n *= d
        assert rho.shape == (n,) and u.shape == (D, n) and tau > 0.5 and what


def test_defaults_are_the_contract():
    sys_argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        a = bench.parse()
    finally:
        sys.argv = sys_argv
    assert a.gpus == 1 and a.workload == "tgv3d" and a.impl == "native" and a.warmup >= 3
    w = bench.workload(a)
    assert w["dims"] == (512, 512, 512) and w["prec"] == bench.PREC["f16s"]


@pytest.mark.parametrize("world", [1, 2, 4])
def test_aggregate_is_weak_scaling(world):
    g = bench.aggregate(world, 1000, 10, [2.0] * world)
    assert abs(g - world * 1000 * 10 / 2e-3 / 1e9) < 1e-12


def test_fp64_pipe_record_of_the_fp64_storage_path():
    w = bench.workload(Args("tgv3d"))
    launch = {"kernel": 1, "threads": 128, "blocks": 2432}
    pipe = bench.fp64_pipe(w["name"], 0, launch, 2.44, 2070.0)
    assert pipe is not None and 200 < pipe["fp64_thread_inst_per_cell_update"] < 300
    assert 0.5 < pipe["frac"] < 1.05
    assert bench.fp64_pipe(w["name"], 0, dict(launch, threads=256), 2.44, 2070.0) is None
