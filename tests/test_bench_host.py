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

    def __init__(self, workload):
        self.workload = workload


def test_traffic_records_match_the_sources_and_workloads():
    recs = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    names = {bench.workload(Args(w))["name"] for w in ("tgv3d", "shear2d", "batch", "turb3d")}
    for r in recs:
        assert r["workload"] in names
        assert os.path.exists(os.path.join(ROOT, r["profile"]))
        assert r["source_hash"] == bench.source_hash(), "kernel sources changed since the capture"
    w = bench.workload(Args("tgv3d"))
    per_cell = bench.ncu_traffic("k_step_tma", w["name"], 1)
    assert 90 < per_cell <= 108  # binary16 D3Q27: at most the algorithmic 108 B per cell update


def test_traffic_is_null_once_the_kernel_changed(monkeypatch):
    w = bench.workload(Args("tgv3d"))
    monkeypatch.setattr(bench, "source_hash", lambda: "0000000000000000")
    assert bench.ncu_traffic("k_step_tma", w["name"], 512 ** 3) is None


def test_fp64_flop_counts():
    counts = [bench.fp64_flops_per_cell(eq, bulk) for eq in range(3) for bulk in range(2)]
    assert counts == [116, 122, 107, 112, 100, 105]


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
