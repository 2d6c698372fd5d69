"""Host logic of bench.py that its JSON line rests on: the DoFs-smoothed count, the roofline
object for each slab-solve arithmetic, the p99 of a sample and the replica throughput."""
import math

import pytest

import bench


def test_smoothed_per_cycle_counts_fine_level_sweeps():
    # V(2,2) with S^2 A S^2 before and after the coarse correction: 8 sweeps of S per V-cycle
    assert bench.smoothed_per_cycle(1000, 2, 2) == 8000
    assert bench.smoothed_per_cycle(1000, 1, 1) == 4000


@pytest.mark.parametrize("prec,bound", [(0, "alu"), (1, "alu"), (2, "alu"), (3, "tensor")])
def test_roofline_object_follows_the_arithmetic(prec, bound):
    r = bench.roofline_of(prec, achieved=1.0, fp64_peak=1.25, slab_ms=10.0)
    assert r["bound"] == bound and r["unit"] == "TFLOP/s" and r["ms_per_launch_group"] == 10.0
    assert math.isclose(r["frac"], r["achieved"] / r["peak"])
    if prec == 0:
        assert r["peak"] == 1.25 and r["traffic"] == bench.SLAB_SOLVE_TRAFFIC_FP64
    elif prec == 3:
        assert r["peak"] == bench.measured_peak("bf16_tflops") and r["traffic"] is None
    else:
        assert math.isclose(r["peak"], 152 * 128 * 2 * 2.07e9 / 1e12) and r["traffic"] is None


def test_percentile99_nearest_rank():
    assert bench.percentile99([5.0]) == 5.0
    assert bench.percentile99([3.0, 1.0, 2.0]) == 3.0
    assert bench.percentile99(list(range(101))) == 99


def test_replica_value_is_whole_job_throughput():
    # two replicas, 1000 DoFs smoothed per V-cycle each, 4 V-cycles in 2 ms on the slowest
    assert math.isclose(bench.replica_value(2, 1000.0, 4, 2.0), 2 * 1000.0 * 4 / 2e-3)


def test_cpu_baseline_counts_every_worker_over_the_slowest():
    # two workers, three sweeps each of 1000 DoFs; the first sweep of each is warm-up
    res = {"workers": 2, "times": [[9.0, 1.0, 1.0], [9.0, 2.0, 2.0]], "dofs_per_sweep": 1000,
           "setup_s": 5.0, "wall_s": 13.0}
    d = bench.cpu_baseline_desc(res, 16, skip=1)
    assert d["cores"] == 2 and d["kind"] == "oracle"
    # 4 timed sweeps of 1000 DoFs; the slowest worker needed 4 s for its two
    assert math.isclose(d["value"], 4 * 1000 / 4.0)
    assert math.isclose(d["sweep_s_median"], 1.5)


def test_both_arms_name_the_same_workload():
    c = bench.workload_config()
    assert c["workload"] == bench.WORKLOAD["name"] and c["dofs"] == 26416 * 256 * 2
