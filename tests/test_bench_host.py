"""The benchmark's CPU-baseline leg on the CPU: the oracle timed on every host
core and on one core, on a small sample, with the thread count restored."""
import pytest


def test_cpu_baseline_reports_all_cores_and_one(oracle_mod):
    import bench
    wl = bench.make_workload("dmr", 24, 8)
    threads = oracle_mod.num_threads()
    out = bench.cpu_baseline(wl, steps=2, max_seconds=5.0, single_core_seconds=2.0)
    assert out["kind"] == "oracle" and out["unit"] == bench.UNIT and out["cores"] == threads
    assert out["value"] > 0 and out["single_core"]["value"] > 0 and out["single_core"]["cores"] == 1
    assert str(wl.mesh.nt) in out["sample"]
    assert oracle_mod.num_threads() == threads
