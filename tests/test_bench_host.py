"""Host-side pieces of bench.py that need no GPU: the CPU oracle baselines
(one core and all cores, the latter as spawned worker processes)."""
import workloads as WL


def test_cpu_oracle_baselines_run_and_add_up():
    import bench
    A = WL.pr1(seed=0, n=1500)
    one, times = bench.cpu_oracle_baseline(A, steps=2, budget_s=0.2)
    assert one["cores"] == 1 and one["value"] > 0 and len(times) >= 2
    allc = bench.cpu_oracle_all_cores(A, budget_s=0.2, workers=2)
    assert allc["cores"] == 2 and allc["value"] > 0 and allc["kind"] == "oracle"
    assert "2 row blocks" in allc["sample"]
