"""bench.py's cpu_baseline leg on the host: the oracle on a bounded sample of
the workload (same cell size and particle density), repeated to a minimum
duration, reported in the line's unit."""
import bench
from paper_2501_10622_gb300 import synth


def test_cpu_baseline_leg_reports_the_oracle_rate():
    wl = synth.WORKLOADS["clumped-512cube-grid1024-L500"]
    r = bench.cpu_baseline_leg(wl, 16, min_seconds=0.2, max_runs=3)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["unit"] == bench.UNIT
    assert r["value"] > 0 and r["seconds"] > 0
    assert "16^3 grid" in r["sample"] and r["sample"].endswith("runs")
    runs = int(r["sample"].rsplit(";", 1)[1].split()[0])
    assert 1 <= runs <= 3
