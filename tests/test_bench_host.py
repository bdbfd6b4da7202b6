"""Host-side pieces of bench.py: the CPU description and the serving
stream's oracle baseline on a spawned process pool (a small sample)."""
import os

import bench


def test_host_cpu_reports_model_and_cores():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count()
    assert h["cpu_model"] and h["machine"]


def test_serving_cpu_baseline_on_a_pool():
    r = bench.serving_cpu_baseline(every=1024)          # 4 of the 4096 requests
    assert r["kind"] == "oracle" and r["cores"] == os.cpu_count()
    assert r["value"] > 0 and r["unit"] == bench.UNIT
    assert "4 of 4096" in r["sample"]
