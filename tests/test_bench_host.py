"""Host-side pieces of bench.py: the CPU description and the serving
stream's oracle baseline on a spawned process pool (a small sample)."""
import os

import numpy as np

import bench


def test_host_cpu_reports_model_and_cores():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count()
    assert h["cpu_model"] and h["machine"]


def test_serving_cpu_baseline_on_a_pool():
    """4 of the 4096 requests on a spawned pool; the comparison counts a
    result equal only when every cell is (one planted difference here)."""
    from oracle import oracle as O
    from paper_2604_06947_gb300 import inputs as I
    reqs = I.serving_stream()
    want = {}
    for i in range(0, len(reqs), 1024):
        p = I.materialise(reqs[i])
        want[i] = O.step(O.quantise(p.u0, p.delta), p.flux, p.delta, p.dx, p.dt, p.steps,
                         a=p.a, alpha=p.alpha)
        p.u0 = None
    planted = 2048
    got = {i: (q if i != planted else q + (np.arange(q.size) == 7)) for i, q in want.items()}
    r, check = bench.serving_cpu_baseline(lambda i: got[i], reqs, every=1024)
    assert r["kind"] == "oracle" and r["cores"] == os.cpu_count()
    assert r["value"] > 0 and r["unit"] == bench.UNIT
    assert "4 of 4096" in r["sample"]
    assert check["requests_checked"] == 4 and check["requests_equal"] == 3
    assert not check["equal"]
