"""FQNM_TUNE_CACHE: tuned plans persist across processes (child processes,
each with its own library state)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json
from oracle import oracle as orc
from paper_2604_06947_gb300 import fqnm as F, inputs as I
p = I.burgers_problem(n=1 << 16, steps=0)
s = F.Solver.for_problem(p, autotune=1).load(orc.quantise(p.u0, p.delta))
st = s.stats()
print(json.dumps({k: st[k] for k in ("layout", "cells_per_thread", "block", "k")}))
"""


def run(env):
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    import json
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tuned_plans_persist(tmp_path):
    path = tmp_path / "tune.txt"
    env = dict(os.environ, FQNM_TUNE_CACHE=str(path), PYTHONPATH=ROOT)
    first = run(env)
    lines = path.read_text().split("\n")
    assert any(l.strip() for l in lines)
    # the second process takes the plan from the file: rewrite it to a plan
    # the tuner would not pick by itself, and check that it is used
    fields = [l.split() for l in lines if l.strip()]
    forced = [f[:3] + ["1", "4", "64", "16", "1"] for f in fields]
    path.write_text("\n".join(" ".join(f) for f in forced) + "\ngarbage line\n")
    second = run(env)
    assert second == {"layout": 1, "cells_per_thread": 4, "block": 64, "k": 16}
    # an unsupported plan in the file is ignored (tuned again)
    path.write_text("\n".join(" ".join(f[:3] + ["2", "7", "64", "16", "1"]) for f in fields))
    third = run(env)
    assert third["cells_per_thread"] in (4, 8, 16, 32)
