"""The checked build (-DFQNM_CHECKED): every computed index that is not
bounded by construction is verified before its access.  Small cases of each
kernel family run through it in a child process and must report no bounds
error and match the oracle (the stand-in for a sanitizer, which this pool
does not offer)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r"""
import numpy as np
from oracle import oracle as orc
from paper_2604_06947_gb300 import fqnm as F, inputs as I
assert F.checked_build()
# 1-D tiles: every layout, V, one-warp and wide blocks, ragged size
p = I.burgers_problem(n=5000 + 37, steps=0)
q0 = orc.quantise(p.u0, p.delta)
want = orc.step(q0, p.flux, p.delta, p.dx, p.dt, 130, alpha=p.alpha)
for plan in (dict(layout=1, cells_per_thread=4, block=32, k=8),
             dict(layout=2, cells_per_thread=8, block=128, k=64),
             dict(layout=2, cells_per_thread=32, block=512, k=128),
             dict(layout=3, cells_per_thread=16, block=32, k=7),
             dict(layout=4, cells_per_thread=16, block=64, k=64), dict(kernel=1)):
    s = F.Solver.for_problem(p, graph=0, **plan).load(q0)
    s.step(130)
    assert np.array_equal(s.state(), want), plan
    s.close()
# 2-D walk, tiles and march; 3-D march
for dims, opts in (((150, 70), dict()), ((150, 70), dict(nd_tile=3)), ((150, 70), dict(kernel=1)),
                   ((9, 11), dict()), ((20, 9, 13), dict())):
    g = I.burgers_nd_problem(dims)
    q = orc.quantise(g.u0, g.delta).reshape(dims[::-1])
    s = F.Solver.for_problem(g, **opts)
    s.set_grid(g.dims)
    s.load(q.reshape(-1)).step(9)
    assert np.array_equal(s.state().reshape(dims[::-1]),
                          orc.step_nd(q, "burgers_lf", g.delta, g.dx, g.dt, 9, alpha=g.alpha))
    s.close()
# Euler
e = I.sod_problem(n=1000)
s = F.Solver(F.make_flux("euler_roe", gamma=e.gamma), list(e.delta), e.dx, e.dt, "transmissive")
s.load_field(np.stack(e.U0)).step(50)
qe = np.stack([orc.quantise(e.U0[k], e.delta[k]) for k in range(3)])
assert np.array_equal(s.state(), orc.euler_step(qe, e.gamma, e.delta, e.dx, e.dt, 50)[0])
s.close()
# level statistics (radix sort, compaction)
s = F.Solver.for_problem(p).load(q0)
s.step(100)
s.level_step()
s.level_transitions()
s.close()
print("checked ok")
"""


def test_checked_build_runs_clean():
    env = dict(os.environ, FQNM_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked ok" in r.stdout
