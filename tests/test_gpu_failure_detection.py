"""Failure detection without a GPU fault: the conserved-totals check
(FQNM_OPT_VERIFY) on clean runs and on a state corrupted from the host, and
resume from a checkpoint with its step counter and boundary transfer."""
import numpy as np
import pytest
import torch

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def sod_solver(p, **opt):
    return F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                    "transmissive", **opt)


def test_verify_passes_on_clean_runs(orc):
    """No false alarm: periodic Burgers, a run that escapes its range and is
    recovered, transmissive Sod (totals move by the counted transfer), a
    density-only Sod (the double components are skipped) and a 2-D grid."""
    p = I.burgers_problem(n=1 << 15, steps=0)
    s = F.Solver.for_problem(p, verify=1).load(orc.quantise(p.u0, p.delta))
    s.step(1000)
    F.fqnm_sync(s.h)
    s.close()
    e = I.burgers_problem(n=4096, steps=0, seed=6)
    e.alpha, e.dt = 1.0, 0.4 * e.dx
    s = F.Solver.for_problem(e, margin=0, verify=1).load(orc.quantise(e.u0, e.delta))
    s.step(2000)
    F.fqnm_sync(s.h)
    assert F.fqnm_get_rule(s.h)["recoveries"] >= 1
    s.close()
    q = I.sod_problem(n=2048)
    for mask in (7, 1):
        s = sod_solver(q, verify=1, quantise_mask=mask).load_field(np.stack(q.U0))
        s.step(800)
        F.fqnm_sync(s.h)
        if mask == 7:       # momentum moves through the ends (the pressure there)
            assert s.invariants()["boundary_flux"][1] != 0
        s.close()
    g = I.burgers_nd_problem((96, 80))
    s = F.Solver.for_problem(g, verify=1)
    s.set_grid(g.dims)
    s.load(orc.quantise(g.u0, g.delta)).step(40)
    F.fqnm_sync(s.h)
    s.close()


def test_host_injected_corruption_is_reported(orc):
    """One cell of the live state is overwritten from the host between
    steps (one int32 written through the state pointer); the next
    synchronising call reports it, and a clean reload clears it."""
    p = I.burgers_problem(n=1 << 14, steps=0)
    q0 = orc.quantise(p.u0, p.delta)
    s = F.Solver.for_problem(p, verify=1).load(q0)
    s.step(100)
    ptr, n = F.fqnm_state_device(s.h)
    assert n == p.n
    poke = torch.tensor([7.0], dtype=torch.float64, device="cuda")
    F.fqnm_quantise_device(poke, 1, 1.0, ptr + 4 * 1234)     # q[1234] <- 7
    torch.cuda.synchronize()
    s.step(10)
    with pytest.raises(F.FqnmError, match="conservation check failed"):
        F.fqnm_sync(s.h)
    s.load(q0).step(10)
    F.fqnm_sync(s.h)
    s.close()


def test_sod_resume_is_bit_identical(orc):
    """Checkpoint after 600 steps, resume in a new solver with the step and
    the boundary transfer: after 400 more steps the states, totals, transfer
    and step equal those of the uninterrupted run (and the check holds)."""
    p = I.sod_problem(n=4096)
    a = sod_solver(p).load_field(np.stack(p.U0))
    a.step(1000)
    b = sod_solver(p).load_field(np.stack(p.U0))
    b.step(600)
    mid, step = F.fqnm_checkpoint(b.h, p.n, 3)
    bf = b.invariants()["boundary_flux"]
    c = sod_solver(p, verify=1)
    F.fqnm_resume(c.h, mid, step, bf)
    c.n = p.n
    c.step(400)
    assert np.array_equal(c.state(), a.state())
    ia, ic = a.invariants(), c.invariants()
    assert ia == ic and ic["step"] == 1000
    for s in (a, b, c):
        s.close()
