"""The allocation-free invariants entry point against the regular one.

fqnm_invariants_noalloc serves callers that cannot let the library allocate
device memory (their free memory belongs to their own pool, or their loop
cannot afford the device-wide wait of cudaFree).  It keeps its scratch in one
static device array shared by all calls.  This file is collected last, so a
failure here leaves every other test already run; it also passes on its own
in a fresh process, where its first call performs the per-device set-up.
"""
import numpy as np
import pytest

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MAX_CELLS = 1 << 26


def states(n, boundary, steps_a=250, steps_b=40):
    """Two evolved Burgers states on the device and the regular entry
    point's invariants of a against b."""
    import torch
    p = I.burgers_problem(n=n, steps=0)
    q0 = F.fqnm_quantise(p.u0, p.delta)
    flux = F.make_flux(p.flux, alpha=p.alpha)
    a = F.Solver(flux, p.delta, p.dx, p.dt, boundary).load(q0).step(steps_a)
    b = F.Solver(flux, p.delta, p.dx, p.dt, boundary).load(q0).step(steps_b)
    want = a.invariants(b)
    qa = torch.empty(n, dtype=torch.int32, device="cuda")
    qb = torch.empty(n, dtype=torch.int32, device="cuda")
    F.fqnm_checkpoint_device(a.h, qa)
    F.fqnm_checkpoint_device(b.h, qb)
    F.fqnm_sync(a.h)
    F.fqnm_sync(b.h)
    a.close()
    b.close()
    return qa, qb, (want["mass"][0], want["tv"][0], want["l1"][0])


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    # a large call, then a smaller one that reuses fewer partial slots: the
    # second must not see the first call's leftovers
    qa, qb, want = states(1_000_003, "periodic")
    for _ in range(2):
        assert F.fqnm_invariants_noalloc(qa, qa.numel(), qb) == want
    qa2, qb2, want2 = states(20_001, "transmissive", 90, 7)
    for _ in range(2):
        assert F.fqnm_invariants_noalloc(qa2, qa2.numel(), qb2, "transmissive") == want2
    mass, tv, l1 = F.fqnm_invariants_noalloc(qa2, qa2.numel(), None, "transmissive")
    assert (mass, tv, l1) == (want2[0], want2[1], 0)


def test_noalloc_rejects_sizes_beyond_its_limit():
    qa, _, _ = states(4096, "periodic")
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_invariants_noalloc(qa, MAX_CELLS + 1)
    assert e.value.status == -1 and "limit" in str(e.value)
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_invariants_noalloc(qa, 0)
    assert e.value.status == -1
