"""Batched serving: every result bit-exact, the same alone and in the mix,
admission bounded by the memory budget and the slots."""
import numpy as np
import pytest

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I
from paper_2604_06947_gb300 import serve as S

pytestmark = pytest.mark.gpu


def oracle_result(orc, rq, q0_gpu):
    """The oracle's final state of one request (large ones from dependency
    windows in parallel host processes).  The oracle quantises the request's
    field itself; the GPU's initial state must equal it."""
    p = I.materialise(rq)
    q0 = orc.quantise(p.u0, p.delta)
    p.u0 = None
    assert np.array_equal(np.asarray(q0_gpu, dtype=np.int64), q0)
    if p.n * p.steps > 50_000_000:
        return orc.step_by_windows(q0, p.steps, p.flux, p.delta, p.dx, p.dt, a=p.a,
                                   alpha=p.alpha)
    return orc.step(q0, p.flux, p.delta, p.dx, p.dt, p.steps, a=p.a, alpha=p.alpha)


def small_stream(n_requests=48, seed=7, n_max=1 << 14, steps_max=800):
    return I.serving_stream(n_requests=n_requests, rate_hz=20_000.0, n_min=256,
                            n_max=n_max, steps_min=50, steps_max=steps_max, seed=seed)


def test_batched_results_equal_single_and_oracle(orc):
    reqs = small_stream()
    q0s = S.prepare(reqs)
    # 6 slots and an 8 MiB budget (a Burgers problem needs about 3.1 MB):
    # requests wait for slots and memory
    bat = S.serve_batched(reqs, q0s, budget_bytes=8 << 20, max_slots=6, deadline_s=120)
    one = S.serve_one_by_one(reqs, q0s)
    for i in range(len(reqs)):
        assert np.array_equal(bat["results"][i], one["results"][i]), i
    for i in range(len(reqs)):                  # every request against the oracle
        want = oracle_result(orc, reqs[i], q0s[i])
        assert np.array_equal(bat["results"][i].astype(np.int64), want), i
    assert bat["epochs"] >= max(r.problem.steps for r in reqs) // 32
    assert bat["p99_ms"] >= bat["p50_ms"] > 0


def test_same_alone_and_in_the_mix():
    reqs = small_stream(seed=9)
    q0s = S.prepare(reqs)
    mix = S.serve_batched(reqs, q0s, budget_bytes=64 << 20, max_slots=64)
    for i in (3, 17, 40):
        alone = S.serve_batched([reqs[i]], [q0s[i]], budget_bytes=64 << 20, max_slots=1)
        assert np.array_equal(alone["results"][0], mix["results"][i])


@pytest.mark.parametrize("plan", [dict(cells_per_thread=4, block=256, k=16, layout=2),
                                  dict(cells_per_thread=16, block=128, k=64, layout=2),
                                  dict(cells_per_thread=8, block=256, k=32, layout=1)])
def test_every_batch_plan_gives_the_same_results(plan):
    reqs = small_stream(n_requests=24, seed=11)
    q0s = S.prepare(reqs)
    ref = S.serve_one_by_one(reqs, q0s)
    bat = S.serve_batched(reqs, q0s, budget_bytes=64 << 20, max_slots=16, plan=plan)
    for i in range(len(reqs)):
        assert np.array_equal(bat["results"][i], ref["results"][i]), (plan, i)


def test_online_autotune_keeps_results():
    reqs = small_stream(n_requests=40, seed=12)
    q0s = S.prepare(reqs)
    ref = S.serve_one_by_one(reqs, q0s)
    bat = S.serve_batched(reqs, q0s, budget_bytes=64 << 20, max_slots=8, plan="autotune")
    for i in range(len(reqs)):
        assert np.array_equal(bat["results"][i], ref["results"][i]), i
    assert bat["plan"]["cells_per_thread"] in (8, 16)


def test_device_submission_and_device_results(orc):
    import torch
    reqs = small_stream(n_requests=20, seed=14)
    dev = S.DeviceStream(reqs)
    S.serve_batched(reqs, dev=dev, budget_bytes=32 << 20, max_slots=4)
    out = torch.empty_like(dev.out)
    S.serve_one_by_one(reqs, dev=dev, out=out)
    assert torch.equal(out, dev.out)
    for i, rq in enumerate(reqs):
        want = oracle_result(orc, rq, dev.q0(i).cpu().numpy())
        assert np.array_equal(dev.result(i).cpu().numpy().astype(np.int64), want), i


def test_large_problems_in_the_mix(orc):
    """Problems up to 2^20 cells next to small ones: every final state equal
    to the oracle's, and to one-at-a-time execution."""
    reqs = I.serving_stream(n_requests=12, rate_hz=5000.0, n_min=256, n_max=1 << 20,
                            steps_min=100, steps_max=1500, seed=13)
    q0s = S.prepare(reqs)
    bat = S.serve_batched(reqs, q0s, budget_bytes=1 << 30, max_slots=32)
    for i, rq in enumerate(reqs):
        want = oracle_result(orc, rq, q0s[i])
        assert np.array_equal(bat["results"][i].astype(np.int64), want), i
    one = S.serve_one_by_one(reqs, q0s)
    for i in range(len(reqs)):
        assert np.array_equal(bat["results"][i], one["results"][i])


def test_range_escapes_restart_inside_the_pipeline(orc):
    """Maps built with no margin around an under-dissipative Burgers split
    (alpha = 1 against max|u| = 1.3: states leave their initial range): each
    escape is seen one epoch late, with the next epoch already enqueued, and
    restarts only that problem with a wider map; every result still equals
    the oracle's, next to ordinary requests in the same stream."""
    base = small_stream(n_requests=10, seed=31)
    reqs = []
    for i, rq in enumerate(base):
        p = I.materialise(rq)
        if i % 3 == 0:                                   # the escaping problems
            e = I.burgers_problem(n=4096, steps=600 + 100 * i, seed=6 + i)
            e.alpha, e.dt = 1.0, 0.4 * e.dx
            p = e
        reqs.append(I.ServeRequest(rq.rid, rq.arrival_s, p, rq.data_seed))
    q0s = [F.fqnm_quantise(rq.problem.u0, rq.problem.delta) for rq in reqs]
    # the same escape on the single-problem path (it recovers there too)
    e = reqs[0].problem
    s = F.Solver.for_problem(e, margin=0).load(q0s[0])
    s.step(e.steps)
    F.fqnm_sync(s.h)
    assert F.fqnm_get_rule(s.h)["recoveries"] >= 1
    s.close()
    bat = S.serve_batched(reqs, q0s, budget_bytes=64 << 20, max_slots=4, margin=0,
                          plan=dict(cells_per_thread=8, block=128, k=16, layout=2))
    for i, rq in enumerate(reqs):
        p = rq.problem
        want = orc.step(orc.quantise(p.u0, p.delta), p.flux, p.delta, p.dx, p.dt, p.steps,
                        a=p.a, alpha=p.alpha)
        assert np.array_equal(bat["results"][i].astype(np.int64), want), i


def test_tight_budget_admits_one_at_a_time():
    """A budget that holds one problem's tables at a time (and the states of
    several): admission must still make progress, in order."""
    reqs = small_stream(n_requests=10, seed=21)
    q0s = S.prepare(reqs)
    ref = S.serve_one_by_one(reqs, q0s)
    for budget in (3_300_000, 5 << 20):
        bat = S.serve_batched(reqs, q0s, budget_bytes=budget, max_slots=6, deadline_s=60)
        for i in range(len(reqs)):
            assert np.array_equal(bat["results"][i], ref["results"][i])


def test_batch_rejections_are_statuses():
    p = I.burgers_problem(n=4096, steps=10)
    q0 = F.fqnm_quantise(p.u0, p.delta)
    b = F.fqnm_batch_create(4 << 20, 4)
    try:
        with pytest.raises(F.FqnmError) as e:            # larger than the budget
            F.fqnm_batch_submit(b, F.make_spec(I.burgers_problem(n=1 << 20, steps=1)),
                                np.zeros(1 << 20, dtype=np.int32), 1)
        assert e.value.status == -5
        spec = F.make_spec(p)
        spec.boundary = 1
        with pytest.raises(F.FqnmError) as e:            # transmissive is not served
            F.fqnm_batch_submit(b, spec, q0, 10)
        assert e.value.status == -1
        spec = F.make_spec(p)
        spec.dt = 2 * p.dx / p.alpha
        with pytest.raises(F.FqnmError) as e:            # Courant number 2
            F.fqnm_batch_submit(b, spec, q0, 10)
        assert e.value.status == -2
        rid = F.fqnm_batch_submit(b, F.make_spec(p), q0, 10)
        while not F.fqnm_batch_completed(b, 8):
            F.fqnm_batch_progress(b, 4)
        q, lat = F.fqnm_batch_poll(b, rid, p.n)
        assert q is not None and lat > 0
        with pytest.raises(F.FqnmError) as e:            # handed out already
            F.fqnm_batch_poll(b, rid, p.n)
        assert e.value.status == -8
    finally:
        F.fqnm_batch_destroy(b)
