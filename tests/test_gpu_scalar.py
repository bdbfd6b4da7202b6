"""Parity of the CUDA scalar path with the oracle: bit-exact integer states.

All states are compared element by element with the oracle on the same
seeded inputs; at the full 2^24-cell size the oracle computes sampled cells
one by one from their dependency cones.
"""
import numpy as np
import pytest

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def oracle_kw(p):
    return dict(kind=p.flux, delta=p.delta, dx=p.dx, dt=p.dt, a=p.a, alpha=p.alpha)


def gpu_q0(p, rounding="half_even"):
    """The initial state: the GPU's quantisation, checked equal to the
    oracle's; the oracle's array is what both sides start from (no oracle
    input comes from the CUDA path)."""
    from oracle import oracle as O
    want = O.quantise(p.u0, p.delta, rounding)
    got = F.fqnm_quantise(p.u0, p.delta, rounding)
    assert np.array_equal(got.astype(np.int64), want)
    return want.astype(np.int32)


def run_and_compare(orc, p, q0, steps, every, boundary="periodic", **opts):
    """Step GPU and oracle side by side; compare at every checkpoint."""
    s = F.Solver.for_problem(p, **opts)
    if boundary != "periodic":
        s.close()
        s = F.Solver(F.make_flux(p.flux, a=p.a, alpha=p.alpha), p.delta, p.dx, p.dt,
                     boundary, **opts)
    s.load(q0)
    q = q0.astype(np.int64)
    done = 0
    while done < steps:
        k = min(every, steps - done)
        s.step(k)
        if p.flux == "burgers_godunov":           # the oracle's two-point form
            q = orc.step_two_point(q, p.flux, p.delta, p.dx, p.dt, k, boundary=boundary)
        else:
            q = orc.step(q, p.flux, p.delta, p.dx, p.dt, k, a=p.a, alpha=p.alpha,
                         boundary=boundary)
        done += k
        got = s.state()
        assert np.array_equal(got.astype(np.int64), q), \
            "mismatch after %d steps at %s" % (done, np.flatnonzero(got != q)[:8])
    stats = s.stats()
    s.close()
    return q, stats


# ---------------------------------------------------------------------------
# quantisation and the transfer rule
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rounding", ["half_even", "half_away", "floor"])
def test_quantise_matches_oracle(orc, rounding):
    p = I.linear_advection_problem(n=4096)
    u = np.concatenate([p.u0, (np.arange(-50, 50) + 0.5) * p.delta])   # exact ties
    got = F.fqnm_quantise(u, p.delta, rounding)
    assert np.array_equal(got.astype(np.int64), orc.quantise(u, p.delta, rounding))
    got64 = F.fqnm_quantise(u * 2 ** 20, p.delta, rounding, state_bits=64)
    assert np.array_equal(got64, orc.quantise(u * 2 ** 20, p.delta, rounding))


def test_quantise_overflow_is_a_status(fq):
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_quantise(np.array([1.0, 3e9]), 1.0)
    assert e.value.status == -4


TABLE_CASES = [
    ("linear_advection", lambda: I.linear_advection_problem(), "half_even"),
    ("burgers", lambda: I.burgers_problem(n=1 << 14), "half_even"),
    ("burgers_floor", lambda: I.burgers_problem(n=1 << 14), "floor"),
    ("burgers_away", lambda: I.burgers_problem(n=1 << 14), "half_away"),
    ("high_frequency", lambda: I.high_frequency_problem(n=1 << 14, steps=10), "half_even"),
]


@pytest.mark.parametrize("name,make,rounding", TABLE_CASES, ids=[c[0] for c in TABLE_CASES])
def test_tables_match_oracle(orc, name, make, rounding):
    p = make()
    s = F.Solver.for_problem(p, rounding=rounding)
    s.load(gpu_q0(p))
    lo, tp, tm = F.fqnm_get_tables(s.h)
    op, om = orc.split_table(p.flux, p.delta, p.dx, p.dt, lo, tp.shape[0], a=p.a,
                             alpha=p.alpha, rounding=rounding)
    assert np.array_equal(tp.astype(np.int64), op)
    assert np.array_equal(tm.astype(np.int64), om)
    s.close()


def test_closed_forms_found_and_verified(orc):
    cases = [(I.linear_advection_problem(), (1, 2)),
             (I.high_frequency_problem(n=1 << 14, steps=10), (9, 10)),
             (I.burgers_problem(n=1 << 12), None)]
    for p, nd in cases:
        s = F.Solver.for_problem(p)
        s.load(gpu_q0(p))
        r = s.rule()
        if nd is None:
            assert r["evaluator"] == 1 and r["has_minus"]
        else:
            assert r["evaluator"] == 2 and (r["num"], r["den"]) == nd
        s.close()


def test_rule_reused_only_for_the_same_range_and_settings(orc):
    """A load whose state range and settings match the last rule built keeps
    that rule; another range, or an option set in between, builds afresh.
    Every run gives the oracle's states."""
    p = I.burgers_problem(n=1 << 12, steps=0)
    q0 = gpu_q0(p)
    want = orc.step(q0, p.flux, p.delta, p.dx, p.dt, 150, alpha=p.alpha)
    s = F.Solver.for_problem(p)
    s.load(q0).step(150)
    r1 = s.rule()
    assert np.array_equal(s.state().astype(np.int64), want)
    s.load(q0).step(150)                                  # same range: rule kept
    assert s.rule() == r1
    assert np.array_equal(s.state().astype(np.int64), want)
    q1 = q0 + 3000                                        # shifted range: rebuilt
    want1 = orc.step(q1, p.flux, p.delta, p.dx, p.dt, 150, alpha=p.alpha)
    s.load(q1).step(150)
    assert s.rule()["lo"] == r1["lo"] + 3000
    assert np.array_equal(s.state().astype(np.int64), want1)
    s.close()
    # a closed form, then the same state with closed forms off, then on again
    p = I.linear_advection_problem()
    q0 = gpu_q0(p)
    want = orc.step(q0, p.flux, p.delta, p.dx, p.dt, 50, a=p.a)
    s = F.Solver.for_problem(p)
    for closed, evaluator in ((1, 2), (0, 1), (1, 2)):
        F.fqnm_set_option(s.h, "closed_form", closed)
        s.load(q0).step(50)
        assert s.rule()["evaluator"] == evaluator
        assert np.array_equal(s.state().astype(np.int64), want)
    s.close()


def test_monotonicity_certificate(orc):
    s = F.Solver.for_problem(I.high_frequency_problem(n=1 << 12, steps=10))
    s.load(gpu_q0(I.high_frequency_problem(n=1 << 12, steps=10)))
    assert s.rule()["monotone"] == 1
    s.close()
    p = I.burgers_problem(n=1 << 12)
    s = F.Solver.for_problem(p)
    s.load(gpu_q0(p))
    assert s.rule()["monotone"] == 0          # split-rounded LF Burgers (measured)
    s.close()


# ---------------------------------------------------------------------------
# parity of the step
# ---------------------------------------------------------------------------

def test_linear_advection_1k_full(orc):
    """Square wave + sine, N = 1024, 2000 steps, checked every 100 steps."""
    p = I.linear_advection_problem()
    q, _ = run_and_compare(orc, p, gpu_q0(p), p.steps, 100)
    assert q.sum() == gpu_q0(p).astype(np.int64).sum()


PLANS = [dict(kernel=1), dict(kernel=4)] + [
    dict(kernel=2, layout=L, cells_per_thread=v, block=b, k=k)
    for L in (1, 2) for v in (4, 8, 16) for b in (64, 256) for k in (1, 7, 32)
] + [dict(kernel=2, layout=1, cells_per_thread=8, block=512, k=64),
     dict(kernel=2, layout=2, cells_per_thread=16, block=512, k=64)] + [
    dict(kernel=2, layout=L, cells_per_thread=v, block=32, k=k)     # one warp per block
    for L in (1, 2) for v in (4, 8, 16) for k in (1, 7, 32)
] + [
    dict(kernel=2, layout=L, cells_per_thread=v, block=b, k=k)      # runs of 4 or 8 cells
    for L, v in ((3, 8), (3, 16), (3, 32), (4, 16), (4, 32)) for b in (32, 64) for k in (1, 7, 32)
] + [dict(kernel=2, layout=3, cells_per_thread=16, block=256, k=64),
     dict(kernel=2, layout=2, cells_per_thread=32, block=32, k=64)]


@pytest.mark.parametrize("plan", PLANS, ids=lambda d: "-".join("%s%s" % kv for kv in d.items()))
def test_every_plan_bit_exact(orc, plan):
    """Every execution plan the tuner can pick, on sizes with ragged tails."""
    for n in (1, 3, 33, 1000, 5003):
        p = I.burgers_problem(n=n, steps=0)
        q0 = gpu_q0(p)
        run_and_compare(orc, p, q0, 75, 75, graph=0, **plan)
    p = I.high_frequency_problem(n=9001, steps=0)
    run_and_compare(orc, p, gpu_q0(p), 75, 75, graph=0, **plan)


@pytest.mark.parametrize("flux", ["burgers_lf", "linear_upwind_closed", "linear_upwind_table",
                                  "burgers_godunov", "burgers_lf_pack16"])
def test_resident_kernel_bit_exact(orc, flux):
    """The one-block kernel (every step of a call in one launch) with each
    evaluator, on lines of one cell, a partial last warp, V = 1, 2, 4, 8 and
    the full 1024 threads; one run (the default plan of a 96-cell line)
    crosses the 65,536-step launch limit."""
    opts = {"linear_upwind_closed": {}, "linear_upwind_table": {"closed_form": 0},
            "burgers_lf_pack16": {"pack16": 1}}.get(flux, {})
    for n in (1, 2, 33, 250, 1000, 1024, 4096, 6000, 8192):
        if flux.startswith("linear"):
            p = I.linear_advection_problem(n=n, steps=0)
        else:
            # delta 2^-12 keeps both maps within int16 for the packed table
            p = I.burgers_problem(n=n, steps=0, delta=2.0 ** (-12 if "pack16" in flux else -16))
            if flux == "burgers_godunov":
                p.flux = "burgers_godunov"
        q0 = gpu_q0(p)
        _, st = run_and_compare(orc, p, q0, 150, 50, kernel=4, **opts)
        assert st["kernel"] == 4 and st["k"] == 0, (n, st)
        assert n % st["cells_per_thread"] == 0 and n // st["cells_per_thread"] == st["block"]
    p = I.burgers_problem(n=96, steps=0)
    if flux == "burgers_lf":                       # the default plan for a short line
        _, st = run_and_compare(orc, p, gpu_q0(p), 70_000, 70_000)
        assert st["kernel"] == 4


def test_graph_replay_bit_exact(orc):
    p = I.burgers_problem(n=70_001, steps=0)
    _, st = run_and_compare(orc, p, gpu_q0(p), 8 * 64 * 2 + 13, 8 * 64 * 2 + 13,
                            k=8, graph=1)
    assert st["graph"] == 1


def test_burgers_1m_full(orc):
    """N = 2^20 Burgers, 10^4 steps, every integer state checked every 100
    steps against the oracle (the bench's workload, the tuned plan)."""
    p = I.burgers_problem()
    q, st = run_and_compare(orc, p, gpu_q0(p), p.steps, 100, autotune=1)
    assert st["kernel"] == 2


def test_high_frequency_reduced_full(orc):
    p = I.high_frequency_problem(n=1 << 16)
    run_and_compare(orc, p, gpu_q0(p), p.steps, 100)


def test_high_frequency_16m_full_state(orc):
    """Full size (2^24 cells, 2000 steps, tuned plan): every cell of the
    final state equal to the oracle's (assembled from dependency windows
    evaluated in parallel host processes), 24 cells checked at step 1000
    from their cones, exact mass and the max principle."""
    p = I.high_frequency_problem()
    q0 = gpu_q0(p)
    q0_64 = q0.astype(np.int64)
    s = F.Solver.for_problem(p, autotune=1)
    s.load(q0)
    s.step(p.steps // 2)
    q_half = s.state()
    rng = np.random.default_rng(11)
    idx = np.concatenate([[0, 1, p.n - 1, p.n // 2], rng.integers(0, p.n, 20)])
    for i in idx:
        want = orc.cone(q0_64, int(i), p.steps // 2, p.flux, p.delta, p.dx, p.dt, a=p.a)
        assert q_half[i] == want, (i, q_half[i], want)
    s.step(p.steps - p.steps // 2)
    q = s.state()
    want = orc.step_by_windows(q0_64, p.steps, p.flux, p.delta, p.dx, p.dt, a=p.a)
    bad = np.flatnonzero(q.astype(np.int64) != want)
    assert bad.size == 0, (bad.size, bad[:8])
    inv = s.invariants()
    assert inv["mass"][0] == int(q0_64.sum())
    assert q.min() >= q0.min() and q.max() <= q0.max()        # certificate holds
    s.close()


def test_transmissive_ends_and_boundary_flux(orc):
    p = I.burgers_problem(n=3001, steps=0)
    q0 = gpu_q0(p)
    q, _ = run_and_compare(orc, p, q0, 400, 100, boundary="transmissive")
    s = F.Solver(F.make_flux(p.flux, alpha=p.alpha), p.delta, p.dx, p.dt, "transmissive")
    s.load(q0).step(400)
    inv = s.invariants()
    _, bf = orc.step(q0, p.flux, p.delta, p.dx, p.dt, 400, alpha=p.alpha,
                     boundary="transmissive", return_bflux=True)
    assert inv["boundary_flux"][0] == bf
    assert inv["mass"][0] == int(q0.astype(np.int64).sum()) - bf
    s.close()


def test_other_fluxes_and_roundings(orc):
    for kind, a, alpha, rounding in (("linear_lf", -0.6, 0.9, "half_even"),
                                     ("linear_lf", 0.6, 0.6, "floor"),
                                     ("burgers_eo", 0.0, 1.3, "half_away"),
                                     ("linear_upwind", -1.0, 0.0, "half_even")):
        p = I.burgers_problem(n=2047, steps=0)
        p.flux, p.a, p.alpha = kind, a, alpha
        p.dt = 0.45 * p.dx / max(abs(a), alpha, 1e-9)
        q0 = gpu_q0(p)
        s = F.Solver(F.make_flux(kind, a=a, alpha=alpha, rounding=rounding), p.delta,
                     p.dx, p.dt)
        s.load(q0).step(333)
        q = orc.step(q0, kind, p.delta, p.dx, p.dt, 333, a=a, alpha=alpha,
                     rounding=rounding)
        assert np.array_equal(s.state().astype(np.int64), q), (kind, rounding)
        s.close()


# ---------------------------------------------------------------------------
# invariants, observable, checkpoints, device interop
# ---------------------------------------------------------------------------

def test_invariants_match_oracle(orc):
    p = I.burgers_problem(n=50_000, steps=0)
    q0 = gpu_q0(p)
    a = F.Solver.for_problem(p).load(q0).step(321)
    b = F.Solver.for_problem(p).load(q0).step(17)
    inv = a.invariants(b)
    qa = orc.step(q0, p.flux, p.delta, p.dx, p.dt, 321, alpha=p.alpha)
    qb = orc.step(q0, p.flux, p.delta, p.dx, p.dt, 17, alpha=p.alpha)
    mass, tv, l1 = orc.invariants(qa, qb)
    assert (inv["mass"][0], inv["tv"][0], inv["l1"][0]) == (mass, tv, l1)
    assert inv["step"] == 321
    a.close(); b.close()


def test_observe_is_delta_times_q(orc):
    p = I.burgers_problem(n=12_345, steps=0)
    s = F.Solver.for_problem(p).load(gpu_q0(p)).step(50)
    q = s.state()
    u = s.observe()
    assert np.array_equal(u, p.delta * q.astype(np.float64))
    import torch
    d32 = torch.empty(p.n, dtype=torch.float32, device="cuda")
    F.fqnm_observe_device(s.h, d32, fp32=True)
    F.fqnm_sync(s.h)
    assert np.array_equal(d32.cpu().numpy(), (p.delta * q.astype(np.float64)).astype(np.float32))
    s.close()


def test_checkpoint_resume_is_bit_identical(orc):
    p = I.burgers_problem(n=40_000, steps=0)
    q0 = gpu_q0(p)
    a = F.Solver.for_problem(p).load(q0).step(500)
    b = F.Solver.for_problem(p).load(q0).step(300)
    mid, step = F.fqnm_checkpoint(b.h, p.n)
    assert step == 300
    c = F.Solver.for_problem(p).load(mid).step(200)
    assert np.array_equal(a.state(), c.state())
    for s in (a, b, c):
        s.close()


def test_torch_device_buffers_and_stream(orc):
    import torch
    p = I.burgers_problem(n=100_000, steps=0)
    u = torch.from_numpy(p.u0).cuda()
    q = torch.empty(p.n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    F.fqnm_quantise_device(u, p.n, p.delta, q, stream=stream)
    s = F.Solver.for_problem(p)
    F.fqnm_set_stream(s.h, stream)
    s.load_device(q, p.n).step(250)
    out = torch.empty(p.n, dtype=torch.int32, device="cuda")
    F.fqnm_checkpoint_device(s.h, out)
    stream.synchronize()
    want = orc.step(orc.quantise(p.u0, p.delta), p.flux, p.delta, p.dx, p.dt, 250,
                    alpha=p.alpha)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), want)
    s.close()


# ---------------------------------------------------------------------------
# range escape: detection and exact recovery (no fault, a status)
# ---------------------------------------------------------------------------

def escaping_problem():
    p = I.burgers_problem(n=4096, steps=0, seed=6)
    p.alpha = 1.0
    p.dt = 0.4 * p.dx / p.alpha
    return p


def test_range_escape_is_recovered_exactly(orc):
    """With alpha = 1.0 below max|u| = 1.3 the LF split is not monotone and the
    states overshoot the initial range (by up to 70 quanta for this seed).
    With no margin the state leaves the table; the library widens the map and
    replays from its last checkpoint, and the result is still bit-exact."""
    p = escaping_problem()
    q0 = gpu_q0(p)
    # the oracle trajectory leaves [min q0, max q0] at some step
    q, escaped = q0.astype(np.int64), False
    for _ in range(100):
        q = orc.step(q, p.flux, p.delta, p.dx, p.dt, 20, alpha=p.alpha)
        escaped |= bool(q.max() > q0.max() or q.min() < q0.min())
    assert escaped
    s = F.Solver.for_problem(p, margin=0)
    s.load(q0).step(2000)
    got = s.state()
    assert np.array_equal(got.astype(np.int64), q)
    assert s.rule()["recoveries"] >= 1
    s.close()


@pytest.mark.parametrize("kernel", [1, 2, 4])
def test_degenerate_inputs(orc, kernel):
    """Empty input and states too close to the int32 limits are statuses; a
    zero-step call changes nothing; a constant state is stationary on every
    kernel (the flux differences vanish identically)."""
    p = I.burgers_problem(n=256, steps=0)
    s = F.Solver.for_problem(p, kernel=kernel)
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_load_states(s.h, np.zeros(0, dtype=np.int32))
    assert e.value.status == -1
    with pytest.raises(F.FqnmError) as e:
        s.load(np.full(256, 2 ** 31 - 100, dtype=np.int32))
    assert e.value.status == -4
    q0 = gpu_q0(p)
    s.load(q0)
    s.step(0)
    assert np.array_equal(s.state(), q0)
    s.load(np.full(256, 12345, dtype=np.int32))
    s.step(333)
    assert (s.state() == 12345).all()
    assert s.stats()["kernel"] == kernel
    s.close()


@pytest.mark.parametrize("plan", [{}, dict(layout=2, cells_per_thread=8, block=128, k=64),
                                  dict(layout=4, cells_per_thread=16, block=64, k=128)])
def test_range_escape_on_a_long_line(orc, plan):
    """The same overshoot on 2^18 cells (the runs-of-8 default and two other
    tiled plans, CUDA-graph replay): the escape is reported, the map widened
    and the run replayed from its checkpoint, bit-exact; with recovery off
    it is a status."""
    p = I.burgers_problem(n=1 << 18, steps=0, seed=6)
    p.alpha = 1.0
    p.dt = 0.4 * p.dx / p.alpha
    q0 = gpu_q0(p)
    want = orc.step(q0.astype(np.int64), p.flux, p.delta, p.dx, p.dt, 1000, alpha=p.alpha)
    s = F.Solver.for_problem(p, margin=0, **plan)
    s.load(q0).step(1000)
    assert np.array_equal(s.state().astype(np.int64), want)
    assert s.rule()["recoveries"] >= 1
    s.close()
    s = F.Solver.for_problem(p, margin=0, recover=0, **plan)
    s.load(q0).step(1000)
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_sync(s.h)
    assert e.value.status == -3
    s.close()


def test_range_escape_without_recovery_is_a_status(orc):
    p = escaping_problem()
    s = F.Solver.for_problem(p, margin=0, recover=0)
    s.load(gpu_q0(p)).step(2000)
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_sync(s.h)
    assert e.value.status == -3
    s.close()


def test_user_supplied_transfer_table(orc):
    """The transfer rule as the primitive object: caller-supplied maps."""
    p = I.burgers_problem(n=3000, steps=0)
    q0 = gpu_q0(p)
    lo, hi = int(q0.min()) - 500, int(q0.max()) + 500
    tp, tm = orc.split_table("burgers_eo", p.delta, p.dx, p.dt, lo, hi - lo + 1)
    h = F.fqnm_create_table(tp.astype(np.int32), tm.astype(np.int32), lo, p.delta)
    F.fqnm_load_states(h, q0)
    F.fqnm_step(h, 200)
    got, _ = F.fqnm_checkpoint(h, p.n)
    want = orc.step(q0, "burgers_eo", p.delta, p.dx, p.dt, 200)
    assert np.array_equal(got.astype(np.int64), want)
    F.fqnm_destroy(h)
