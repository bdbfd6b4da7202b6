"""Pins of the Euler/Roe oracle, the exact Riemann solver and the FV oracle.

Checked against mathematics that does not come from the oracle's own
formulas: Rankine-Hugoniot jump conditions, isentropic relations and Riemann
invariants across the waves of the exact solution, the paper's printed shock
window, flux consistency, upwinding of the Roe flux for supersonic states,
mirror symmetry, exact integer conservation with boundary-flux accounting, and
convergence of the density error as the grid is refined.
"""
import json
import os

import numpy as np
import pytest

from paper_2604_06947_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
FACTS = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))
G = 1.4
L, R = I.SOD_LEFT, I.SOD_RIGHT


def cons(rho, u, p, g=G):
    return np.array([rho, rho * u, p / (g - 1) + 0.5 * rho * u * u])


def phys_flux(U, g=G):
    rho, m, E = U
    u = m / rho
    p = (g - 1) * (E - 0.5 * rho * u * u)
    return np.array([m, m * u + p, u * (E + p)])


# ---------------------------------------------------------------------------
# exact Riemann solution
# ---------------------------------------------------------------------------

def test_sod_star_state_satisfies_jump_conditions(orc):
    ps, us, rsL, rsR = orc.riemann_star(G, L, R)
    # right-moving shock: Rankine-Hugoniot in the lab frame, speed S
    S = orc.riemann_right_shock_speed(G, L, R)
    Ur, Us = cons(*R), cons(rsR, us, ps)
    lhs = phys_flux(Us) - phys_flux(Ur)
    rhs = S * (Us - Ur)
    assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-12)
    # left rarefaction: isentropic, and u + 2c/(g-1) constant
    assert abs(ps / rsL ** G - L[2] / L[0] ** G) < 1e-12
    cL = np.sqrt(G * L[2] / L[0])
    csL = np.sqrt(G * ps / rsL)
    assert abs((L[1] + 2 * cL / (G - 1)) - (us + 2 * csL / (G - 1))) < 1e-12
    # shock entropy condition: faster than the flow behind it
    assert S > us and ps > R[2]


def test_sod_shock_in_paper_window(orc):
    lo, hi = FACTS["sod_zoom_window"]["value"]
    S = orc.riemann_right_shock_speed(G, L, R)
    xs = 0.5 + 0.2 * S
    assert lo < xs < hi
    x = np.linspace(0.0, 1.0, 20001)
    rho, u, p = orc.riemann_sample(G, L, R, 0.5, 0.2, x)
    # pressure is continuous across the contact: its only jump is the shock
    jump = x[np.argmin(np.diff(p))]
    assert lo < jump < hi
    assert np.all(rho[x > hi] == R[0]) and np.all(rho[(x > 0.7) & (x < lo)] > R[0])


def test_riemann_sample_continuity_and_limits(orc):
    x = np.linspace(0.0, 1.0, 4001)
    rho, u, p = orc.riemann_sample(G, L, R, 0.5, 0.2, x)
    assert rho[0] == L[0] and p[0] == L[2] and rho[-1] == R[0]
    # pressure and velocity are continuous across the contact
    ps, us, _, _ = orc.riemann_star(G, L, R)
    xc = 0.5 + 0.2 * us
    k = np.searchsorted(x, xc)
    assert abs(p[k - 2] - ps) < 1e-12 and abs(p[k + 2] - ps) < 1e-12
    assert abs(u[k - 2] - us) < 1e-12 and abs(u[k + 2] - us) < 1e-12
    # the rarefaction fan is monotone
    fan = (x > 0.5 - 0.2 * np.sqrt(G)) & (x < 0.5 + 0.2 * (us - 0.0) - 0.05)
    assert np.all(np.diff(rho[fan]) <= 1e-15)


# ---------------------------------------------------------------------------
# Roe flux
# ---------------------------------------------------------------------------

def test_roe_flux_consistency(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        U = cons(rng.uniform(0.1, 2), rng.uniform(-2, 2), rng.uniform(0.1, 2))
        F = orc.roe_flux(G, U, U)
        # equal up to the rounding of a differently grouped f(U)
        assert np.allclose(F, phys_flux(U), rtol=1e-14, atol=1e-15)


def test_roe_flux_upwinds_supersonic_states(orc):
    """All Roe eigenvalues positive => F = f(U_L); all negative => f(U_R).
    This holds only if every wave strength, eigenvector and sign is right."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        rl, rr = rng.uniform(0.5, 2, 2)
        pl, pr = rng.uniform(0.2, 1, 2)
        v = rng.uniform(4.0, 6.0)                  # |u| > c for these states
        for sgn in (+1, -1):
            UL = cons(rl, sgn * v, pl)
            UR = cons(rr, sgn * (v + rng.uniform(-0.5, 0.5)), pr)
            F = orc.roe_flux(G, UL, UR)
            want = phys_flux(UL) if sgn > 0 else phys_flux(UR)
            assert np.allclose(F, want, rtol=1e-12, atol=1e-12)


def test_roe_flux_mirror_symmetry(orc):
    """Reflecting x -> -x swaps the states, negates momentum: the mass and
    energy fluxes change sign, the momentum flux does not."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        UL = cons(rng.uniform(0.1, 2), rng.uniform(-1, 1), rng.uniform(0.1, 2))
        UR = cons(rng.uniform(0.1, 2), rng.uniform(-1, 1), rng.uniform(0.1, 2))
        F = orc.roe_flux(G, UL, UR)
        mir = lambda U: np.array([U[0], -U[1], U[2]])
        Fm = orc.roe_flux(G, mir(UR), mir(UL))
        assert np.allclose(Fm, [-F[0], F[1], -F[2]], rtol=1e-12, atol=1e-12)


def test_roe_flux_single_contact_is_exact(orc):
    """An isolated contact (equal u, p) is resolved exactly by Roe: the
    dissipation acts only through the contact wave, |u| times the jump."""
    UL, UR = cons(1.0, 0.5, 1.0), cons(0.3, 0.5, 1.0)
    F = orc.roe_flux(G, UL, UR)
    want = phys_flux(UL) if 0.5 > 0 else phys_flux(UR)
    assert np.allclose(F, want, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# integer Euler step (componentwise quantised Roe transfer)
# ---------------------------------------------------------------------------

def sod_q0(orc, p):
    return np.stack([orc.quantise(p.U0[k], p.delta[k]) for k in range(3)])


def test_sod_integer_conservation_with_boundary_flux(orc):
    p = I.sod_problem(n=256)
    q0 = sod_q0(orc, p)
    q, bf = orc.euler_step(q0, p.gamma, p.delta, p.dx, p.dt, p.steps)
    # exact integer balance: each total changes by its boundary transfer only
    for k in range(3):
        assert q[k].sum() == q0[k].sum() - bf[k]
    # momentum: the ends push p*dt/dx/delta per step (p_L != p_R)
    assert bf[1] * p.delta[1] == pytest.approx(
        p.steps * p.dt / p.dx * (R[2] - L[2]), rel=1e-6)
    # mass and energy: the exact solution has no flux through the ends; the
    # discrete one only the rounding-level tail of its wave profiles
    assert abs(bf[0]) * p.delta[0] < 1e-6 and abs(bf[2]) * p.delta[2] < 1e-6


def test_sod_integer_density_converges_to_exact(orc):
    errs = []
    for n in (128, 256, 512):
        p = I.sod_problem(n=n)
        q, _ = orc.euler_step(sod_q0(orc, p), p.gamma, p.delta, p.dx, p.dt, p.steps)
        rho = p.delta[0] * q[0].astype(np.float64)
        rex, _, _ = orc.riemann_sample(G, L, R, 0.5, 0.2, I.cell_centres(n))
        errs.append(p.dx * np.abs(rho - rex).sum())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.01
    assert errs[0] / errs[2] > 1.6        # about first order (0.5..1 per halving)


def test_sod_integer_tracks_fp_roe_within_quanta(orc):
    """Same Roe flux in FP64 vs quantised transfer at delta = 2^-32: the
    reconstructed states agree to O(steps * delta)."""
    p = I.sod_problem(n=128)
    q, _ = orc.euler_step(sod_q0(orc, p), p.gamma, p.delta, p.dx, p.dt, p.steps)
    U = orc.euler_fv_step(p.U0, p.gamma, p.dx, p.dt, p.steps)
    for k in range(3):
        d = np.abs(p.delta[k] * q[k] - U[k]).max()
        assert d < 4 * p.steps * p.delta[k] * 10
        assert d > 0


# ---------------------------------------------------------------------------
# floating-point finite-volume oracle
# ---------------------------------------------------------------------------

def test_fv64_unit_courant_is_exact_shift(orc):
    n = 500
    rng = np.random.default_rng(5)
    u = rng.integers(-2 ** 20, 2 ** 20, n) * 2.0 ** -20     # dyadic: exact ops
    u1 = orc.fv_step(u, "linear_upwind", 1.0 / n, 1.0 / n, 1, a=1.0)
    assert np.array_equal(u1, np.roll(u, 1))


@pytest.mark.parametrize("kind,a,alpha", [("burgers_lf", 0.0, 1.3),
                                          ("linear_upwind", 1.0, 0.0)])
def test_fv32_close_to_fv64(orc, kind, a, alpha):
    p = I.burgers_problem(n=4096, steps=0)
    u0 = p.delta * orc.quantise(p.u0, p.delta).astype(np.float64)
    u64 = orc.fv_step(u0, kind, p.dx, p.dt, 200, a=a, alpha=alpha)
    u32 = orc.fv_step(u0, kind, p.dx, p.dt, 200, a=a, alpha=alpha, precision="f32")
    rel = np.abs(u32.astype(np.float64) - u64).sum() / np.abs(u64).sum()
    assert rel < 1e-5
    assert rel > 0


def test_fv64_mass_drifts_only_by_rounding(orc):
    """Remark (why floating point cannot give exact invariance): the FP sum
    is conserved only up to rounding, the integer sum exactly."""
    p = I.burgers_problem(n=4096, steps=0)
    q0 = orc.quantise(p.u0, p.delta)
    u0 = p.delta * q0.astype(np.float64)
    u = orc.fv_step(u0, "burgers_lf", p.dx, p.dt, 500, alpha=p.alpha)
    assert abs(u.sum() - u0.sum()) < 1e-9 * np.abs(u0).sum()
    q = orc.step(q0, "burgers_lf", p.delta, p.dx, p.dt, 500, alpha=p.alpha)
    assert q.sum() == q0.sum()


# ---------------------------------------------------------------------------
# partial quantisation (§3.3: the density channel alone on the integer grid)
# ---------------------------------------------------------------------------

def _masked_start(orc, p, mask):
    q = np.zeros((3, p.n), dtype=np.int64)
    for k in range(3):
        if (mask >> k) & 1:
            q[k] = orc.quantise(p.U0[k], p.delta[k])
    return q, np.array(p.U0, dtype=np.float64)


def test_mask_all_is_the_componentwise_step(orc):
    p = I.sod_problem(n=300)
    q0, uf0 = _masked_start(orc, p, 7)
    q, _, bf = orc.euler_step_mask(q0, uf0, 7, p.gamma, p.delta, p.dx, p.dt, 250)
    qc, bfc = orc.euler_step(q0, p.gamma, p.delta, p.dx, p.dt, 250)
    assert np.array_equal(q, qc) and np.array_equal(bf, bfc)


def test_mask_none_is_the_fp64_roe_scheme(orc):
    p = I.sod_problem(n=300)
    q0, uf0 = _masked_start(orc, p, 0)
    q, uf, bf = orc.euler_step_mask(q0, uf0, 0, p.gamma, p.delta, p.dx, p.dt, 250)
    assert np.array_equal(uf, orc.euler_fv_step(p.U0, p.gamma, p.dx, p.dt, 250))
    assert not q.any() and not bf.any()


@pytest.mark.parametrize("mask", [1, 2, 4, 5])
def test_masked_rows_conserve_exactly_and_others_track_fp(orc, mask):
    """Integer rows: mass changes by exactly the counted boundary transfers.
    Every row stays within a few quanta (integer) or a tiny relative
    distance (double) of the all-double scheme over 300 steps."""
    p = I.sod_problem(n=400)
    q0, uf0 = _masked_start(orc, p, mask)
    q, uf, bf = orc.euler_step_mask(q0, uf0, mask, p.gamma, p.delta, p.dx, p.dt, 300)
    ref = orc.euler_fv_step(p.U0, p.gamma, p.dx, p.dt, 300)
    for k in range(3):
        if (mask >> k) & 1:
            assert int(q[k].sum()) == int(q0[k].sum()) - int(bf[k])
            assert np.abs(p.delta[k] * q[k] - ref[k]).max() < 1e-6
        else:
            assert bf[k] == 0
            assert np.abs(uf[k] - ref[k]).max() < 1e-6


def test_mask_rejected_outside_range(orc):
    p = I.sod_problem(n=16)
    q0, uf0 = _masked_start(orc, p, 7)
    with pytest.raises(Exception):
        orc.euler_step_mask(q0, uf0, 9, p.gamma, p.delta, p.dx, p.dt, 1)


def test_euler_fv64_converges_and_conserves(orc):
    """The FP64 Roe finite-volume oracle on its own: its density error
    against the exact Riemann solution falls as the grid is refined, the
    mass and energy totals change only by the flux through the ends (zero
    here: the end states are at rest), up to rounding, and a constant state
    at rest is a fixed point."""
    errs = []
    for n in (128, 512):
        p = I.sod_problem(n=n)
        U = orc.euler_fv_step(p.U0, p.gamma, p.dx, p.dt, p.steps)
        x = I.cell_centres(n)
        rex, _, _ = orc.riemann_sample(G, L, R, 0.5, 0.2, x)
        errs.append(p.dx * np.abs(U[0] - rex).sum())
        for k in (0, 2):
            tot0, tot = p.U0[k].sum(), U[k].sum()
            assert abs(tot - tot0) <= 1e-9 * abs(tot0)
    assert errs[1] < errs[0] / 1.8
    U0 = np.array([np.full(64, 0.7), np.zeros(64), np.full(64, 2.0)])
    assert np.array_equal(orc.euler_fv_step(U0, G, 1.0 / 64, 0.002, 50), U0)


# ---------------------------------------------------------------------------
# windowed evaluation (the dependency-window argument used for sampled and
# parallel parity at large grids)
# ---------------------------------------------------------------------------

def test_euler_window_matches_full_run(orc):
    """Cell runs evaluated from their dependency windows alone (clipped at
    the transmissive ends, where the ghost copy applies) equal those cells of
    the full run: runs at either end, across the diaphragm, one cell, the
    whole tube; and the state assembled from windows in parallel processes
    equals the full run."""
    p = I.sod_problem(n=1000)
    q0 = np.stack([orc.quantise(p.U0[k], p.delta[k]) for k in range(3)]).astype(np.int64)
    steps = 150
    full, _ = orc.euler_step(q0, p.gamma, p.delta, p.dx, p.dt, steps)
    assert not np.array_equal(full, q0)
    for first, count in ((0, 10), (0, 1000), (990, 10), (400, 200), (3, 5), (500, 1),
                         (850, 150), (100, 700), (999, 1)):
        got = orc.euler_window(q0, first, count, steps, p.gamma, p.delta, p.dx, p.dt)
        assert np.array_equal(got, full[:, first:first + count]), (first, count)
    for parts, procs in ((7, 1), (4, 2)):
        got = orc.euler_step_by_windows(q0, steps, p.gamma, p.delta, p.dx, p.dt,
                                        parts=parts, procs=procs)
        assert np.array_equal(got, full), (parts, procs)


def test_euler_window_on_a_moving_state(orc):
    """The same on a state with flow everywhere (a smooth density and
    velocity wave), so that every window's faces carry nonzero transfer."""
    n, steps = 600, 120
    x = I.cell_centres(n)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
    u = 0.3 + 0.1 * np.cos(2 * np.pi * x)
    pr = 1.0 + 0.1 * np.sin(4 * np.pi * x)
    U0 = cons(rho, u, pr)
    delta = [2.0 ** -32] * 3
    dx = 1.0 / n
    dt = 0.4 * dx / 2.0
    q0 = np.stack([orc.quantise(U0[k], delta[k]) for k in range(3)]).astype(np.int64)
    full, _ = orc.euler_step(q0, G, delta, dx, dt, steps)
    for first, count in ((0, 50), (550, 50), (200, 64), (0, 600), (333, 1)):
        got = orc.euler_window(q0, first, count, steps, G, delta, dx, dt)
        assert np.array_equal(got, full[:, first:first + count]), (first, count)
