"""Pins of the d-dimensional oracle step (Theorem, Cartesian extension by
directional composition; eqs. nd_transfer_rule, nd_flux_definition).

Checked against: the pinned one-dimensional step (d = 1; states constant
along all but one axis, where the other axes' face fluxes cancel), an
independent face-by-face exchange written here from the maps of the pinned
table builder, transposition symmetry (the same rule on every axis), exact
conservation (part (i) of the Theorem), and the closed form of linear upwind
at nu = 1/2 on even states (q' = (q_{i-x} + q_{i-y}) / 2 in 2-D).
"""
import numpy as np
import pytest

from paper_2604_06947_gb300 import inputs as I


def burgers_params(n=64):
    p = I.burgers_problem(n=n)
    return dict(kind="burgers_lf", delta=p.delta, dx=p.dx, dt=p.dt / 2, alpha=p.alpha)


def rand_state(rng, shape, delta, lo=-0.3, hi=1.3):
    return np.round(rng.uniform(lo, hi, shape) / delta).astype(np.int64)


def test_d1_is_the_one_dimensional_step(orc):
    P = burgers_params()
    q = rand_state(np.random.default_rng(1), 300, P["delta"])
    got = orc.step_nd(q, P["kind"], P["delta"], P["dx"], P["dt"], 40, alpha=P["alpha"])
    want = orc.step(q, P["kind"], P["delta"], P["dx"], P["dt"], 40, alpha=P["alpha"])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("axis", [0, 1])
def test_states_constant_along_an_axis_evolve_in_one_dimension(orc, axis):
    P = burgers_params()
    line = rand_state(np.random.default_rng(2), 37, P["delta"])
    q = np.tile(line, (23, 1)) if axis == 0 else np.tile(line[:, None], (1, 23))
    got = orc.step_nd(q, P["kind"], P["delta"], P["dx"], P["dt"], 25, alpha=P["alpha"])
    want = orc.step(line, P["kind"], P["delta"], P["dx"], P["dt"], 25, alpha=P["alpha"])
    want2 = np.tile(want, (23, 1)) if axis == 0 else np.tile(want[:, None], (1, 23))
    assert np.array_equal(got, want2)


def test_3d_slab_constant_in_z_is_the_2d_step(orc):
    P = burgers_params()
    q2 = rand_state(np.random.default_rng(3), (9, 11), P["delta"])
    q3 = np.tile(q2, (5, 1, 1))
    got = orc.step_nd(q3, P["kind"], P["delta"], P["dx"], P["dt"], 12, alpha=P["alpha"])
    want = orc.step_nd(q2, P["kind"], P["delta"], P["dx"], P["dt"], 12, alpha=P["alpha"])
    for z in range(5):
        assert np.array_equal(got[z], want)


def face_exchange(q, phip, phim, lo, steps):
    """Every face of every axis moves F = phi+(left) + phi-(right) quanta from
    its left cell to its right cell, all from the state before the step."""
    q = q.copy()
    for _ in range(steps):
        old = q.copy()
        for ax in range(q.ndim):
            right = np.roll(old, -1, axis=ax)
            F = phip[old - lo] + phim[right - lo]
            q -= F
            q += np.roll(F, 1, axis=ax)
    return q


@pytest.mark.parametrize("shape", [(7, 5), (4, 6, 3), (1, 9)])
def test_cell_form_equals_face_exchange(orc, shape):
    P = burgers_params()
    q = rand_state(np.random.default_rng(4), shape, P["delta"])
    lo, hi = int(q.min()) - 2000, int(q.max()) + 2000
    phip, phim = orc.split_table(P["kind"], P["delta"], P["dx"], P["dt"], lo, hi - lo + 1,
                                 alpha=P["alpha"])
    got = orc.step_nd(q, P["kind"], P["delta"], P["dx"], P["dt"], 6, alpha=P["alpha"])
    assert np.array_equal(got, face_exchange(q, phip, phim, lo, 6))


def test_transposition_symmetry_and_conservation(orc):
    P = burgers_params()
    q = rand_state(np.random.default_rng(5), (16, 24), P["delta"])
    a = orc.step_nd(q, P["kind"], P["delta"], P["dx"], P["dt"], 30, alpha=P["alpha"])
    b = orc.step_nd(q.T.copy(), P["kind"], P["delta"], P["dx"], P["dt"], 30, alpha=P["alpha"])
    assert np.array_equal(a, b.T)
    assert a.sum() == q.sum()
    q3 = rand_state(np.random.default_rng(6), (6, 7, 8), P["delta"])
    c = orc.step_nd(q3, P["kind"], P["delta"], P["dx"], P["dt"], 30, alpha=P["alpha"])
    assert c.sum() == q3.sum()


def test_linear_upwind_half_courant_closed_form(orc):
    """phi+(q) = q/2 exactly on even q, phi- = 0: one 2-D step gives
    q' = q - 2 (q/2) + q_{i-x}/2 + q_{i-y}/2."""
    rng = np.random.default_rng(7)
    q = 2 * rng.integers(-500, 500, (10, 13))
    got = orc.step_nd(q, "linear_upwind", 1.0, 1.0, 0.5, 1, a=1.0)
    want = (np.roll(q, 1, axis=1) + np.roll(q, 1, axis=0)) // 2
    assert np.array_equal(got, want)
