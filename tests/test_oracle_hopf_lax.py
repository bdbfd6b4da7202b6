"""Pins of the Hopf-Lax reference oracle (the entropy reference of the
paper's Burgers test, §3.2), from the mathematics of inviscid Burgers:
the smooth solution by characteristics before the shock forms, constant
data, the monotonicity of the minimiser in x (Oleinik's one-sided bound
u(x+z) - u(x) <= z / t, exact on the candidate grid), the shock position
fixed by the symmetry of u0 = 0.5 + sin(2 pi x) (in the frame moving at 0.5
the data are odd about 1/2, so the shock stays at 1/2: x_s = 0.5 + 0.5 t),
and conservation of the mean.
"""
import math

import numpy as np
import pytest

from oracle import hopf_lax as HL

A, B = 0.5, 1.0
T_SHOCK = 1.0 / (2.0 * math.pi * B)


def test_primitive_is_the_integral_of_u0():
    y = np.linspace(-1.0, 2.0, 301)
    U = HL.sine_primitive(y, A, B)
    dU = np.gradient(U, y)
    assert np.abs(dU[5:-5] - (A + B * np.sin(2 * math.pi * y[5:-5]))).max() < 1e-3
    assert abs(HL.sine_primitive(1.0, A, B) - HL.sine_primitive(0.0, A, B) - A) < 1e-15


@pytest.mark.parametrize("t", [0.05, 0.1, 0.15])
def test_smooth_solution_before_the_shock(t):
    """Before t_shock = 1/(2 pi) the objective is strictly convex in y, so
    the grid argmin is one of the two candidates around the continuous
    minimiser: |u - u_exact| <= h / t with h the candidate spacing."""
    ny = 4096
    x = (np.arange(512) + 0.5) / 512
    y, U = HL.periodic_candidates(ny, A, B)
    u, _ = HL.hopf_lax(x, y, U, t)
    ue = HL.characteristics(x, t, A, B)
    assert np.abs(ue - (A + B * np.sin(2 * math.pi * (x - ue * t)))).max() < 1e-13
    assert np.abs(u - ue).max() <= (1.0 / ny) / t


def test_constant_data():
    y, U = HL.periodic_candidates(1024, 0.7, 0.0)
    x = (np.arange(100) + 0.5) / 100
    u, _ = HL.hopf_lax(x, y, U, 0.3)
    assert np.abs(u - 0.7).max() <= (1.0 / 1024) / 0.3


@pytest.mark.parametrize("t", [0.2, 0.3, 0.45])
def test_oleinik_bound_and_shock_position(t):
    """After the shock: minimisers nondecreasing in x, hence
    u_{i+1} - u_i <= dx / t; one large downward jump, at 0.5 + 0.5 t."""
    nx, ny = 4096, 2048
    x = (np.arange(nx) + 0.5) / nx
    y, U = HL.periodic_candidates(ny, A, B)
    u, idx = HL.hopf_lax(x, y, U, t)
    ystar = y[idx]
    assert np.all(np.diff(ystar) >= 0)
    assert np.all(np.diff(u) <= (1.0 / nx) / t + 1e-12)
    jump = np.argmin(np.diff(u))
    xs = 0.5 * (x[jump] + x[jump + 1])
    assert abs(xs - (0.5 + 0.5 * t) % 1.0) <= 2.0 / nx + (1.0 / ny) / t
    assert np.diff(u)[jump] < -0.5                     # a genuine shock
    # conservation: the sampled mean is 0.5 up to the jump and grid errors
    assert abs(u.mean() - A) <= 2.0 * B / nx + (1.0 / ny) / t


def test_symmetry_about_the_shock():
    """u - 0.5 is odd about the shock in the moving frame."""
    t, nx, ny = 0.3, 2000, 8192
    xs = 0.5 + 0.5 * t
    s = (np.arange(1, nx) / nx) * 0.4
    y, U = HL.periodic_candidates(ny, A, B)
    ur, _ = HL.hopf_lax(xs + s, y, U, t)
    ul, _ = HL.hopf_lax(xs - s, y, U, t)
    assert np.abs((ur - A) + (ul - A)).max() <= 2.0 * (1.0 / ny) / t


def test_input_generator_matches_the_pinned_primitive():
    """The shared input module's candidates equal the oracle's (whose
    primitive is pinned above to the integral of u0)."""
    from paper_2604_06947_gb300 import inputs as I
    y, U = I.sine_candidates(1000)
    wy, wU = HL.periodic_candidates(1000, I.SINE_MEAN, I.SINE_AMP)
    assert np.array_equal(y, wy)
    assert np.abs(U - wU).max() < 1e-15
