"""Seeded synthetic inputs for the five workloads of the FQNM hot path.

This module is shared by the CUDA path, the oracle, the tests and the bench.
It produces only problem *inputs*: grid geometry, time step, quantum, flux
parameters and the sampled initial field u0(x_i) in float64.  It holds none of
the method's arithmetic: quantisation (eq. quantisation), the transfer maps
(eq. flux_table) and the update (eq. update_rule) are done by each side on its
own.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented here from its
published definition so that every machine draws the same stream.

Grid convention (a reading of §2, where the paper writes x_i = i*dx): cell
centres x_i = (i + 1/2)/N on [0, 1), and u0 is point-sampled at the centres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction
from typing import List, Optional

import numpy as np

MASK64 = (1 << 64) - 1
BASE_SEED = 20260412


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood 2014), 64-bit state."""

    GOLDEN = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive), by scaling a 53-bit draw."""
        span = hi - lo + 1
        return lo + min(int(self.uniform() * span), span - 1)


def cell_centres(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


# ---------------------------------------------------------------------------
# Scalar problem description
# ---------------------------------------------------------------------------

@dataclass
class ScalarProblem:
    """One scalar conservation-law problem: inputs only, no method arithmetic."""

    name: str
    flux: str                 # "linear_upwind" | "linear_lf" | "burgers_lf"
    n: int
    delta: float
    dx: float
    dt: float
    steps: int
    a: float = 0.0            # advection speed (linear fluxes)
    alpha: float = 0.0        # LF dissipation bound (alpha >= max|f'|)
    boundary: str = "periodic"
    u0: Optional[np.ndarray] = field(default=None, repr=False)
    check_every: int = 100


def square_sine_u0(n: int) -> np.ndarray:
    """Square wave of height 1 on [0.25, 0.5) plus 0.25*sin(2*pi*x)."""
    x = cell_centres(n)
    sq = ((x >= 0.25) & (x < 0.5)).astype(np.float64)
    return sq + 0.25 * np.sin(2.0 * math.pi * x)


def burgers_steps_u0(n: int, seed: int, n_steps_pos: int = 16,
                     amp: float = 0.3) -> np.ndarray:
    """0.5 + 0.5*sin(2*pi*x) plus a seeded periodic step function.

    Reading of "random steps of amplitude <= 0.3 at 16 random positions":
    16 breakpoints b_j ~ U[0,1) (sorted) and 16 levels s_j ~ U[-amp, amp];
    s(x) = s_j on [b_j, b_{j+1}), wrapping periodically so that x < b_0 takes
    the last level.  The field stays in [-0.3, 1.3].
    """
    rng = SplitMix64(seed)
    b = sorted(rng.uniform() for _ in range(n_steps_pos))
    s = [amp * (2.0 * rng.uniform() - 1.0) for _ in range(n_steps_pos)]
    x = cell_centres(n)
    idx = np.searchsorted(np.asarray(b), x, side="right") - 1   # -1 => wrap
    steps = np.asarray(s)[idx]                                   # idx -1 -> last
    return 0.5 + 0.5 * np.sin(2.0 * math.pi * x) + steps


def high_frequency_u0(n: int, seed: int, n_modes: int = 8) -> np.ndarray:
    """1 + sum of 8 sines, amplitude 1/8, integer wavenumbers in [N/8, N/2-1].

    The phase 2*pi*k*x_i is reduced exactly in integers:
    k*x_i = k*(2i+1)/(2N), so the angle is 2*pi*((k*(2i+1)) mod 2N)/(2N).
    """
    rng = SplitMix64(seed)
    ks = [rng.randint(n // 8, n // 2 - 1) for _ in range(n_modes)]
    phases = [2.0 * math.pi * rng.uniform() for _ in range(n_modes)]
    i2p1 = 2 * np.arange(n, dtype=np.int64) + 1
    u = np.ones(n, dtype=np.float64)
    for k, ph in zip(ks, phases):
        r = (np.int64(k) * i2p1) % (2 * n)
        u += 0.125 * np.sin(2.0 * math.pi * (r.astype(np.float64) / (2 * n)) + ph)
    return u


def linear_advection_problem(n: int = 1024, delta: float = 2.0 ** -12,
                             courant: float = 0.5, steps: int = 2000,
                             with_u0: bool = True) -> ScalarProblem:
    """u_t + u_x = 0 on [0,1), periodic, square wave + sine (upwind split)."""
    dx = 1.0 / n
    dt = courant * dx / 1.0
    p = ScalarProblem("linear_advection_square_sine", "linear_upwind", n, delta,
                      dx, dt, steps, a=1.0)
    if with_u0:
        p.u0 = square_sine_u0(n)
    return p


BURGERS_ALPHA = 1.3   # a-priori bound of max|f'(u)| = max|u| over [-0.3, 1.3]


def burgers_problem(n: int = 1 << 20, delta: float = 2.0 ** -16,
                    courant: float = 0.4, steps: int = 10_000,
                    seed: int = BASE_SEED + 1,
                    with_u0: bool = True) -> ScalarProblem:
    """Inviscid Burgers, LF split with alpha = 1.3, periodic, seeded steps."""
    dx = 1.0 / n
    dt = courant * dx / BURGERS_ALPHA
    p = ScalarProblem("burgers_lf_steps", "burgers_lf", n, delta, dx, dt,
                      steps, alpha=BURGERS_ALPHA)
    if with_u0:
        p.u0 = burgers_steps_u0(n, seed)
    return p


# The paper's Burgers test (§3.2): u0 = 0.5 + sin(2 pi x), past the shock
# time 1/(2 pi); a fixed dt that lands on t_end exactly.
SINE_MEAN, SINE_AMP = 0.5, 1.0
SINE_ALPHA = SINE_MEAN + SINE_AMP      # max |f'| = max |u0| (the range only shrinks)


def burgers_sine_problem(n: int = 128, delta: float = 2.0 ** -16, t_end: float = 0.3,
                         courant: float = 0.4) -> ScalarProblem:
    """Inviscid Burgers, LF split with alpha = max|u0| = 1.5, periodic,
    u0 = 0.5 + sin(2 pi x) at the cell centres, steps = ceil(t_end / dt0)
    with dt0 = courant dx / alpha, then dt = t_end / steps."""
    dx = 1.0 / n
    steps = int(np.ceil(t_end / (courant * dx / SINE_ALPHA)))
    dt = t_end / steps
    p = ScalarProblem("burgers_sine", "burgers_lf", n, delta, dx, dt, steps,
                      alpha=SINE_ALPHA)
    p.u0 = SINE_MEAN + SINE_AMP * np.sin(2.0 * np.pi * cell_centres(n))
    return p


def sine_candidates(ny: int, images=(-1, 0, 1)):
    """Candidates (y, U0(y)) of the Hopf-Lax reference for u0 = 0.5 + sin(2 pi x):
    ny points y_j = j / ny of one period and their periodic images y_j + m,
    with the primitive U0(y) = 0.5 y + (1 - cos 2 pi y) / (2 pi) (input data:
    the integral of the initial field)."""
    base = np.arange(ny, dtype=np.float64) / ny
    U = SINE_MEAN * base + SINE_AMP * (1.0 - np.cos(2.0 * np.pi * base)) / (2.0 * np.pi)
    y = np.concatenate([base + m for m in images])
    U0 = np.concatenate([U + SINE_MEAN * m for m in images])
    return y, U0


def burgers_nd_problem(dims=(1024, 1024), delta: float = 2.0 ** -16, courant: float = 0.4,
                       steps: int = 1000, seed: int = BASE_SEED + 5) -> ScalarProblem:
    """Burgers on a periodic d-dimensional grid (dims x-fastest), LF with
    alpha = 1.3 on every axis, d * nu = courant: u0 = 0.5 + 0.5 prod_m
    sin(2 pi (x_m + phase_m)) + seeded steps along x (the one-dimensional
    Burgers family's 16 random levels), so u0 lies in [-0.3, 1.3].
    p.u0 is flat, x fastest; p.dims holds the shape."""
    d = len(dims)
    nx = dims[0]
    dx = 1.0 / nx
    dt = courant / d * dx / BURGERS_ALPHA
    n = int(np.prod(dims))
    p = ScalarProblem("burgers_%dd" % d, "burgers_lf", n, delta, dx, dt, steps,
                      alpha=BURGERS_ALPHA)
    rng = SplitMix64(seed)
    phases = [rng.uniform() for _ in range(d)]
    axes = [(np.arange(m) + 0.5) / m for m in dims]
    grids = np.meshgrid(*axes[::-1], indexing="ij")          # (.., y, x)
    prod = np.ones(grids[0].shape)
    for m in range(d):
        prod = prod * np.sin(2.0 * np.pi * (grids[d - 1 - m] + phases[m]))
    steps_x = burgers_steps_u0(nx, seed + 1) - (0.5 + 0.5 * np.sin(2.0 * np.pi * axes[0]))
    u0 = 0.5 + 0.5 * prod + 0.3 * np.clip(steps_x / 0.3, -1.0, 1.0)
    p.u0 = np.clip(u0, -0.3, 1.3).reshape(-1)
    p.dims = tuple(dims)
    return p


def high_frequency_problem(n: int = 1 << 24, delta: float = 2.0 ** -20,
                           courant: float = 0.9, steps: int = 2000,
                           seed: int = BASE_SEED + 2,
                           with_u0: bool = True) -> ScalarProblem:
    """Periodic advection near Nyquist: 8 high-wavenumber sines, upwind."""
    dx = 1.0 / n
    dt = courant * dx / 1.0
    p = ScalarProblem("high_frequency_transport", "linear_upwind", n, delta,
                      dx, dt, steps, a=1.0)
    if with_u0:
        p.u0 = high_frequency_u0(n, seed)
    return p


# ---------------------------------------------------------------------------
# Sod shock tube (1-D Euler)
# ---------------------------------------------------------------------------

SOD_GAMMA = 1.4
SOD_LEFT = (1.0, 0.0, 1.0)      # rho, u, p
SOD_RIGHT = (0.125, 0.0, 0.1)
SOD_T_END = 0.2
SOD_SMAX = 2.2                  # a-priori bound of |u|+c over the Sod solution


@dataclass
class EulerProblem:
    name: str
    n: int
    gamma: float
    delta: tuple
    dx: float
    dt: float
    steps: int
    t_end: float
    x0: float = 0.5
    U0: Optional[np.ndarray] = field(default=None, repr=False)  # (3, n) float64


def sod_problem(n: int = 1 << 16, courant: float = 0.5,
                delta: float = 2.0 ** -32, with_u0: bool = True,
                steps: Optional[int] = None) -> EulerProblem:
    """Sod tube on [0,1), transmissive ends, run to t = 0.2 with fixed dt.

    Reading: dt = 0.2/n_steps with n_steps = ceil(0.2*S/(courant*dx)) and
    S = 2.2 >= max(|u|+c) of the exact solution, so t = 0.2 is hit exactly.
    Conserved variables are (rho, m = rho*u, E = p/(gamma-1) + rho*u^2/2).
    """
    dx = 1.0 / n
    n_steps = int(math.ceil(SOD_T_END * SOD_SMAX / (courant * dx)))
    dt = SOD_T_END / n_steps
    p = EulerProblem("sod", n, SOD_GAMMA, (delta, delta, delta), dx, dt,
                     n_steps if steps is None else steps, SOD_T_END)
    if with_u0:
        x = cell_centres(n)
        left = x < p.x0
        U = np.empty((3, n), dtype=np.float64)
        # E = p/(gamma-1) + rho*u^2/2 in exact rationals (gamma = 7/5), then
        # rounded once, so that E_L = 2.5 and E_R = 0.25 exactly.
        gm1 = Fraction(SOD_GAMMA).limit_denominator(1000) - 1
        for side, (rho, u, pr) in ((left, SOD_LEFT), (~left, SOD_RIGHT)):
            U[0, side] = rho
            U[1, side] = rho * u
            U[2, side] = float(Fraction(pr) / gm1
                               + Fraction(1, 2) * Fraction(rho) * Fraction(u) ** 2)
        p.U0 = U
    return p


# ---------------------------------------------------------------------------
# Batched serving stream
# ---------------------------------------------------------------------------

@dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    problem: ScalarProblem
    data_seed: int


def serving_stream(n_requests: int = 4096, rate_hz: float = 2000.0,
                   n_min: int = 256, n_max: int = 1 << 20,
                   steps_min: int = 100, steps_max: int = 10_000,
                   delta: float = 2.0 ** -16, seed: int = BASE_SEED + 4,
                   with_u0: bool = False) -> List[ServeRequest]:
    """Independent problems with Poisson arrivals (exponential gaps).

    Half are linear advection (square wave + sine family, upwind, Courant
    0.5) and half Burgers (seeded-steps family, LF, Courant 0.4); the kinds
    are a seeded shuffle of an exact half/half split.  Grid sizes and step
    counts are log-uniform (rounded to integers) in the stated ranges.
    """
    rng = SplitMix64(seed)
    kinds = [0] * (n_requests // 2) + [1] * (n_requests - n_requests // 2)
    for i in range(n_requests - 1, 0, -1):          # Fisher-Yates
        j = rng.randint(0, i)
        kinds[i], kinds[j] = kinds[j], kinds[i]
    t = 0.0
    reqs = []
    ln_n = (math.log(n_min), math.log(n_max))
    ln_s = (math.log(steps_min), math.log(steps_max))
    for r in range(n_requests):
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        n = int(round(math.exp(ln_n[0] + rng.uniform() * (ln_n[1] - ln_n[0]))))
        n = min(max(n, n_min), n_max)
        st = int(round(math.exp(ln_s[0] + rng.uniform() * (ln_s[1] - ln_s[0]))))
        st = min(max(st, steps_min), steps_max)
        dseed = rng.next_u64()
        if kinds[r] == 0:
            p = linear_advection_problem(n, delta, 0.5, st, with_u0=False)
        else:
            p = burgers_problem(n, delta, 0.4, st, seed=dseed, with_u0=False)
        reqs.append(ServeRequest(r, t, p, dseed))
    if with_u0:
        for rq in reqs:
            materialise(rq)
    return reqs


def materialise(rq: ServeRequest) -> ScalarProblem:
    """Fill in u0 for a serving request (kept lazy: the stream is large)."""
    p = rq.problem
    if p.u0 is None:
        if p.flux == "linear_upwind":
            p.u0 = square_sine_u0(p.n)
        else:
            p.u0 = burgers_steps_u0(p.n, rq.data_seed)
    return p


WORKLOADS = {
    "linear_advection_1k": linear_advection_problem,
    "burgers_1m": burgers_problem,
    "high_frequency_16m": high_frequency_problem,
}
