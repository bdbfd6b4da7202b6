"""The Hopf-Lax (Lax-Oleinik) entropy solution of inviscid Burgers on a
candidate grid: the accuracy reference of the paper's Burgers test (§3.2,
the dense-grid entropy reference).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by bench.py's CPU-baseline
leg, never by the library.

For u_t + (u^2/2)_x = 0 with u(., 0) = u0 and U0(y) = int_0^y u0,
    u(x, t) = (x - y*) / t,   y* = argmin_y [ U0(y) + (x - y)^2 / (2 t) ].
On a candidate grid y_j the minimisation is taken over the grid, ties to the
smallest j.  The objective is evaluated as U0_j + ((x - y_j) * (x - y_j)) *
inv2t with inv2t = 1 / (2 t), each operation rounded once (numpy does not
contract), so a GPU evaluation in the same order is bit-identical.

For the paper's data u0 = a + b sin(2 pi x) (periodic, mean a):
    U0(y) = a y + b (1 - cos 2 pi y) / (2 pi),
and a period's N_y base points y_j = j / N_y with their images y_j + m,
m in {-1, 0, 1} (U0(y + m) = U0(y) + a m), cover every minimiser for
x in [0, 1) and t (max|u0|) <= 1.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np


def sine_primitive(y, a: float, b: float) -> np.ndarray:
    """U0(y) for u0 = a + b sin(2 pi y)."""
    y = np.asarray(y, dtype=np.float64)
    return a * y + b * (1.0 - np.cos(2.0 * math.pi * y)) / (2.0 * math.pi)


def periodic_candidates(ny: int, a: float, b: float, images=(-1, 0, 1)) -> Tuple[np.ndarray, np.ndarray]:
    """Candidates y and U0(y): N_y base points of one period and their images."""
    base = np.arange(ny, dtype=np.float64) / ny
    U = sine_primitive(base, a, b)
    ys = np.concatenate([base + m for m in images])
    Us = np.concatenate([U + a * m for m in images])
    return ys, Us


def hopf_lax(x, y, U0y, t: float) -> Tuple[np.ndarray, np.ndarray]:
    """(u, argmin index) at the points x from candidates (y, U0(y))."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    U0y = np.asarray(U0y, dtype=np.float64)
    inv2t = 1.0 / (2.0 * t)
    idx = np.empty(x.size, dtype=np.int64)
    for s in range(0, x.size, 256):                # rows in chunks (memory)
        d = x[s:s + 256, None] - y[None, :]
        obj = U0y[None, :] + (d * d) * inv2t
        idx[s:s + 256] = np.argmin(obj, axis=1)    # first minimum: smallest j
    u = (x - y[idx]) / t
    return u, idx


def characteristics(x, t: float, a: float, b: float, tol: float = 1e-15) -> np.ndarray:
    """The smooth solution before the shock forms (t < 1 / (2 pi b)):
    u = u0(x - u t) solved by bisection in u on [a - b, a + b] (the map is
    monotone there while t < t_shock)."""
    x = np.asarray(x, dtype=np.float64)
    lo = np.full(x.shape, a - abs(b))
    hi = np.full(x.shape, a + abs(b))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        g = mid - (a + b * np.sin(2.0 * math.pi * (x - mid * t)))
        lo = np.where(g < 0, mid, lo)
        hi = np.where(g < 0, hi, mid)
        if np.max(hi - lo) < tol:
            break
    return 0.5 * (lo + hi)
