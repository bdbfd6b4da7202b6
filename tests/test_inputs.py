"""Seeded input generators: determinism, published PRNG outputs, shapes."""
import math

import numpy as np

from paper_2604_06947_gb300 import inputs as I


def test_splitmix64_published_outputs():
    # Reference outputs of SplitMix64 (Steele, Lea & Flood 2014; the public
    # C reference implementation) for seed 0.
    r = I.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_determinism():
    a = I.SplitMix64(7)
    b = I.SplitMix64(7)
    xs = [a.uniform() for _ in range(1000)]
    assert xs == [b.uniform() for _ in range(1000)]
    assert min(xs) >= 0.0 and max(xs) < 1.0
    assert 0.45 < float(np.mean(xs)) < 0.55


def test_square_sine_family():
    p = I.linear_advection_problem()
    assert p.u0.shape == (1024,) and p.dt == 0.5 * p.dx
    x = I.cell_centres(1024)
    inside = (x >= 0.25) & (x < 0.5)
    assert np.allclose(p.u0[inside] - 1.0, 0.25 * np.sin(2 * np.pi * x[inside]))
    assert np.allclose(p.u0[~inside], 0.25 * np.sin(2 * np.pi * x[~inside]))


def test_burgers_family_range():
    p = I.burgers_problem(n=1 << 14)
    assert p.u0.min() >= -0.3 - 1e-12 and p.u0.max() <= 1.3 + 1e-12
    # 16 step positions -> at most 16 jumps of the step part
    smooth = 0.5 + 0.5 * np.sin(2 * np.pi * I.cell_centres(1 << 14))
    s = p.u0 - smooth
    jumps = np.count_nonzero(np.abs(np.diff(np.concatenate([s, s[:1]]))) > 1e-9)
    assert 1 <= jumps <= 16
    assert p.alpha * p.dt / p.dx == np.float64(0.4 * p.dx / 1.3) * 1.3 / p.dx


def test_high_frequency_family():
    n = 1 << 12
    p = I.high_frequency_problem(n=n, steps=10)
    assert p.u0.min() >= 0.0 and p.u0.max() <= 2.0
    # every mode sits in [N/8, N/2-1]: the spectrum has no energy below N/8
    spec = np.abs(np.fft.rfft(p.u0 - 1.0))
    assert spec[: n // 8].max() < 1e-9 * spec.max()
    assert np.count_nonzero(spec > 0.01 * spec.max()) <= 8


def test_sod_initial_state():
    p = I.sod_problem(n=64)
    assert p.U0.shape == (3, 64)
    assert np.all(p.U0[0, :32] == 1.0) and np.all(p.U0[0, 32:] == 0.125)
    assert np.all(p.U0[2, :32] == 2.5) and np.all(p.U0[2, 32:] == 0.25)
    assert p.steps * p.dt == 0.2 or math.isclose(p.steps * p.dt, 0.2, rel_tol=1e-15)


def test_serving_stream_shape():
    reqs = I.serving_stream()
    assert len(reqs) == 4096
    kinds = [r.problem.flux for r in reqs]
    assert kinds.count("linear_upwind") == 2048
    ns = np.array([r.problem.n for r in reqs])
    st = np.array([r.problem.steps for r in reqs])
    assert ns.min() >= 256 and ns.max() <= 1 << 20
    assert st.min() >= 100 and st.max() <= 10_000
    # log-uniform: median near the geometric mean of the range
    assert 0.5 < np.median(ns) / math.sqrt(256 * 2 ** 20) < 2.0
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 1800 < 4096 / t[-1] < 2200          # about 2000 requests/s
