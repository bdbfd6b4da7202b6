"""Parity of the CUDA Hopf-Lax entropy reference with the oracle, and the
convergence of the GPU solver to it as delta/dx -> 0 (§2.3 consistency and
convergence; the Burgers test of §3.2).

The Hopf-Lax argmin indices are integers taken from doubles evaluated in the
same operation order on both sides, so they and u are compared bit for bit.
"""
import math

import numpy as np
import pytest

from oracle import hopf_lax as HL
from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_paper_configuration_bit_exact():
    """N_x = 128 grid points, N_y = 2048 candidates per period, t = 0.3."""
    x = I.cell_centres(128)
    y, U = I.sine_candidates(2048)
    u, idx = F.fqnm_hopf_lax(x, y, U, 0.3)
    wu, widx = HL.hopf_lax(x, y, U, 0.3)
    assert np.array_equal(idx, widx) and np.array_equal(u, wu)


@pytest.mark.parametrize("nx,ny,t", [(1, 1, 0.1), (3, 5, 0.2), (1003, 777, 0.2),
                                     (4099, 3000, 0.45)])
def test_ragged_sizes_bit_exact(nx, ny, t):
    x = np.linspace(-0.1, 1.1, nx)
    y, U = I.sine_candidates(ny)
    u, idx = F.fqnm_hopf_lax(x, y, U, t)
    wu, widx = HL.hopf_lax(x, y, U, t)
    assert np.array_equal(idx, widx) and np.array_equal(u, wu)


def test_ties_go_to_the_smallest_index_and_nan_candidates():
    y = np.array([0.0, 0.25, 0.25, 0.5, 0.5])
    U = np.zeros(5)
    x = np.array([0.25, 0.5, 0.375])
    u, idx = F.fqnm_hopf_lax(x, y, U, 1.0)
    assert list(idx) == [1, 3, 1]                  # 0.375: equidistant from 0.25 and 0.5
    u, idx = F.fqnm_hopf_lax(np.array([0.1]), np.array([0.0]), np.array([np.nan]), 1.0)
    assert idx[0] == -1 and np.isnan(u[0])
    # infinities and NaN among finite candidates: NaN is never the minimum,
    # -inf always is, +inf only loses
    y = np.array([0.0, 0.1, 0.2, 0.3])
    for U, want in (([np.nan, 1.0, 2.0, np.inf], 1), ([1.0, -np.inf, np.nan, 0.5], 1),
                    ([np.inf, np.inf, np.nan, np.nan], -1), ([-0.0, 0.0, 0.0, 1.0], 0)):
        u, idx = F.fqnm_hopf_lax(np.array([0.0]), y, np.array(U), 1e6)
        assert idx[0] == want, U


def test_ties_across_candidate_chunks():
    """The candidates listed twice (40,000 entries, split into many chunks):
    every minimum occurs in two chunks, and the first copy's index wins, as
    in the oracle's single scan."""
    y1, U1 = I.sine_candidates(20000 // 3)
    y = np.concatenate([y1, y1])
    U = np.concatenate([U1, U1])
    x = np.linspace(0.0, 1.0, 67)
    u, idx = F.fqnm_hopf_lax(x, y, U, 0.3)
    wu, widx = HL.hopf_lax(x, y, U, 0.3)
    assert np.array_equal(idx, widx) and np.array_equal(u, wu)
    assert (idx < y1.size).all()


def test_device_variant_dense_grid_sampled():
    """Device arrays on a torch stream at 2^14 points x 3 * 2^16 candidates;
    512 sampled rows against the oracle."""
    torch = pytest.importorskip("torch")
    nx = 1 << 14
    x = I.cell_centres(nx)
    y, U = I.sine_candidates(1 << 16)
    dx_, dy, dU = (torch.from_numpy(a).cuda() for a in (x, y, U))
    du = torch.empty(nx, dtype=torch.float64, device="cuda")
    di = torch.empty(nx, dtype=torch.int64, device="cuda")
    st = torch.cuda.Stream()
    F.fqnm_hopf_lax(dx_, dy, dU, 0.3, nx=nx, ny=y.size, u=du, idx=di, stream=st)
    st.synchronize()
    rows = np.random.default_rng(0).choice(nx, 512, replace=False)
    wu, widx = HL.hopf_lax(x[rows], y, U, 0.3)
    assert np.array_equal(di.cpu().numpy()[rows], widx)
    assert np.array_equal(du.cpu().numpy()[rows], wu)


def test_errors():
    with pytest.raises(F.FqnmError):
        F.fqnm_hopf_lax(np.zeros(3), np.zeros(2), np.zeros(2), 0.0)
    with pytest.raises(F.FqnmError):
        F.fqnm_hopf_lax(np.zeros(0), np.zeros(2), np.zeros(2), 0.3)
    with pytest.raises(ValueError):
        F.fqnm_hopf_lax(np.zeros(3), np.zeros(2), np.zeros(3), 0.3)


def sweep_delta(k: int) -> float:
    return 2.0 ** -math.ceil(1.5 * k)               # delta / dx = dx^(1/2) -> 0


def test_convergence_to_the_entropy_solution(orc):
    """The paper's Burgers data to t = 0.3 (past the shock time 1/(2 pi)) on
    N = 2^7 .. 2^13 cells with delta = dx^(3/2): the GPU states equal the
    oracle's, the integer mass is exactly conserved, and the L1 distance to
    the Hopf-Lax solution falls at first order (a monotone conservative
    scheme converging to the entropy solution)."""
    errs = []
    for k in range(7, 14):
        n = 1 << k
        p = I.burgers_sine_problem(n=n, delta=sweep_delta(k))
        q0 = orc.quantise(p.u0, p.delta)
        s = F.Solver.for_problem(p).load(q0)
        s.step(p.steps)
        q = s.state()
        assert np.array_equal(q, orc.step(q0, "burgers_lf", p.delta, p.dx, p.dt, p.steps,
                                          alpha=p.alpha))
        assert int(q.astype(np.int64).sum()) == int(q0.sum())
        y, U = I.sine_candidates(16 * n)
        ue, _ = F.fqnm_hopf_lax(I.cell_centres(n), y, U, 0.3)
        errs.append(p.dx * np.abs(p.delta * q - ue).sum())
        s.close()
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.85) and np.all(rates < 1.2), rates
    assert errs[0] < 0.03
