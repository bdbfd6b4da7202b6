"""Parity of the CUDA Euler/Roe integer path and the FP finite-volume
baselines with the oracle."""
import numpy as np
import pytest

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

pytestmark = pytest.mark.gpu
G = I.SOD_GAMMA


def sod_q0(p):
    return np.stack([F.fqnm_quantise(p.U0[k], p.delta[k], state_bits=64) for k in range(3)])


def euler_solver(p):
    s = F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                 "transmissive")
    return s


def test_sod_quantised_initial_state_is_exact(orc):
    p = I.sod_problem(n=1024)
    q0 = sod_q0(p)
    for k in range(3):
        assert np.array_equal(q0[k], orc.quantise(p.U0[k], p.delta[k]))
    assert q0[0, 0] == 2 ** 32 and q0[2, 0] == 10 * 2 ** 30 and q0[2, -1] == 2 ** 30


@pytest.mark.parametrize("n", [1000, 1 << 12])
def test_sod_full_run_bit_exact(orc, n):
    """Componentwise-quantised Roe transfer to t = 0.2, checked every 200
    steps against the oracle, with exact boundary-flux accounting."""
    p = I.sod_problem(n=n)
    q0 = sod_q0(p)
    s = euler_solver(p).load(q0)
    q = q0.copy()
    bf_total = np.zeros(3, dtype=np.int64)
    done = 0
    while done < p.steps:
        k = min(200, p.steps - done)
        s.step(k)
        q, bf = orc.euler_step(q, p.gamma, p.delta, p.dx, p.dt, k)
        bf_total += bf
        done += k
        assert np.array_equal(s.state(), q), done
    inv = s.invariants()
    for k in range(3):
        assert inv["boundary_flux"][k] == bf_total[k]
        assert inv["mass"][k] == int(q0[k].sum()) - int(bf_total[k])
    s.close()


def test_sod_65k_first_2000_steps_bit_exact(orc):
    p = I.sod_problem(n=1 << 16)
    q0 = sod_q0(p)
    s = euler_solver(p).load(q0)
    q = q0.copy()
    for _ in range(4):
        s.step(500)
        q, _ = orc.euler_step(q, p.gamma, p.delta, p.dx, p.dt, 500)
        assert np.array_equal(s.state(), q)
    s.close()


def test_sod_65k_full_run_density_error_and_conservation(orc):
    """Full run to t = 0.2 at 2^16 cells (57,672 steps): beyond the oracle's
    2000-step parity window, check exact conservation with boundary
    accounting, the density error against the exact Riemann solution, and
    the shock in the paper's window."""
    p = I.sod_problem(n=1 << 16)
    q0 = sod_q0(p)
    s = euler_solver(p).load(q0)
    s.step(p.steps)
    u = s.observe()
    inv = s.invariants()
    for k in range(3):
        assert inv["mass"][k] == int(q0[k].sum()) - inv["boundary_flux"][k]
    x = I.cell_centres(p.n)
    rex, _, pex = orc.riemann_sample(G, I.SOD_LEFT, I.SOD_RIGHT, 0.5, 0.2, x)
    l1 = p.dx * np.abs(u[0] - rex).sum()
    assert l1 < 2e-3
    rho = u[0]
    shock = x[np.argmax(rho < 0.5 * (0.125 + 0.2655737))]
    assert 0.84 < shock < 0.86
    s.close()


# ---------------------------------------------------------------------------
# floating-point finite-volume baselines
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,a,alpha", [("burgers_lf", 0.0, 1.3), ("linear_upwind", 1.0, 0.0)])
@pytest.mark.parametrize("boundary", ["periodic", "transmissive"])
def test_fv64_bitwise_equal_to_cpu(orc, kind, a, alpha, boundary):
    p = I.burgers_problem(n=7777, steps=0)
    u0 = p.delta * orc.quantise(p.u0, p.delta).astype(np.float64)
    h = F.fqnm_fv_create(F.make_flux(kind, a=a, alpha=alpha), p.dx, p.dt, boundary, 64)
    F.fqnm_fv_load(h, u0)
    F.fqnm_fv_step(h, 300)
    got = F.fqnm_fv_observe(h, p.n)
    want = orc.fv_step(u0, kind, p.dx, p.dt, 300, a=a, alpha=alpha, boundary=boundary)
    assert np.array_equal(got, want)
    F.fqnm_fv_destroy(h)


@pytest.mark.parametrize("kind,a,alpha", [("burgers_lf", 0.0, 1.3), ("linear_upwind", 1.0, 0.0)])
def test_fv32_matches_cpu_and_fv64(orc, kind, a, alpha):
    p = I.burgers_problem(n=7777, steps=0)
    u0 = p.delta * orc.quantise(p.u0, p.delta).astype(np.float64)
    h = F.fqnm_fv_create(F.make_flux(kind, a=a, alpha=alpha), p.dx, p.dt, "periodic", 32)
    F.fqnm_fv_load(h, u0)
    F.fqnm_fv_step(h, 300)
    got = F.fqnm_fv_observe(h, p.n)
    want32 = orc.fv_step(u0, kind, p.dx, p.dt, 300, a=a, alpha=alpha, precision="f32")
    assert np.array_equal(got, want32.astype(np.float64))
    want64 = orc.fv_step(u0, kind, p.dx, p.dt, 300, a=a, alpha=alpha)
    rel = np.abs(got - want64).sum() / np.abs(want64).sum()
    assert rel <= 1e-5
    F.fqnm_fv_destroy(h)


def test_euler_fv64_bitwise_equal_to_cpu(orc):
    p = I.sod_problem(n=2000)
    h = F.fqnm_fv_create(F.make_flux("euler_roe", gamma=G), p.dx, p.dt, "transmissive", 64)
    F.fqnm_fv_load(h, p.U0)
    F.fqnm_fv_step(h, 400)
    got = F.fqnm_fv_observe(h, p.n, 3)
    want = orc.euler_fv_step(p.U0, G, p.dx, p.dt, 400)
    assert np.array_equal(got, want)
    F.fqnm_fv_destroy(h)
