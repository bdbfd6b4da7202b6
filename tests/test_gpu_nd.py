"""Parity of the CUDA d-dimensional step (Theorem, Cartesian extension by
directional composition) with the oracle, bit for bit, on 2-D and 3-D
periodic grids with ragged sizes; exact conservation and the axis-summed
total variation."""
import numpy as np
import pytest

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def solver_for(p, **opt):
    s = F.Solver.for_problem(p, **opt)
    s.set_grid(p.dims)
    return s


def tv_nd(q):
    return int(sum(np.abs(np.roll(q, -1, axis=a) - q).sum() for a in range(q.ndim)))


@pytest.mark.parametrize("dims", [(96, 80), (33, 7), (24, 20, 18), (5, 3, 31)])
def test_burgers_nd_bit_exact(orc, dims):
    p = I.burgers_nd_problem(dims)
    shape = dims[::-1]
    q0 = orc.quantise(p.u0, p.delta).reshape(shape)
    s = solver_for(p).load(q0.reshape(-1))
    q = q0.copy()
    for k in (1, 7, 40):
        s.step(k)
        q = orc.step_nd(q, "burgers_lf", p.delta, p.dx, p.dt, k, alpha=p.alpha)
        assert np.array_equal(s.state().reshape(shape), q), k
    inv = s.invariants()
    assert inv["mass"][0] == int(q0.sum())
    assert inv["tv"][0] == tv_nd(q)
    s.close()


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("k", [1, 3, 4, 7, 8])
def test_every_2d_plan_bit_exact(orc, tile, k):
    """Every register tile and the pipelined walk (6), several K
    (ragged step counts; the walk rounds 7 down to 6), on a ragged grid, a
    grid smaller than one strip and one with a single row."""
    for dims in ((150, 70), (9, 11), (130, 1), (1, 40)):
        p = I.burgers_nd_problem(dims)
        shape = dims[::-1]
        q0 = orc.quantise(p.u0, p.delta).reshape(shape)
        s = solver_for(p, nd_tile=tile, k=k).load(q0.reshape(-1))
        s.step(10)
        want = orc.step_nd(q0, "burgers_lf", p.delta, p.dx, p.dt, 10, alpha=p.alpha)
        assert np.array_equal(s.state().reshape(shape), want), dims
        s.close()


@pytest.mark.parametrize("dims", [(100, 60), (1, 5), (31, 1), (33, 150), (64, 129), (7, 3, 2),
                                  (40, 30, 70), (30, 8, 5), (31, 9, 33), (1, 1, 6), (61, 17, 45),
                                  (2, 50, 300)])
def test_one_step_marching_kernel(orc, dims):
    """The one-step kernels (2-D: warps walk y; 3-D: warps stream z slabs)
    on shapes narrower than a warp, with one row, with several z chunks
    (ragged last chunk), whole and ragged 30-column strips and 8-row blocks."""
    p = I.burgers_nd_problem(dims)
    shape = dims[::-1]
    q0 = orc.quantise(p.u0, p.delta).reshape(shape)
    s = solver_for(p, kernel=1).load(q0.reshape(-1))
    s.step(9)
    want = orc.step_nd(q0, "burgers_lf", p.delta, p.dx, p.dt, 9, alpha=p.alpha)
    assert np.array_equal(s.state().reshape(shape), want)
    s.close()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7])
def test_3d_walk_bit_exact(orc, k):
    """The pipelined 3-D walk (blocks of 16 rows x 64 columns walking z, K
    levels per launch; 7 is taken as 4 + 3) on ragged grids, grids smaller
    than one block in x and y, a single slice and a single row."""
    for dims in ((70, 21, 40), (24, 20, 18), (5, 3, 31), (130, 1, 9), (1, 1, 12), (33, 40, 1)):
        p = I.burgers_nd_problem(dims)
        shape = dims[::-1]
        q0 = orc.quantise(p.u0, p.delta).reshape(shape)
        s = solver_for(p, k=k).load(q0.reshape(-1))
        s.step(11)
        want = orc.step_nd(q0, "burgers_lf", p.delta, p.dx, p.dt, 11, alpha=p.alpha)
        assert np.array_equal(s.state().reshape(shape), want), dims
        s.close()


@pytest.mark.parametrize("opt", [{}, {"pack16": 0}, {"k": 2}, {"k": 2, "pack16": 0}])
def test_3d_walk_evaluators(orc, opt):
    """The 3-D one-step kernel (default) and the walk with the verified closed
    form (upwind, nu = 0.3 per axis) and with the table evaluators
    (Lax-Friedrichs split, 16-bit pack by default on d-D grids, the two-word
    table)."""
    dims = (48, 36, 30)
    shape = dims[::-1]
    p = I.burgers_nd_problem(dims)
    q0 = orc.quantise(p.u0, p.delta).reshape(shape)
    s = solver_for(p, **opt).load(q0.reshape(-1))
    s.step(13)
    want = orc.step_nd(q0, "burgers_lf", p.delta, p.dx, p.dt, 13, alpha=p.alpha)
    assert np.array_equal(s.state().reshape(shape), want)
    s.close()
    p.flux, p.a, p.alpha = "linear_upwind", 1.0, 0.0
    p.dt = 0.3 * p.dx
    s = solver_for(p, **opt).load(q0.reshape(-1))
    s.step(13)
    want = orc.step_nd(q0, "linear_upwind", p.delta, p.dx, p.dt, 13, a=1.0)
    assert np.array_equal(s.state().reshape(shape), want)
    s.close()


@pytest.mark.parametrize("opt", [{}, {"k": 2}])
def test_full_size_3d_grid(orc, opt):
    """160^3 cells, 16 steps (sixteen launches of the default one-step
    kernel, or eight of the walk at K = 2), against the oracle; exact mass."""
    dims = (160, 160, 160)
    shape = dims[::-1]
    p = I.burgers_nd_problem(dims)
    q0 = orc.quantise(p.u0, p.delta).reshape(shape)
    s = solver_for(p, **opt).load(q0.reshape(-1))
    s.step(16)
    want = orc.step_nd(q0, "burgers_lf", p.delta, p.dx, p.dt, 16, alpha=p.alpha)
    assert np.array_equal(s.state().reshape(shape), want)
    assert s.invariants()["mass"][0] == int(q0.sum())
    s.close()


@pytest.mark.parametrize("dims", [(150, 70), (96, 64, 40)])
def test_autotuned_nd_plan_bit_exact(orc, dims):
    """The d-D autotuner's choice (walk depths, in 2-D register tiles, in 3-D
    the one-step kernel, timed at load) gives the oracle's states; an
    explicit K turns it off."""
    p = I.burgers_nd_problem(dims)
    shape = dims[::-1]
    q0 = orc.quantise(p.u0, p.delta).reshape(shape)
    s = solver_for(p, autotune=1).load(q0.reshape(-1))
    st = s.stats()
    assert st["kernel"] in ((1, 5) if len(dims) == 3 else (5, 6)) and st["k"] >= 1
    s.step(13)
    want = orc.step_nd(q0, "burgers_lf", p.delta, p.dx, p.dt, 13, alpha=p.alpha)
    assert np.array_equal(s.state().reshape(shape), want)
    s.close()
    s = solver_for(p, autotune=1, k=3).load(q0.reshape(-1))
    st = s.stats()
    assert st["kernel"] == 5 and st["k"] == 3
    s.close()


def test_linear_upwind_closed_form_2d(orc):
    """Upwind a = 1 at nu = 0.45 per axis (d nu = 0.9): phi+ = R(9 q / 20),
    the verified closed form replaces the table."""
    p = I.burgers_nd_problem((64, 48))
    p.flux, p.a, p.alpha = "linear_upwind", 1.0, 0.0
    p.dt = 0.45 * p.dx
    q0 = orc.quantise(p.u0, p.delta).reshape(48, 64)
    s = solver_for(p).load(q0.reshape(-1))
    s.step(30)
    want = orc.step_nd(q0, "linear_upwind", p.delta, p.dx, p.dt, 30, a=1.0)
    assert np.array_equal(s.state().reshape(48, 64), want)
    s.close()


def test_full_size_2d_grid(orc):
    """2048 x 2048 cells (16 MiB of state), 20 steps, against the oracle."""
    p = I.burgers_nd_problem((2048, 2048))
    q0 = orc.quantise(p.u0, p.delta).reshape(2048, 2048)
    s = solver_for(p).load(q0.reshape(-1))
    s.step(20)
    want = orc.step_nd(q0, "burgers_lf", p.delta, p.dx, p.dt, 20, alpha=p.alpha)
    assert np.array_equal(s.state().reshape(2048, 2048), want)
    assert s.invariants()["mass"][0] == int(q0.sum())
    s.close()


def test_grid_errors():
    p = I.burgers_nd_problem((16, 16))
    s = F.Solver.for_problem(p)
    with pytest.raises(F.FqnmError):
        F.fqnm_set_grid(s.h, (16, 0))
    s.set_grid((16, 16))
    with pytest.raises(F.FqnmError):
        s.load(np.zeros(100, dtype=np.int32))           # not 16 x 16 cells
    s.load(np.zeros(256, dtype=np.int32))
    with pytest.raises(F.FqnmError):
        F.fqnm_set_grid(s.h, (16, 16))                  # after loading
    s.close()
    q = I.burgers_nd_problem((16, 16))
    q.dt = 0.5 * q.dx / q.alpha                          # nu = 0.5 per axis
    s = F.Solver.for_problem(q)
    F.fqnm_set_grid(s.h, (16, 16))                       # d nu = 1: allowed
    s.close()
    q.dt = 0.6 * q.dx / q.alpha
    s = F.Solver.for_problem(q)
    with pytest.raises(F.FqnmError):
        F.fqnm_set_grid(s.h, (16, 16))                   # d nu = 1.2
    s.close()


def test_int32_headroom_scales_with_dimension():
    """One update moves a state by at most 2 d (max|phi+| + max|phi-|), and
    the d-D kernels sum in int32, so the rule build refuses a range closer
    than that to the int32 limits.  Upwind with nu = 0.3 (phi+ = 0.3 q,
    phi- = 0): a constant 8e8-quanta state passes the 1-D bound (1.6 q) but
    not the 3-D one (2.8 q > 2^31); 7e8 passes both, and constant states
    stay constant."""
    p = I.burgers_nd_problem((8, 8, 8))
    p.flux, p.a, p.alpha = "linear_upwind", 1.0, 0.0
    p.dt = 0.3 * p.dx
    big = np.full(p.n, 800_000_000, dtype=np.int32)
    s = F.Solver.for_problem(p)                          # the same cells as a 1-D line
    s.load(big).step(3)
    assert (s.state() == big).all()
    s.close()
    s = solver_for(p)
    with pytest.raises(F.FqnmError) as e:
        s.load(big)
    assert e.value.status == -4
    s.close()
    ok = np.full(p.n, 700_000_000, dtype=np.int32)
    s = solver_for(p).load(ok)
    s.step(3)
    assert (s.state() == ok).all()
    s.close()
