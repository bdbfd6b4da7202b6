"""The integer-pipe IEEE double steps of the integer Roe step (FQNM_OPT_FP64)
against the GPU's FP64 instructions, bit for bit, on operands drawn to reach
every branch: random exponents and fractions, fractions of all zeros and all
ones, quotients and roots that land on exact values, integers at rounding
ties, zeros, subnormals, infinities and NaN (where the FP64 instruction takes
over).  And the Roe step in every FP64 mode against the oracle."""
import numpy as np
import pytest

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MASK52 = (1 << 52) - 1


def doubles(rng, n, e_lo=1, e_hi=2046, neg=True):
    sign = (rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)) if neg else 0
    e = rng.integers(e_lo, e_hi + 1, n, dtype=np.uint64) << np.uint64(52)
    f = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    # a fifth of the fractions all zeros or all ones, or one unit from them
    k = rng.integers(0, 10, n)
    f = np.where(k == 0, 0, f)
    f = np.where(k == 1, MASK52, f)
    f = np.where(k == 2, 1, f)
    f = np.where(k == 3, MASK52 - 1, f).astype(np.uint64)
    return (sign | e | f).view(np.float64)


def specials():
    v = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
         2.225073858507201e-308, 1.7976931348623157e308, 1.0, -1.0, 2.0, 0.5, 3.0, 1e-300,
         1e300]
    return np.array(v, dtype=np.float64)


def run(op, a, b, rounding="half_even"):
    import torch
    n = a.size
    da = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    db = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    oi = torch.empty(n, dtype=torch.int64, device="cuda")
    of = torch.empty(n, dtype=torch.int64, device="cuda")
    op_ = torch.empty(n, dtype=torch.int32, device="cuda")
    F.fqnm_fp64_check(op, da, db, n, oi, of, op_, rounding=rounding)
    torch.cuda.synchronize()
    return oi.cpu().numpy(), of.cpu().numpy(), op_.cpu().numpy()


def assert_same(got, want, a, b=None):
    bad = np.flatnonzero(got != want)
    if bad.size:
        i = bad[0]
        raise AssertionError("%d of %d differ; first a=%r b=%r int=%x fp64=%x"
                             % (bad.size, got.size, a[i], None if b is None else b[i],
                                got[i] & 0xffffffffffffffff, want[i] & 0xffffffffffffffff))


def test_division_matches_fp64():
    rng = np.random.default_rng(101)
    n = 1 << 22
    # quotients across the whole exponent range, and near its ends
    a = doubles(rng, n)
    b = doubles(rng, n)
    near = doubles(rng, n, 900, 1150)
    b2 = doubles(rng, n, 900, 1150)
    s = specials()
    sa, sb = np.meshgrid(s, s)
    A = np.concatenate([a, near, sa.ravel(), np.zeros(64), doubles(rng, 64)])
    B = np.concatenate([b, b2, sb.ravel(), doubles(rng, 64), np.zeros(64)])
    # quotients that are exact: (q * b) / b with a short q
    q = rng.integers(1, 1 << 20, 1 << 16).astype(np.float64)
    bb = doubles(rng, 1 << 16, 1000, 1040)
    A = np.concatenate([A, q * bb])
    B = np.concatenate([B, bb])
    gi, gf, path = run(0, A, B)
    assert_same(gi, gf, A, B)
    assert (path[: 2 * n] & 1).mean() > 0.7          # the integer path carries most
    assert (path[2 * n:] & 1).sum() > 0


def test_square_root_matches_fp64():
    rng = np.random.default_rng(102)
    n = 1 << 22
    a = doubles(rng, n, neg=False)
    r = rng.integers(1, 1 << 26, 1 << 18).astype(np.float64)
    sq = r * r                                          # exact squares, exact roots
    s = specials()
    ulp = np.concatenate([np.nextafter(sq, np.inf), np.nextafter(sq, 0)])
    A = np.concatenate([a, sq, ulp, s, -np.abs(doubles(rng, 64))])
    gi, gf, path = run(1, A, np.zeros_like(A))
    assert_same(gi, gf, A)
    assert (path[:n] & 1).all()                         # every positive normal
    assert (path[n: n + sq.size] & 1).all()


def test_scaled_int64_conversion_matches_fp64():
    rng = np.random.default_rng(103)
    n = 1 << 20
    q = rng.integers(-(1 << 62), 1 << 62, n, dtype=np.int64)
    small = rng.integers(-(1 << 40), 1 << 40, n, dtype=np.int64)
    # beyond 2^53: ties of the conversion (low bits exactly half an ulp)
    big = (rng.integers(1 << 53, 1 << 62, n // 4, dtype=np.int64) >> 11 << 11) | (1 << 10)
    edge = np.array([0, 1, -1, (1 << 63) - 1, -(1 << 63), 1 << 53, (1 << 53) + 1,
                     -(1 << 53) - 1], dtype=np.int64)
    Q = np.concatenate([q, small, big, -big, edge])
    e = rng.integers(-60, 61, Q.size).astype(np.float64)
    e[: n] = -32.0
    gi, gf, _ = run(2, Q.view(np.float64), e)
    assert_same(gi, gf, Q, e)


@pytest.mark.parametrize("rounding", ["half_even", "half_away", "floor"])
def test_scaled_rounding_matches_fp64(rounding):
    rng = np.random.default_rng(104)
    n = 1 << 20
    y = doubles(rng, n, 980, 1080)                       # |y| 2^32 around the integers
    ties = (rng.integers(-(1 << 40), 1 << 40, n) + 0.5) * 2.0 ** -32
    ints = rng.integers(-(1 << 40), 1 << 40, n) * 2.0 ** -32
    tiny = doubles(rng, 4096, 1, 990)
    huge = doubles(rng, 4096, 1050, 2046)
    Y = np.concatenate([y, ties, ints, tiny, huge, specials()])
    e = np.full(Y.size, 32.0)
    e[-4096 - 17: -17] = rng.integers(0, 80, 4096)
    gi, gf, path = run(3, Y, e, rounding=rounding)
    assert_same(gi, gf, Y, e)
    assert np.array_equal((path >> 1) & 1, (path >> 2) & 1)   # out of range alike


def test_multiplication_matches_fp64():
    rng = np.random.default_rng(106)
    n = 1 << 22
    a = doubles(rng, n)
    b = doubles(rng, n)
    near_a = doubles(rng, n, 800, 1250)
    near_b = doubles(rng, n, 800, 1250)
    # products with few significant bits (exact) and at rounding ties:
    # (2^26 + odd)^2 has its discarded half exactly at the rounding bit
    x = (rng.integers(1 << 26, 1 << 27, 1 << 16) | 1).astype(np.float64)
    s = specials()
    sa, sb = np.meshgrid(s, s)
    A = np.concatenate([a, near_a, x, x * 3.0, sa.ravel(), np.zeros(64)])
    B = np.concatenate([b, near_b, x, x, sb.ravel(), doubles(rng, 64)])
    gi, gf, path = run(5, A, B)
    assert_same(gi, gf, A, B)
    assert (path[n: 2 * n] & 1).all()


def test_halving_and_doubling_match_fp64():
    rng = np.random.default_rng(105)
    n = 1 << 20
    x = np.concatenate([doubles(rng, n), doubles(rng, 4096, 1, 3), doubles(rng, 4096, 2044, 2046),
                        specials()])
    for k in (-1.0, 1.0):
        gi, gf, path = run(4, x, np.full(x.size, k))
        assert_same(gi, gf, x)
        assert (path[:n] & 1).mean() > 0.99


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("mask", [7, 1])
def test_roe_step_every_fp64_mode_matches_oracle(orc, mode, mask):
    """A Sod tube (and the density-only variant) for 300 steps in each FP64
    mode: the same states as the oracle."""
    p = I.sod_problem(n=4096)
    q0 = np.stack([orc.quantise(p.U0[k], p.delta[k]) for k in range(3)]).astype(np.int64)
    s = F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                 "transmissive", quantise_mask=mask, fp64=mode)
    if mask == 7:
        s.load(q0).step(300)
        want, _ = orc.euler_step(q0, p.gamma, p.delta, p.dx, p.dt, 300)
        assert np.array_equal(s.state().reshape(3, -1), want)
    else:
        s.load_field(np.stack(p.U0)).step(300)
        uf = np.array(p.U0, dtype=np.float64)
        wq, wu, _ = orc.euler_step_mask(q0, uf, mask, p.gamma, p.delta, p.dx, p.dt, 300)
        got = s.state().reshape(3, -1)
        assert np.array_equal(got[0], wq[0])
        assert np.array_equal(got[1:], wu[1:].view(np.int64))
    s.close()
