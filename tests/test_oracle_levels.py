"""Pins of the level-statistics oracle (Supplementary Information, Entropy
and Statistical Structure).

Checked against what the definitions and the appendix's results fix without
the oracle's own code: the log-count proposition (uniform occupation of m
levels gives S = log m), a transition worked by hand, the marginal identities
of the count matrix (columns sum to c^n, rows to c^{n+1}), p^{n+1} = M p^n in
exact rationals, the Theorem (a doubly stochastic M never lowers S, and
raises it strictly unless p^{n+1} is a permutation of p^n) over an
exhaustive family of tiny transitions, relabelling and exact-shift special
cases, and agreement with the independent C entropy routine.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import levels as LV
from paper_2604_06947_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
FACTS = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))


def test_log_count_proposition():
    for m in (1, 2, 5, 33):
        q = np.repeat(np.arange(m) * 7 - 3, 13)
        assert abs(LV.entropy(q) - math.log(m)) < 1e-14
        assert abs(LV.n_eff(q) - m) < 1e-12 * m
    assert LV.entropy(np.full(10, 4)) == 0.0


def test_hand_worked_mixing_example():
    ex = FACTS["level_mixing_example"]["value"]
    qn, qn1 = np.array(ex["q_n"]), np.array(ex["q_n1"])
    k, kp, cnt = LV.transition_counts(qn, qn1)
    assert [[a, b, c] for a, b, c in zip(k, kp, cnt)] == ex["transitions"]
    rho, _ = LV.row_sum_defect(qn, qn1, exact=True)
    assert rho == ex["rho"]
    assert abs(LV.entropy(qn) - 1.5 * math.log(2)) < 1e-15
    assert abs(LV.entropy(qn1) - (0.75 * math.log(8 / 3) + 0.5 * math.log(2))) < 1e-15
    assert LV.entropy(qn1) > LV.entropy(qn)


def _check_marginals(qn, qn1):
    k, kp, cnt = LV.transition_counts(qn, qn1)
    lev0, c0 = LV.level_counts(qn)
    lev1, c1 = LV.level_counts(qn1)
    col = {}
    row = {}
    for a, b, m in zip(k.tolist(), kp.tolist(), cnt.tolist()):
        col[a] = col.get(a, 0) + m
        row[b] = row.get(b, 0) + m
    assert col == dict(zip(lev0.tolist(), c0.tolist()))          # sum_k' N_k'k = c_k^n
    assert row == dict(zip(lev1.tolist(), c1.tolist()))          # sum_k N_k'k = c_k'^{n+1}
    # p^{n+1} = M p^n, exactly
    n = len(qn)
    cn = dict(zip(lev0.tolist(), c0.tolist()))
    Mp = {}
    for a, b, m in zip(k.tolist(), kp.tolist(), cnt.tolist()):
        Mp[b] = Mp.get(b, Fraction(0)) + Fraction(m, cn[a]) * Fraction(cn[a], n)
    assert Mp == {b: Fraction(c, n) for b, c in zip(lev1.tolist(), c1.tolist())}


def test_marginals_on_random_and_real_transitions(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(1, 40))
        qn = rng.integers(-3, 4, n)
        qn1 = rng.integers(-3, 4, n)
        _check_marginals(qn, qn1)
    p = I.burgers_problem(n=512)
    q = orc.quantise(p.u0, p.delta)
    for _ in range(3):
        q1 = orc.step(q, "burgers_lf", p.delta, p.dx, p.dt, 1, alpha=p.alpha)
        _check_marginals(q, q1)
        q = orc.step(q1, "burgers_lf", p.delta, p.dx, p.dt, 40, alpha=p.alpha)


def test_theorem_bistochastic_mixing_never_lowers_entropy():
    """Every transition of 6 cells over levels {0, 1, 2} (q^n taken sorted:
    the statistics depend only on the multiset of pairs (q^n_i, q^{n+1}_i)):
    where the exact row-sum defect is 0 (M doubly stochastic), S^{n+1} >= S^n,
    strictly when p^{n+1} is not a permutation of p^n.  Transitions with a
    nonzero defect are not constrained, and some of them lower S."""
    seen_ds = seen_strict = seen_drop = 0
    sources = list(itertools.combinations_with_replacement(range(3), 6))
    targets = list(itertools.product(range(3), repeat=6))
    for a in sources:
        for b in targets:
            qn, qn1 = np.array(a), np.array(b)
            rho, _ = LV.row_sum_defect(qn, qn1, exact=True)
            s0, s1 = LV.entropy(qn), LV.entropy(qn1)
            if rho == 0:
                seen_ds += 1
                assert s1 >= s0 - 1e-15
                perm = sorted(LV.level_counts(qn)[1]) == sorted(LV.level_counts(qn1)[1])
                if not perm:
                    seen_strict += 1
                    assert s1 > s0 + 1e-12
            elif s1 < s0 - 1e-12:
                seen_drop += 1
    assert seen_ds > 100 and seen_strict > 0 and seen_drop > 0


def test_level_relabelling_is_a_permutation_matrix():
    rng = np.random.default_rng(5)
    qn = rng.integers(0, 6, 200)
    relabel = np.array([4, 0, 5, 1, 3, 2]) + 10
    qn1 = relabel[qn]
    rho, _ = LV.row_sum_defect(qn, qn1, exact=True)
    assert rho == 0
    assert abs(LV.entropy(qn1) - LV.entropy(qn)) < 1e-15
    assert LV.transition_counts(qn, qn1)[0].size == np.unique(qn).size


def test_exact_shift_keeps_the_level_distribution(orc):
    """Linear upwind at unit Courant number is the exact shift
    q_i^{n+1} = q_{i-1}^n: the level histogram and S are unchanged, and the
    count matrix is the distribution of neighbouring pairs."""
    p = I.linear_advection_problem()
    q = orc.quantise(p.u0, p.delta)
    q1 = orc.step(q, "linear_upwind", p.delta, p.dx, p.dx, 1, a=1.0)
    assert np.array_equal(q1, np.roll(q, 1))
    assert LV.entropy(q1) == LV.entropy(q)
    k, kp, cnt = LV.transition_counts(q, q1)
    pairs, c = np.unique(np.stack([q, np.roll(q, 1)], axis=1), axis=0, return_counts=True)
    assert np.array_equal(k, pairs[:, 0]) and np.array_equal(kp, pairs[:, 1])
    assert np.array_equal(cnt, c)


def test_double_row_sums_match_exact_ones(orc):
    p = I.burgers_problem(n=2048)
    q = orc.quantise(p.u0, p.delta)
    q = orc.step(q, "burgers_lf", p.delta, p.dx, p.dt, 300, alpha=p.alpha)
    q1 = orc.step(q, "burgers_lf", p.delta, p.dx, p.dt, 1, alpha=p.alpha)
    ex = LV.row_sums(q, q1, exact=True)
    fp = LV.row_sums(q, q1)
    assert ex.keys() == fp.keys()
    for key in ex:
        assert abs(fp[key] - float(ex[key])) <= 2 ** -52 * max(1.0, float(ex[key]))
    rho_e, arg_e = LV.row_sum_defect(q, q1, exact=True)
    rho_f, arg_f = LV.row_sum_defect(q, q1)
    assert abs(rho_f - float(rho_e)) < 1e-15 and 0 < rho_e


def test_entropy_agrees_with_the_c_routine(orc):
    p = I.burgers_problem(n=4096)
    q = orc.quantise(p.u0, p.delta)
    assert abs(LV.entropy(q) - orc.level_entropy(q)) < 1e-12
