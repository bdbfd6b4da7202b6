"""Level statistics of integer states: the CPU oracle of the entropy
diagnostics of the Supplementary Information (Entropy and Statistical
Structure).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by bench.py's CPU-baseline
leg, never by the library.

Plain numpy, written from the definitions:
  c_k = #{i : q_i = k},  p_k = c_k / N                       eq. pk_definition
  S = -sum_k p_k log p_k  (natural log)                       eq. discrete_entropy
  N_eff = exp(S)                                              eq. neff
  N_{k'k} = #{i : q_i^n = k and q_i^{n+1} = k'}               Definition (level transition)
  M_{k'k} = N_{k'k} / c_k^n  (0 where c_k^n = 0)              eq. empirical_M
  rho = max_{k'} | sum_k M_{k'k} - 1 |                        the row-sum defect

The row-sum defect runs over the occupied levels k' of p^{n+1}: only those
rows of M can be nonzero.  (Over the union of both supports a level that the
step vacates would count as an empty row with defect 1, so even a pure
relabelling of levels would not be a permutation.)  With this reading rho = 0
makes the block of M on rows supp p^{n+1} and columns supp p^n square and
doubly stochastic (its entries sum to the number of columns and to the
number of rows), which is what the appendix's Theorem needs.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Dict, Tuple

import numpy as np


def level_counts(q) -> Tuple[np.ndarray, np.ndarray]:
    """(occupied levels ascending, their counts c_k)."""
    q = np.asarray(q, dtype=np.int64).ravel()
    k, c = np.unique(q, return_counts=True)
    return k.astype(np.int64), c.astype(np.int64)


def entropy(q) -> float:
    """S = -sum p_k log p_k over the occupied levels (eq. discrete_entropy);
    the terms are summed with a correctly rounded sum."""
    q = np.asarray(q, dtype=np.int64).ravel()
    if q.size == 0:
        return 0.0
    _, c = level_counts(q)
    p = c.astype(np.float64) / float(q.size)
    return -math.fsum(float(x) for x in p * np.log(p))


def n_eff(q) -> float:
    """N_eff = exp(S), the effective number of occupied levels (eq. neff)."""
    return math.exp(entropy(q))


def transition_counts(qn, qn1) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The nonzero entries of N^n as (k, k', N_{k'k}), sorted by k then k'."""
    a = np.asarray(qn, dtype=np.int64).ravel()
    b = np.asarray(qn1, dtype=np.int64).ravel()
    if a.shape != b.shape:
        raise ValueError("states of different sizes")
    if a.size == 0:
        e = np.zeros(0, dtype=np.int64)
        return e, e, e
    pairs, cnt = np.unique(np.stack([a, b], axis=1), axis=0, return_counts=True)
    return pairs[:, 0].copy(), pairs[:, 1].copy(), cnt.astype(np.int64)


def row_sums(qn, qn1, exact: bool = False) -> Dict[int, object]:
    """sum_k M_{k'k} for every occupied level k' of p^{n+1}; exact rationals
    with exact=True, else doubles (each N/c rounded once, then a correctly
    rounded sum)."""
    k, kp, cnt = transition_counts(qn, qn1)
    lev, c = level_counts(qn)
    cn = dict(zip(lev.tolist(), c.tolist()))
    terms: Dict[int, list] = {}
    for a, b, m in zip(k.tolist(), kp.tolist(), cnt.tolist()):
        terms.setdefault(b, []).append((m, cn[a]))
    out: Dict[int, object] = {}
    for kp_ in sorted(terms):
        t = terms[kp_]
        if exact:
            out[kp_] = sum((Fraction(m, ck) for m, ck in t), Fraction(0))
        else:
            out[kp_] = math.fsum(m / ck for m, ck in t)
    return out


def row_sum_defect(qn, qn1, exact: bool = False) -> Tuple[object, int]:
    """(rho, the smallest k' attaining it)."""
    r = row_sums(qn, qn1, exact)
    if not r:
        return (Fraction(0) if exact else 0.0), 0
    best, arg = None, None
    for kp_, v in r.items():                 # ascending k'
        d = abs(v - 1)
        if best is None or d > best:
            best, arg = d, kp_
    return best, arg


def stats(qn, qn1) -> dict:
    """Everything one transition reports, for parity with the GPU record."""
    a = np.asarray(qn, dtype=np.int64).ravel()
    b = np.asarray(qn1, dtype=np.int64).ravel()
    rho, arg = row_sum_defect(a, b)
    return {"n_cells": int(a.size),
            "occupied_prev": int(level_counts(a)[0].size),
            "occupied": int(level_counts(b)[0].size),
            "S_prev": entropy(a), "S": entropy(b), "n_eff": n_eff(b),
            "rho": float(rho), "rho_level": int(arg),
            "pairs": int(transition_counts(a, b)[0].size),
            "moved": int(np.count_nonzero(a != b))}
