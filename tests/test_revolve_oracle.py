"""Pins of the checkpointing optimum used to judge the product's schedule.

The exhaustive search assumes nothing about the form of an optimal schedule;
the recursive split (first-sweep checkpoints, then binomial reversal) must
agree with it, and its inner reversal cost must equal Griewank's closed form
t L - binom(f + 1 + t, t - 1) (Griewank 1992, "Achieving logarithmic growth of
temporal and spatial complexity in reverse automatic differentiation").
"""
from math import comb

import pytest

from oracle import revolve_dp as R


@pytest.mark.parametrize("s,nmax", [(0, 9), (1, 10), (2, 10), (3, 8)])
def test_recursive_split_matches_exhaustive_search(s, nmax):
    for n in range(1, nmax + 1):
        assert R.min_advances_bruteforce(n, s) == R.min_advances_dp(n, s), (n, s)


def _beta(s, t):
    return comb(s + t, s)


def test_segment_reversal_equals_griewank_closed_form():
    for f in range(0, 7):
        for L in range(1, 200):
            S = f + 1                       # slots including the stored segment start
            t = 0
            while _beta(S, t) < L:
                t += 1
            closed = 0 if L <= 1 else t * L - _beta(S + 1, t - 1)
            assert R._A(L, f) == closed, (L, f)


def test_no_slots_is_quadratic_and_more_slots_never_hurt():
    for n in range(1, 40):
        assert R.min_advances_dp(n, 0) == (n - 1) * (n - 2) // 2
        vals = [R.min_advances_dp(n, s) for s in range(0, 6)]
        assert all(a >= b for a, b in zip(vals, vals[1:]))
