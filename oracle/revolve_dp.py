"""Optimal-recomputation counts for wavefield checkpointing, by exhaustive search.

TEST INFRASTRUCTURE ONLY (used by tests/test_revolve.py to pin the product's
binomial checkpoint schedule).

Model of the reversal (the adjoint sweep of the Hessian apply, paper section 3,
reverses the forward time loop):

* the forward state after step i is x_i = (u^i, u^{i-1}); x_0 = 0 is free;
* the adjoint of time step i needs x_i as the current state;
* the first (forward) sweep visits x_1 .. x_{n-1} in order and may store up to
  ``s`` of them in snapshot slots; it ends holding x_{n-1};
* afterwards, restoring a stored state (or x_0) is free, storing the current
  state into a slot is free, and every forward advance x_j -> x_{j+1} costs 1.

``min_advances_bruteforce`` searches all strategies of this model (0/1
Dijkstra over (next adjoint step, current state, stored set)), so it assumes
nothing about the shape of an optimal schedule.  ``min_advances_dp`` is the
classical recursive split (first-sweep checkpoints, then binomial reversal of
each segment); the tests check it against the exhaustive search on tiny
chains and use it as the reference for longer ones.
"""
from __future__ import annotations

import heapq
from functools import lru_cache
from itertools import combinations


def min_advances_bruteforce(n: int, s: int) -> int:
    """Exhaustive optimum for reversing n steps with s snapshot slots."""
    if n <= 1:
        return 0
    best = None
    # Choose the set stored during the first sweep; search the reversal.
    for k in range(0, min(s, n - 1) + 1):
        for first in combinations(range(1, n), k):
            start = (n - 1, n - 1, frozenset(first))
            dist = {start: 0}
            heap = [(0, start)]
            found = None
            while heap:
                d, st = heapq.heappop(heap)
                if dist.get(st, 1 << 30) < d:
                    continue
                i, c, stored = st
                if i < 0:
                    found = d
                    break
                moves = []
                if c == i:
                    moves.append((0, (i - 1, c, stored)))
                if c < i:
                    moves.append((1, (i, c + 1, stored)))
                for p in stored | {0}:
                    if p <= i and p != c:
                        moves.append((0, (i, p, stored)))
                if c not in stored and c != 0:
                    if len(stored) < s:
                        moves.append((0, (i, c, stored | {c})))
                    else:
                        for q in stored:
                            moves.append((0, (i, c, (stored - {q}) | {c})))
                for w, nst in moves:
                    # states beyond the next adjoint step are never useful again
                    i2, c2, st2 = nst
                    st2 = frozenset(p for p in st2 if p <= i2)
                    nst = (i2, c2, st2)
                    nd = d + w
                    if nd < dist.get(nst, 1 << 30):
                        dist[nst] = nd
                        heapq.heappush(heap, (nd, nst))
            if found is not None and (best is None or found < best):
                best = found
    return best


@lru_cache(maxsize=None)
def _A(L: int, f: int) -> int:
    """Reverse x_0..x_{L-1} with x_0 restorable, nothing current, f free slots."""
    if L <= 1:
        return 0
    if f == 0:
        return L * (L - 1) // 2
    return min(m + _A(L - m, f - 1) + _A(m, f) for m in range(1, L))


@lru_cache(maxsize=None)
def _W(n: int, f: int) -> int:
    """Reverse a chain of n states whose last is current after the first sweep."""
    if n <= 1:
        return 0
    best = _A(n - 1, f)
    if f >= 1:
        for m in range(1, n):
            best = min(best, _W(n - m, f - 1) + _A(m, f))
    return best


def min_advances_dp(n: int, s: int) -> int:
    """Recursive-split optimum (agrees with the exhaustive search on tiny chains)."""
    return _W(n, s)
