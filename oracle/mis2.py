"""Distance-2 maximal independent set and the aggregation built on it (the
restriction operator R of the paper's AMG experiments, Sec. 5.4, Alg. 3).

TEST INFRASTRUCTURE ONLY.

Alg. 3 in the paper's notation, with these readings:
* a vertex's value in round t is the key of a counter-based generator,
  key(seed, t, v) = ((splitmix64(seed ^ (t * 0xD1B54A32D192ED03) + v) >> 33) << 31) | v
  (SplitMix64 as published by Steele, Lea and Flood / Vigna); the vertex id in
  the low 31 bits makes keys unique, so ties cannot select two neighbours;
* MxV with (min, select2nd) gives, for every vertex, the smallest value among
  its neighbours (the rows of A, diagonal included); applied twice it reaches
  the distance-2 neighbourhood;
* a candidate joins the set when its own value is the smallest within
  distance 2 ("Is2ndSmaller" read as <=, since the distance-2 minimum
  includes the vertex itself);
* the two pruning steps remove the new members, and every candidate within
  distance 2 of them, from the candidates (the printed EwiseMult is read as a
  set difference, which is what the text says the lines do).
Aggregates: each set member v (numbered in increasing vertex order) owns v
and its neighbours; every remaining vertex joins the smallest-numbered
aggregate among its neighbours (the paper assigns the remaining vertices to
aggregates at random for load balance; here the choice is the minimum, so
that it is reproducible).  R is n x (number of aggregates), R(v, agg(v)) = 1.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
INF = np.int64(np.iinfo(np.int64).max)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state x (uint64 array, wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def keys(seed: int, t: int, n: int) -> np.ndarray:
    """key(seed, t, v) for v = 0..n-1 as int64 (non-negative, unique)."""
    v = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = (np.uint64(seed) ^ (np.uint64(t) * np.uint64(0xD1B54A32D192ED03))) & _M64
        h = splitmix64((base + v) & _M64)
    return (((h >> np.uint64(33)) << np.uint64(31)) | v).astype(np.int64)


def min_adjacent(A, x: np.ndarray) -> np.ndarray:
    """(min, select2nd) MxV: y(i) = min over k in A(i,:) of x(k) (INF if none)."""
    rp = np.asarray(A.rowptr, dtype=np.int64)
    col = np.asarray(A.col, dtype=np.int64)
    y = np.full(A.nrows, INF, dtype=np.int64)
    rows = np.repeat(np.arange(A.nrows), np.diff(rp))
    np.minimum.at(y, rows, x[col])
    return y


def mis2(A, seed: int, key_fn=None):
    """Returns (member flags, rounds).  key_fn(t, n) overrides the keys (tests)."""
    n = A.nrows
    cand = np.ones(n, dtype=bool)
    member = np.zeros(n, dtype=bool)
    t = 0
    while cand.any():
        k = keys(seed, t, n) if key_fn is None else key_fn(t, n)
        x = np.where(cand, k, INF)
        m1 = min_adjacent(A, x)
        m2 = min_adjacent(A, m1)
        new = cand & (x <= np.minimum(m1, m2))
        member |= new
        cand &= ~new
        y = np.where(new, np.int64(0), INF)
        a1 = min_adjacent(A, y)
        a2 = min_adjacent(A, a1)
        cand &= ~((a1 < INF) | (a2 < INF))
        t += 1
    return member, t


def aggregate(A, member: np.ndarray) -> np.ndarray:
    """Aggregate id of every vertex (see the module docstring)."""
    n = A.nrows
    ids = np.cumsum(member) - 1
    agg = np.where(member, ids, INF).astype(np.int64)
    near = min_adjacent(A, agg)
    agg = np.where(member, agg, near)
    rest = min_adjacent(A, agg)
    agg = np.where(agg < INF, agg, rest)
    return agg


def restriction(A, seed: int):
    """(R as (rowptr, col, val), number of aggregates, rounds)."""
    member, rounds = mis2(A, seed)
    agg = aggregate(A, member)
    n = A.nrows
    return (np.arange(n + 1, dtype=np.int64), agg, np.ones(n)), int(member.sum()), rounds
