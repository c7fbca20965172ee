"""Pins of the MIS-2 aggregation oracle (Alg. 3): the counter-based generator
against SplitMix64's published first output, a path graph whose keys are the
vertex ids (closed form: every third vertex, one per round), and the defining
properties on grids and random graphs -- no two members within distance 2,
every vertex within distance 2 of a member, aggregates that partition the
vertices around exactly one member each."""
import numpy as np
import pytest

from oracle import mis2
from paper_1510_00844_gb300 import inputs


def test_splitmix64_published_value():
    # SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF
    assert int(mis2.splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


def test_keys_are_unique_and_carry_the_vertex():
    k = mis2.keys(5, 3, 10000)
    assert np.unique(k).size == k.size and (k >= 0).all()
    assert np.array_equal(k & ((1 << 31) - 1), np.arange(10000))


def path(n):
    rows = np.concatenate([np.arange(n), np.arange(n - 1), np.arange(1, n)])
    cols = np.concatenate([np.arange(n), np.arange(1, n), np.arange(n - 1)])
    return inputs.coo_to_csr(n, n, rows, cols, np.ones(rows.size))


@pytest.mark.parametrize("n", [1, 2, 3, 7, 30])
def test_path_graph_closed_form(n):
    """Keys increasing with the vertex id: each round admits exactly the
    smallest remaining vertex, so the set is {0, 3, 6, ...}."""
    A = path(n)
    member, rounds = mis2.mis2(A, 0, key_fn=lambda t, m: np.arange(m, dtype=np.int64))
    assert np.array_equal(np.flatnonzero(member), np.arange(0, n, 3))
    assert rounds == len(range(0, n, 3))
    agg = mis2.aggregate(A, member)
    # member 3j owns 3j-1, 3j, 3j+1 (aggregate j); a last vertex two steps
    # past the last member joins the last aggregate
    last = len(range(0, n, 3)) - 1
    assert np.array_equal(agg, np.minimum((np.arange(n) + 1) // 3, last))


def dist2_pattern(A):
    P = np.zeros((A.nrows, A.ncols), dtype=bool)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    P[rows, np.asarray(A.col, dtype=np.int64)] = True
    P |= P.T
    np.fill_diagonal(P, True)
    P2 = (P.astype(np.int64) @ P.astype(np.int64)) > 0
    return P, P2


@pytest.mark.parametrize("gen", ["grid", "random", "rmat"])
@pytest.mark.parametrize("seed", [1, 2])
def test_mis2_properties(gen, seed):
    if gen == "grid":
        A = inputs.laplacian_7pt(6)
    elif gen == "random":
        R = inputs.random_csr(300, 300, 0.01, seed, value="u01_f64")
        M = inputs.coo_to_csr(300, 300, np.concatenate([np.repeat(np.arange(300), np.diff(R.rowptr)), R.col]),
                              np.concatenate([R.col, np.repeat(np.arange(300), np.diff(R.rowptr))]),
                              np.ones(2 * R.nnz))
        A = M
    else:
        A = inputs.rmat(8, seed=seed)
    member, rounds = mis2.mis2(A, seed)
    P, P2 = dist2_pattern(A)
    idx = np.flatnonzero(member)
    sub = P2[np.ix_(idx, idx)]
    assert not (sub & ~np.eye(idx.size, dtype=bool)).any()     # independent at distance 2
    assert P2[:, idx].any(axis=1).all()                          # maximal
    agg = mis2.aggregate(A, member)
    assert (agg >= 0).all() and (agg < idx.size).all()           # every vertex aggregated
    assert np.array_equal(agg[idx], np.arange(idx.size))         # members own their aggregate
    for j, v in enumerate(idx):
        nb = np.flatnonzero(P[v])
        assert (agg[nb] == j).all()                              # neighbours of a member join it
    for v in range(A.nrows):                                     # aggregates are connected
        if not member[v]:
            assert (agg[np.flatnonzero(P[v]) ] == agg[v]).any()
