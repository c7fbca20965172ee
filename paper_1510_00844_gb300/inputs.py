"""Seeded synthetic inputs for the sparse product C = A.B.

This module builds the matrices both the CUDA path and the CPU oracle consume.
It holds none of the product's arithmetic: it only draws random patterns and
values and lays them out as CSR (row pointers int64, column indices sorted
ascending inside each row, no duplicates).

Workload classes (stand-ins for the paper's matrices, Sec. 5 "Experimental
Results", since the real collections are not part of this project):

* ``er_column_regular``   -- Erdos-Renyi-like: exactly ``d`` distinct uniformly
  random rows in every column.
* ``rmat``                -- R-MAT recursive generator with the Graph500 quadrant
  probabilities a=.57, b=c=.19, d=.05 (Sec. 5), 16 edges per vertex on average,
  symmetrised (A + A^T, duplicates summed) and relabelled by a seeded random
  symmetric permutation P A P^T, as the paper does for load balance (Sec. 5).
* ``laplacian_7pt`` / ``aggregation_2x2x2`` -- AMG model problem for the
  restriction product R^T A R (Sec. 5.4 "Multiplication with the restriction
  operator"), with a piecewise-constant 2x2x2 aggregation in place of MIS-2.
* ``batched_er``          -- many independent uneven ER products.
* ``mcl_transition``      -- column-stochastic Markov matrix M, stored as M^T in
  CSR so that columns of M are rows (Markov clustering expansion, Sec. 5.3).

Every generator is a pure function of its arguments and seed (numpy PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

G500 = (0.57, 0.19, 0.19, 0.05)
BASE_SEED = 20151004


@dataclasses.dataclass
class CSR:
    """Host CSR matrix. ``val`` is None for pattern-only (Boolean) matrices."""

    nrows: int
    ncols: int
    rowptr: np.ndarray          # int64 [nrows+1]
    col: np.ndarray             # int32 or int64 [nnz], ascending within a row
    val: Optional[np.ndarray]   # float64 / float32 / int64 [nnz] or None

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def with_index(self, dtype) -> "CSR":
        return CSR(self.nrows, self.ncols, self.rowptr, self.col.astype(dtype), self.val)

    def with_values(self, val) -> "CSR":
        return CSR(self.nrows, self.ncols, self.rowptr, self.col, val)

    def pattern(self) -> "CSR":
        return CSR(self.nrows, self.ncols, self.rowptr, self.col, None)

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _csr_from_sorted(m, n, rows, cols, vals, index_dtype) -> CSR:
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(m, n, rowptr, cols.astype(index_dtype), vals)


def coo_to_csr(m, n, rows, cols, vals=None, index_dtype=np.int64, sum_duplicates=True) -> CSR:
    """Sort (row, col) lexicographically; duplicates are summed when asked
    (the generator recipe "duplicates summed"), else must not occur."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * np.int64(n) + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    rows = rows[order]
    cols = cols[order]
    if vals is not None:
        vals = np.asarray(vals)[order]
    if key.size:
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        if not first.all():
            if not sum_duplicates:
                raise ValueError("duplicate entries")
            starts = np.flatnonzero(first)
            if vals is not None:
                # sequential per-group sums in stable (draw) order: the r-th
                # duplicate of every group is added in pass r
                out = vals[starts].copy()
                grp = np.cumsum(first) - 1
                rank = np.arange(key.size) - starts[grp]
                r = 1
                while True:
                    sel = np.flatnonzero(rank == r)
                    if sel.size == 0:
                        break
                    out[grp[sel]] = out[grp[sel]] + vals[sel]
                    r += 1
                vals = out
            rows = rows[starts]
            cols = cols[starts]
    return _csr_from_sorted(m, n, rows, cols, vals, index_dtype)


def _distinct_rows_per_column(rng, n_rows, n_cols, d):
    """``d`` distinct row indices in [0, n_rows) for every column, by redraw."""
    if d > n_rows:
        raise ValueError("d > n_rows")
    rows = rng.integers(0, n_rows, size=(n_cols, d), dtype=np.int64)
    while True:
        rows.sort(axis=1)
        dup = np.zeros(rows.shape, dtype=bool)
        dup[:, 1:] = rows[:, 1:] == rows[:, :-1]
        k = int(dup.sum())
        if k == 0:
            return rows
        rows[dup] = rng.integers(0, n_rows, size=k, dtype=np.int64)


def er_column_regular(n, d, seed, n_rows=None, index_dtype=np.int32, value="u01_f64") -> CSR:
    """n_rows x n matrix with exactly ``d`` distinct uniform rows per column.

    Values are drawn in CSR order after the pattern: ``u01_f64`` = U(0,1)
    float64, ``u11_f32`` = U(-1,1) float32, ``int`` = integers in [-3, 3]
    (int64), ``none`` = pattern only."""
    rng = np.random.default_rng(seed)
    m = n if n_rows is None else n_rows
    rows = _distinct_rows_per_column(rng, m, n, d)
    cols = np.repeat(np.arange(n, dtype=np.int64), d)
    A = coo_to_csr(m, n, rows.ravel(), cols, None, index_dtype, sum_duplicates=False)
    return A.with_values(draw_values(rng, A.nnz, value))


def draw_values(rng, nnz, value):
    if value == "u01_f64":
        return rng.random(nnz)
    if value == "u11_f32":
        return (rng.random(nnz) * 2.0 - 1.0).astype(np.float32)
    if value == "int":
        return rng.integers(-3, 4, size=nnz, dtype=np.int64)
    if value == "none":
        return None
    raise ValueError(value)


def rmat_edges(scale, edge_factor, rng, probs=G500):
    """Directed R-MAT edges: per bit, one quadrant draw (no noise)."""
    a, b, c, _ = probs
    E = edge_factor * (1 << scale)
    src = np.zeros(E, dtype=np.int64)
    dst = np.zeros(E, dtype=np.int64)
    for bit in range(scale):
        r = rng.random(E)
        s_bit = r >= a + b                                  # quadrants c, d
        d_bit = ((r >= a) & (r < a + b)) | (r >= a + b + c)  # quadrants b, d
        src |= s_bit.astype(np.int64) << bit
        dst |= d_bit.astype(np.int64) << bit
    return src, dst


def rmat(scale, edge_factor=16, seed=BASE_SEED + 2, probs=G500, index_dtype=np.int32,
         value="u01_f64", symmetrize=True, permute=True) -> CSR:
    """Graph500-style R-MAT matrix of order 2**scale.

    Draw order: edges (scale bit draws), then one value per directed edge, then
    the permutation. Symmetrised as A + A^T with duplicates (and both copies of
    a self loop) summed; then relabelled i -> perm[i] on rows and columns."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, rng, probs)
    vals = draw_values(rng, src.size, "u01_f64")
    if symmetrize:
        rows = np.concatenate([src, dst])
        cols = np.concatenate([dst, src])
        vals = np.concatenate([vals, vals])
    else:
        rows, cols = src, dst
    if permute:
        perm = rng.permutation(n).astype(np.int64)
        rows = perm[rows]
        cols = perm[cols]
    A = coo_to_csr(n, n, rows, cols, vals, index_dtype, sum_duplicates=True)
    if value == "u01_f64":
        return A
    if value == "none":
        return A.pattern()
    return A.with_values(draw_values(rng, A.nnz, value))


def laplacian_7pt(N, index_dtype=np.int32) -> CSR:
    """7-point Laplacian on an N^3 grid (diag 6, neighbours -1), x fastest."""
    n = N * N * N
    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = (idx // N) % N
    z = idx // (N * N)
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 6.0)]
    for (coord, stride) in ((x, 1), (y, N), (z, N * N)):
        for sgn in (-1, 1):
            ok = (coord + sgn >= 0) & (coord + sgn < N)
            rows.append(idx[ok])
            cols.append(idx[ok] + sgn * stride)
            vals.append(np.full(int(ok.sum()), -1.0))
    return coo_to_csr(n, n, np.concatenate(rows), np.concatenate(cols),
                      np.concatenate(vals), index_dtype, sum_duplicates=False)


def aggregation_2x2x2(N, index_dtype=np.int32) -> CSR:
    """Piecewise-constant aggregation R (N^3 x (N/2)^3): one 1.0 per row,
    fine point (x,y,z) -> coarse (x/2, y/2, z/2), lexicographic x fastest."""
    assert N % 2 == 0
    n = N * N * N
    M = N // 2
    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = (idx // N) % N
    z = idx // (N * N)
    agg = (x // 2) + M * ((y // 2) + M * (z // 2))
    rowptr = np.arange(n + 1, dtype=np.int64)
    return CSR(n, M * M * M, rowptr, agg.astype(index_dtype), np.ones(n))


def batched_er(count=512, seed=BASE_SEED + 4, nmin=1024, nmax=65536, dmin=4, dmax=32,
               value="u11_f32", index_dtype=np.int32):
    """``count`` independent products (A_i, B_i): n_i = floor(exp(U(ln nmin,
    ln nmax))), d_i uniform integer in [dmin, dmax] nonzeros per column for
    both operands. Per-product sub-seeds come from one parent stream."""
    rng = np.random.default_rng(seed)
    ns = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(np.int64)
    ds = rng.integers(dmin, dmax + 1, size=count)
    subseeds = rng.integers(0, 2**62, size=(count, 2))
    out = []
    for i in range(count):
        n, d = int(ns[i]), int(ds[i])
        A = er_column_regular(n, d, int(subseeds[i, 0]), index_dtype=index_dtype, value=value)
        B = er_column_regular(n, d, int(subseeds[i, 1]), index_dtype=index_dtype, value=value)
        out.append((A, B))
    return out


def mcl_transition(scale, edge_factor=16, seed=BASE_SEED + 5, index_dtype=np.int32) -> CSR:
    """M^T for a column-stochastic M built from a symmetrised G500 R-MAT graph
    W plus a unit self loop on every vertex: M^T(j,:) = W(j,:) / sum W(j,:)."""
    W = rmat(scale, edge_factor, seed=seed, index_dtype=np.int64)
    n = W.nrows
    rows = np.repeat(np.arange(n, dtype=np.int64), W.row_lengths())
    rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([W.col.astype(np.int64), np.arange(n, dtype=np.int64)])
    vals = np.concatenate([W.val, np.ones(n)])
    W1 = coo_to_csr(n, n, rows, cols, vals, np.int64, sum_duplicates=True)
    rs = np.add.reduceat(W1.val, W1.rowptr[:-1])
    per_entry = np.repeat(rs, W1.row_lengths())
    return CSR(n, n, W1.rowptr, W1.col.astype(index_dtype), W1.val / per_entry)


def random_csr(m, n, density, seed, value="u01_f64", index_dtype=np.int64, empty_rows=0.0) -> CSR:
    """Bernoulli(density) pattern, optionally blanking a fraction of rows."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    if empty_rows > 0:
        mask[rng.random(m) < empty_rows, :] = False
    r, c = np.nonzero(mask)
    A = coo_to_csr(m, n, r, c, None, index_dtype, sum_duplicates=False)
    return A.with_values(draw_values(rng, A.nnz, value))


def permutation(n, seed) -> np.ndarray:
    return np.random.default_rng(seed).permutation(n).astype(np.int64)


def permute_symmetric(A: CSR, perm: np.ndarray) -> CSR:
    """P A P^T with row/col i relabelled perm[i] (pure relabelling)."""
    rows = np.repeat(np.arange(A.nrows, dtype=np.int64), A.row_lengths())
    return coo_to_csr(A.nrows, A.ncols, perm[rows], perm[A.col.astype(np.int64)], A.val,
                      A.col.dtype, sum_duplicates=False)


def identity(n, index_dtype=np.int64, value_dtype=np.float64) -> CSR:
    return CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=index_dtype),
               np.ones(n, dtype=value_dtype))


def complete_graph(n, index_dtype=np.int64) -> CSR:
    """Adjacency of K_n (ones off the diagonal)."""
    r, c = np.nonzero(~np.eye(n, dtype=bool))
    return coo_to_csr(n, n, r, c, np.ones(r.size), index_dtype, sum_duplicates=False)


def transpose_pattern_copy(A: CSR) -> CSR:
    """Data movement only (used to build B^T / A^T operands for tests)."""
    rows = np.repeat(np.arange(A.nrows, dtype=np.int64), A.row_lengths())
    return coo_to_csr(A.ncols, A.nrows, A.col.astype(np.int64), rows, A.val, A.col.dtype,
                      sum_duplicates=False)
