"""Pins for the CPU oracle against facts the mathematics and the paper fix.

None of these re-types the oracle's loop: each compares it with an independent
route (dense matrix products, algebraic identities, closed forms, brute force
on tiny inputs) chosen so that a dropped term, a wrong index, a transposed
operand or a wrong summation order fails at least one of them."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1510_00844_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(M):
    D = np.zeros((M.nrows, M.ncols), dtype=np.float64 if M.val is None or
                 np.issubdtype(np.asarray(M.val).dtype, np.floating) else np.int64)
    rows = np.repeat(np.arange(M.nrows), np.diff(M.rowptr))
    D[rows, np.asarray(M.col, dtype=np.int64)] = 1 if M.val is None else M.val
    return D


def pattern(M):
    P = np.zeros((M.nrows, M.ncols), dtype=bool)
    rows = np.repeat(np.arange(M.nrows), np.diff(M.rowptr))
    P[rows, np.asarray(M.col, dtype=np.int64)] = True
    return P


def assert_valid_csr(C):
    rp = np.asarray(C.rowptr)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(C.col)
    for i in range(C.nrows):
        c = np.asarray(C.col[rp[i]:rp[i + 1]])
        assert np.all(np.diff(c) > 0), f"row {i} not strictly ascending"
        assert c.size == 0 or (c[0] >= 0 and c[-1] < C.ncols)


SHAPES = [(1, 1, 1), (5, 1, 7), (1, 9, 1), (13, 17, 11), (32, 20, 40), (64, 64, 64), (3, 50, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("density", [0.02, 0.15, 0.5])
def test_integer_values_equal_dense_matmul(shape, density):
    m, l, n = shape
    seed = hash((shape, density)) % 2**31
    A = inputs.random_csr(m, l, density, seed, value="int", empty_rows=0.2)
    B = inputs.random_csr(l, n, density, seed + 1, value="int", empty_rows=0.2)
    C = oracle.spgemm(A, B)
    assert_valid_csr(C)
    # pattern = structural product (explicit zeros and cancellations kept)
    P = (pattern(A).astype(np.int64) @ pattern(B).astype(np.int64)) > 0
    assert np.array_equal(pattern(C), P)
    # values = exact integer dense product on the pattern
    D = dense(A) @ dense(B)
    assert np.array_equal(dense(C)[P], D[P])


@pytest.mark.parametrize("shape", SHAPES)
def test_float_values_close_to_dense_matmul(shape):
    m, l, n = shape
    A = inputs.random_csr(m, l, 0.3, 7, value="u01_f64")
    B = inputs.random_csr(l, n, 0.3, 8, value="u01_f64")
    C = oracle.spgemm(A, B)
    D = dense(A) @ dense(B)
    np.testing.assert_allclose(dense(C), D, rtol=1e-13, atol=0)


def brute_force(A, B):
    """Triple loop in pure Python over dense copies; sum in ascending k,
    first structural product starts the sum."""
    dA, dB = pattern(A), pattern(B)
    vA, vB = dense(A), dense(B)
    out = {}
    for i in range(A.nrows):
        for j in range(B.ncols):
            acc = None
            for k in range(A.ncols):
                if dA[i, k] and dB[k, j]:
                    p = float(vA[i, k]) * float(vB[k, j])
                    acc = p if acc is None else acc + p
            if acc is not None:
                out[(i, j)] = acc
    return out


@pytest.mark.parametrize("seed", range(4))
def test_bitexact_against_brute_force_ascending_k(seed):
    A = inputs.random_csr(9, 12, 0.4, 100 + seed, value="u01_f64")
    B = inputs.random_csr(12, 10, 0.4, 200 + seed, value="u01_f64")
    ref = brute_force(A, B)
    C = oracle.spgemm(A, B)
    got = {}
    for i in range(C.nrows):
        for t in range(C.rowptr[i], C.rowptr[i + 1]):
            got[(i, int(C.col[t]))] = float(C.val[t])
    assert got.keys() == ref.keys()
    for key in ref:
        assert got[key] == ref[key], key      # same order -> same bits


def test_explicit_zeros_stay_in_pattern():
    # row 0 of A = [1, 1], B = [[1],[-1]] -> C(0,0) = 0 but structurally present
    A = inputs.CSR(1, 2, np.array([0, 2]), np.array([0, 1]), np.array([1.0, 1.0]))
    B = inputs.CSR(2, 1, np.array([0, 1, 2]), np.array([0, 0]), np.array([1.0, -1.0]))
    C = oracle.spgemm(A, B)
    assert C.nnz == 1 and C.val[0] == 0.0
    Z = inputs.CSR(1, 2, np.array([0, 2]), np.array([0, 1]), np.array([0.0, 0.0]))
    assert oracle.spgemm(Z, B).nnz == 1


@pytest.mark.parametrize("seed", range(3))
def test_transpose_identity_bitexact(seed):
    A = inputs.random_csr(30, 25, 0.2, seed, value="u01_f64")
    B = inputs.random_csr(25, 35, 0.2, seed + 50, value="u01_f64")
    C = oracle.spgemm(A, B)
    Ct = oracle.transpose(C)
    D = oracle.spgemm(oracle.transpose(B), oracle.transpose(A))
    assert np.array_equal(Ct.rowptr, D.rowptr)
    assert np.array_equal(Ct.col, D.col)
    assert np.array_equal(Ct.val, D.val)      # same k order, b*a == a*b


def test_identity_products_bitexact():
    A = inputs.random_csr(40, 33, 0.1, 3, value="u01_f64")
    for C in (oracle.spgemm(A, inputs.identity(33)), oracle.spgemm(inputs.identity(40), A)):
        assert np.array_equal(C.rowptr, A.rowptr)
        assert np.array_equal(C.col, A.col)
        assert np.array_equal(C.val, A.val)


@pytest.mark.parametrize("gen", ["er", "rmat", "random"])
def test_nnz_bounds(gen):
    if gen == "er":
        A = inputs.er_column_regular(512, 8, 1)
        B = A
    elif gen == "rmat":
        A = inputs.rmat(10)
        B = A
    else:
        A = inputs.random_csr(50, 60, 0.05, 4)
        B = inputs.random_csr(60, 70, 0.05, 5)
    C = oracle.spgemm(A, B)
    fl = oracle.row_flops(A, B)
    cnt = np.diff(C.rowptr)
    assert C.nnz <= fl.sum()
    assert np.all(cnt <= np.minimum(fl, B.ncols))
    lenB = np.diff(B.rowptr)
    for i in range(A.nrows):
        ks = np.asarray(A.col[A.rowptr[i]:A.rowptr[i + 1]], dtype=np.int64)
        if ks.size:
            assert cnt[i] >= lenB[ks].max()
    # flops by an independent route: dense pattern products count multiplications
    np.testing.assert_array_equal(
        fl, (pattern(A).astype(np.int64) @ lenB.reshape(-1, 1)).ravel())


def test_complete_graph_closed_forms():
    with open(os.path.join(GOLDEN, "kn_trace.txt")) as fh:
        rows = [tuple(map(int, ln.split())) for ln in fh if ln.strip() and not ln.startswith("#")]
    for n, tr in rows:
        K = inputs.complete_graph(n)
        K2 = oracle.spgemm(K, K)
        D2 = dense(K2)
        # A^2 = (n-2) A + (n-1) I on K_n
        expect = (n - 2) * (1 - np.eye(n)) + (n - 1) * np.eye(n)
        assert np.array_equal(D2, expect)
        K3 = oracle.spgemm(K2, K)
        assert np.trace(dense(K3)) == tr == n * (n - 1) * (n - 2)


def test_column_stochastic_products_stay_stochastic():
    M = inputs.mcl_transition(9)                       # rows of M^T sum to 1
    P = oracle.spgemm(M, M)                            # (M M)^T = M^T M^T
    rs = np.add.reduceat(P.val, P.rowptr[:-1])
    q = np.diff(M.rowptr).max() ** 2                   # terms per row sum
    u = 2.0 ** -53
    assert np.all(np.abs(rs - 1.0) <= 2 * q * u)


def test_permutation_equivariance():
    A = inputs.rmat(9, permute=False)
    perm = inputs.permutation(A.nrows, 11)
    C = oracle.spgemm(A, A)
    PA = inputs.permute_symmetric(A, perm)
    PC = oracle.spgemm(PA, PA)
    ref = inputs.permute_symmetric(inputs.CSR(C.nrows, C.ncols, C.rowptr, C.col, C.val), perm)
    assert np.array_equal(PC.rowptr, ref.rowptr)
    assert np.array_equal(PC.col, ref.col)
    np.testing.assert_allclose(PC.val, ref.val, rtol=1e-12)


def test_boolean_pattern_equals_structural_pattern():
    A = inputs.rmat(9)
    Cb = oracle.spgemm(A.pattern(), A.pattern(), semiring="or_and")
    Cf = oracle.spgemm(A, A)
    assert Cb.val is None
    assert np.array_equal(Cb.rowptr, Cf.rowptr)
    assert np.array_equal(Cb.col, Cf.col)


def test_int64_wraparound():
    big = np.int64(2**62 + 12345)
    A = inputs.CSR(1, 2, np.array([0, 2]), np.array([0, 1]), np.array([big, 3], dtype=np.int64))
    B = inputs.CSR(2, 1, np.array([0, 1, 2]), np.array([0, 0]), np.array([4, big], dtype=np.int64))
    C = oracle.spgemm(A, B)
    expect = (int(big) * 4 + 3 * int(big)) % 2**64
    if expect >= 2**63:
        expect -= 2**64
    assert int(C.val[0]) == expect


def galerkin_closed_form(N, level):
    """R^T A R at level l of the 2x2x2 aggregation hierarchy equals 4^l times
    the 7-point Laplacian on the (N/2^l)^3 grid (integer-valued)."""
    L = inputs.laplacian_7pt(N >> level)
    return L.with_values(L.val * (4.0 ** level))


@pytest.mark.parametrize("N", [8, 16])
def test_amg_galerkin_closed_form(N):
    A = inputs.laplacian_7pt(N)
    level = 0
    with open(os.path.join(GOLDEN, "amg_galerkin.txt")) as fh:
        table = {}
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                g, lv, diag, off, nnz_rta, nnz_rtar = map(int, ln.split())
                table[(g, lv)] = (diag, off, nnz_rta, nnz_rtar)
    while (N >> level) >= 4:
        R = inputs.aggregation_2x2x2(N >> level)
        RtA = oracle.spgemm(oracle.transpose(R), A)
        Ac = oracle.spgemm(RtA, R)
        ref = galerkin_closed_form(N, level + 1)
        assert np.array_equal(Ac.rowptr, ref.rowptr)
        assert np.array_equal(Ac.col, ref.col)
        assert np.array_equal(Ac.val, ref.val)
        diag, off, nnz_rta, nnz_rtar = table[(N >> level, level + 1)]
        assert RtA.nnz == nnz_rta and Ac.nnz == nnz_rtar
        assert set(np.unique(Ac.val)) == {float(diag), float(off)}
        A = inputs.CSR(Ac.nrows, Ac.ncols, Ac.rowptr, Ac.col, Ac.val)
        level += 1


@pytest.mark.parametrize("c", [1, 2, 3, 4, 8, 16])
def test_merge_of_kslices_equals_unsplit(c):
    A = inputs.rmat(9)
    C = oracle.spgemm(A, A)
    parts = [oracle.spgemm(As, Bs) for As, Bs in oracle.kslice(A, A, c)]
    # paper bound on the intermediate (Sec. 4.4): nnz(C^int) <= flops
    assert sum(P.nnz for P in parts) <= oracle.row_flops(A, A).sum()
    assert sum(P.nnz for P in parts) >= C.nnz
    S = oracle.sum_partials(parts)
    assert np.array_equal(S.rowptr, C.rowptr)
    assert np.array_equal(S.col, C.col)
    np.testing.assert_allclose(S.val, C.val, rtol=1e-12)
    if c == 1:
        assert np.array_equal(S.val, C.val)


def test_merge_integer_bitexact_and_empty_slices():
    A = inputs.random_csr(20, 3, 0.5, 1, value="int")
    B = inputs.random_csr(3, 25, 0.5, 2, value="int")
    C = oracle.spgemm(A, B)
    for c in (1, 3, 5, 7):                               # c > l gives empty slices
        parts = [oracle.spgemm(As, Bs) for As, Bs in oracle.kslice(A, B, c)]
        S = oracle.sum_partials(parts)
        assert np.array_equal(S.col, C.col) and np.array_equal(S.val, C.val)


def test_kslice_bounds_cover_inner_dimension():
    for l, c in itertools.product([0, 1, 5, 16, 17, 262144], [1, 2, 3, 4, 16]):
        b = oracle.kslice_bounds(l, c)
        assert b[0][0] == 0 and b[-1][1] == l
        assert all(b[s][1] == b[s + 1][0] for s in range(c - 1))
        assert all(hi - lo in (l // c, l // c + 1) for lo, hi in b)


def test_mcl_prune_renorm():
    M = inputs.mcl_transition(8)
    P = oracle.spgemm(M, M)
    Q = oracle.mcl_prune_renorm(P, 1e-2)
    pv = np.asarray(P.val)
    assert Q.nnz == int((pv >= 1e-2).sum())
    assert np.all(Q.val > 0)
    for i in range(0, Q.nrows, 7):
        a, b = Q.rowptr[i], Q.rowptr[i + 1]
        sel = pv[P.rowptr[i]:P.rowptr[i + 1]] >= 1e-2
        assert np.array_equal(Q.col[a:b], np.asarray(P.col[P.rowptr[i]:P.rowptr[i + 1]])[sel])
        if b > a:
            assert abs(Q.val[a:b].sum() - 1.0) <= 1e-13


def test_pattern_only_sum_of_partials_is_the_union():
    """The Boolean sum of partial products is the union of their patterns
    (Sec. 4.3's merge with duplicate reduction, (or, and) semiring), checked
    against a set union row by row."""
    A = inputs.rmat(8).pattern()
    parts = [oracle.spgemm(As, Bs, semiring="or_and") for As, Bs in oracle.kslice(A, A, 3)]
    S = oracle.sum_partials(parts, semiring="or_and")
    assert S.val is None
    for i in range(A.nrows):
        u = set()
        for P in parts:
            u |= set(np.asarray(P.col)[P.rowptr[i]:P.rowptr[i + 1]].tolist())
        assert np.asarray(S.col)[S.rowptr[i]:S.rowptr[i + 1]].tolist() == sorted(u)


def test_mcl_prune_keeps_entries_equal_to_threshold():
    """Pruning drops entries strictly below the threshold: an entry exactly at
    1e-4 stays.  Hand-written 2 x 4 case: row 0 holds 1e-4 (kept), 9.9e-5
    (dropped) and 0.5 (kept); row 1 holds only 9.99e-5 (dropped), so it ends
    empty.  Kept row 0 renormalised: 1e-4 / (1e-4 + 0.5) and 0.5 / (1e-4 +
    0.5), the sum taken left to right."""
    C = oracle.OCSR(2, 4, np.array([0, 3, 4], dtype=np.int64),
                    np.array([0, 1, 3, 2], dtype=np.int64),
                    np.array([1e-4, 9.9e-5, 0.5, 9.99e-5]))
    Q = oracle.mcl_prune_renorm(C, 1e-4)
    assert Q.nnz == 2                                       # written by hand: 1e-4 and 0.5 survive
    assert list(Q.rowptr) == [0, 2, 2]
    assert list(Q.col) == [0, 3]
    s = 1e-4 + 0.5
    assert Q.val[0] == 1e-4 / s and Q.val[1] == 0.5 / s


# ------------------------------------------------------------ min semirings
# (min, +) and (min, select2nd): the operations MIS-2 aggregation is built
# from (Alg. 3).  A min reduction starts at +inf (int64: INT64_MAX) and keeps
# the running value unless the next term is strictly smaller.

def brute_min(A, B, select2nd: bool):
    """Pure-Python triple loop over structural nonzeros, k ascending."""
    integer = np.issubdtype(np.asarray(A.val).dtype, np.integer)
    ident = np.iinfo(np.int64).max if integer else float("inf")
    out = {}
    for i in range(A.nrows):
        for p in range(A.rowptr[i], A.rowptr[i + 1]):
            k = int(A.col[p])
            for q in range(B.rowptr[k], B.rowptr[k + 1]):
                j = int(B.col[q])
                a, b = A.val[p], B.val[q]
                term = b if select2nd else (int(a) + int(b) if integer else float(a) + float(b))
                cur = out.get((i, j), ident)
                out[(i, j)] = term if term < cur else cur
    return out


@pytest.mark.parametrize("select2nd", [False, True])
@pytest.mark.parametrize("value", ["u01_f64", "int"])
@pytest.mark.parametrize("seed", range(3))
def test_min_semirings_against_brute_force(select2nd, value, seed):
    A = inputs.random_csr(11, 14, 0.35, 300 + seed, value=value)
    B = inputs.random_csr(14, 9, 0.35, 400 + seed, value=value)
    sr = "min_select2nd" if select2nd else "min_plus"
    C = oracle.spgemm(A, B, semiring=sr)
    assert_valid_csr(C)
    ref = brute_min(A, B, select2nd)
    got = {}
    for i in range(C.nrows):
        for t in range(C.rowptr[i], C.rowptr[i + 1]):
            got[(i, int(C.col[t]))] = C.val[t]
    assert got.keys() == ref.keys()
    assert all(got[key] == ref[key] for key in ref)
    # the pattern is the structural product, as for every semiring
    assert np.array_equal(pattern(C), (pattern(A).astype(int) @ pattern(B).astype(int)) > 0)


def test_min_plus_path_graph_closed_form():
    """Path graph 0-1-...-(n-1) with unit weights: (min,+) square gives
    distance-2 walks: C(i,i) = 2 for every vertex with a neighbour, C(i,i+-2)
    = 2, nothing else."""
    n = 12
    rows = np.concatenate([np.arange(n - 1), np.arange(1, n)])
    cols = np.concatenate([np.arange(1, n), np.arange(n - 1)])
    W = inputs.coo_to_csr(n, n, rows, cols, np.ones(rows.size))
    C = oracle.spgemm(W, W, semiring="min_plus")
    D = dense(C)
    for i in range(n):
        for j in range(n):
            expect = 2.0 if (i == j or abs(i - j) == 2) else 0.0
            assert D[i, j] == expect, (i, j)


def test_min_semiring_identity_and_selection():
    """I (zero weights) (min,+) B = B; A (min,select2nd) B takes the minimum
    of the rows of B that A selects (numpy reduction per row)."""
    B = inputs.random_csr(20, 15, 0.3, 9, value="u01_f64")
    Z = inputs.CSR(20, 20, np.arange(21, dtype=np.int64), np.arange(20, dtype=np.int64),
                   np.zeros(20))
    C = oracle.spgemm(Z, B, semiring="min_plus")
    assert np.array_equal(C.rowptr, B.rowptr) and np.array_equal(C.col, B.col)
    assert np.array_equal(C.val, B.val)
    A = inputs.random_csr(7, 20, 0.25, 10, value="u01_f64")
    S = oracle.spgemm(A, B, semiring="min_select2nd")
    DB = np.where(pattern(B), dense(B), np.inf)
    for i in range(A.nrows):
        ks = np.asarray(A.col[A.rowptr[i]:A.rowptr[i + 1]], dtype=np.int64)
        expect = DB[ks].min(axis=0) if ks.size else np.full(B.ncols, np.inf)
        row = np.full(B.ncols, np.inf)
        row[np.asarray(S.col[S.rowptr[i]:S.rowptr[i + 1]], dtype=np.int64)] = \
            S.val[S.rowptr[i]:S.rowptr[i + 1]]
        assert np.array_equal(row, expect)


@pytest.mark.parametrize("sr", ["min_plus", "min_select2nd"])
@pytest.mark.parametrize("c", [2, 5])
def test_min_merge_of_kslices_equals_unsplit(sr, c):
    A = inputs.rmat(9, seed=33, value="u01_f64")
    full = oracle.spgemm(A, A, semiring=sr)
    parts = [oracle.spgemm(As, Bs, semiring=sr) for As, Bs in oracle.kslice(A, A, c)]
    M = oracle.sum_partials(parts, semiring=sr)
    assert np.array_equal(M.rowptr, full.rowptr) and np.array_equal(M.col, full.col)
    assert np.array_equal(M.val, full.val)      # min keeps the first of equal terms


# ------------------------------------------------------------ masks

def test_mask_identities():
    """A full mask keeps C, its complement keeps nothing; a mask and its
    complement split C into two disjoint parts whose union is C; the masked
    product equals the dense product times the 0/1 mask."""
    A = inputs.random_csr(30, 25, 0.2, 11, value="u01_f64")
    B = inputs.random_csr(25, 35, 0.2, 12, value="u01_f64")
    C = oracle.spgemm(A, B)
    full = oracle.mask(C, C)
    assert np.array_equal(full.rowptr, C.rowptr) and np.array_equal(full.col, C.col)
    assert np.array_equal(full.val, C.val)
    assert oracle.mask(C, C, complement=True).col.size == 0
    M = inputs.random_csr(30, 35, 0.3, 13, value="none")
    In, Out = oracle.mask(C, M), oracle.mask(C, M, complement=True)
    assert In.col.size + Out.col.size == C.col.size
    assert not (pattern(In) & pattern(Out)).any()
    assert np.array_equal(pattern(In) | pattern(Out), pattern(C))
    assert np.array_equal(pattern(In), pattern(C) & pattern(M))
    assert np.array_equal(dense(In), dense(C) * pattern(M))
    assert_valid_csr(In)
    assert_valid_csr(Out)
