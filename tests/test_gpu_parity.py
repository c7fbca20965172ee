"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle,
element by element, on seeded inputs that span every row class (empty, the
four hash bins, dense rows with several column chunks), ragged tails, both
index types and every value type."""
import numpy as np
import pytest

import oracle
from paper_1510_00844_gb300 import inputs
from tests.parity import assert_pattern_equal, assert_values_close, rows_subset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


def run(sg, A, B, semiring=0, checked=True):
    dA, dB = sg.to_device(A), sg.to_device(B)
    return sg.spgemm(dA, dB, semiring=semiring, checked=checked, verify=True)


def check_product(sg, A, B, dtype="f64"):
    C = run(sg, A, B)
    R = oracle.spgemm(A, B)
    assert_pattern_equal(C, R)
    assert_values_close(C, R, A, B, dtype)
    return C, R


def test_er_config_small(sg):
    # Erdos-Renyi, n = 16384, exactly 8 distinct rows per column, int32, f64
    A = inputs.er_column_regular(16384, 8, inputs.BASE_SEED + 1)
    C, R = check_product(sg, A, A)
    # same k order and no fused multiply-add: bit-exact in practice
    assert np.array_equal(C.to_host()[2], R.val)


@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 1, 9), (1, 40, 1), (33, 65, 31), (300, 200, 500)])
@pytest.mark.parametrize("density", [0.0, 0.03, 0.3])
def test_random_shapes(sg, shape, density):
    m, l, n = shape
    A = inputs.random_csr(m, l, density, 11 + m, empty_rows=0.2)
    B = inputs.random_csr(l, n, density, 12 + n, empty_rows=0.2)
    check_product(sg, A, B)


@pytest.mark.parametrize("scale", [10, 12, 14])
def test_rmat_dense_rows(sg, scale):
    A = inputs.rmat(scale)
    C, R = check_product(sg, A, A)
    assert np.array_equal(C.to_host()[2], R.val)


def test_rmat_int64_indices(sg):
    A = inputs.rmat(12, index_dtype=np.int64)
    check_product(sg, A, A)


@pytest.mark.parametrize("value", ["int", "u11_f32"])
def test_value_types(sg, value):
    A = inputs.rmat(12, value=value)
    dtype = {"int": "i64", "u11_f32": "f32"}[value]
    C = run(sg, A, A)
    R = oracle.spgemm(A, A)
    assert_pattern_equal(C, R)
    assert_values_close(C, R, A, A, dtype)


def test_boolean_semiring(sg):
    A = inputs.rmat(12)
    Cb = run(sg, A.pattern(), A.pattern(), semiring=1)
    assert Cb.val is None
    R = oracle.spgemm(A.pattern(), A.pattern(), semiring="or_and")
    assert_pattern_equal(Cb, R)
    # OR_AND on valued inputs ignores values
    Cv = run(sg, A, A, semiring=1)
    assert_pattern_equal(Cv, R)


def bin_edge_case():
    """A with rows whose flops sit on every class edge: 0, 1, 32, 33, 128,
    129, 512, 513, 1024, 1025, 4096, plus one row hitting every B row.  B has
    rows of length 1..64 and two long rows (3000 and 20000 columns)."""
    rng = np.random.default_rng(5)
    n = 40000
    lensB = np.concatenate([np.arange(1, 65), [3000, 20000]])
    rowsB, colsB = [], []
    for k, L in enumerate(lensB):
        c = np.sort(rng.choice(n, size=L, replace=False))
        rowsB.append(np.full(L, k))
        colsB.append(c)
    B = inputs.coo_to_csr(len(lensB), n, np.concatenate(rowsB), np.concatenate(colsB),
                          rng.random(int(lensB.sum())), np.int32, sum_duplicates=False)
    targets = [0, 1, 32, 33, 128, 129, 512, 513, 1024, 1025, 4096]
    rowsA, colsA = [], []
    for i, t in enumerate(targets):
        # greedy subset of B rows (distinct k) summing to t
        rem, ks = t, []
        for k in np.argsort(-lensB):
            if lensB[k] <= rem and k not in ks and lensB[k] < 20000:
                ks.append(k)
                rem -= lensB[k]
        assert rem == 0
        rowsA += [i] * len(ks)
        colsA += list(ks)
    i = len(targets)
    rowsA += [i] * len(lensB)
    colsA += list(range(len(lensB)))
    A = inputs.coo_to_csr(i + 1, len(lensB), np.array(rowsA), np.array(colsA),
                          rng.random(len(rowsA)), np.int32, sum_duplicates=False)
    return A, B, targets


def test_class_edges_and_long_rows(sg):
    A, B, targets = bin_edge_case()
    fl = oracle.row_flops(A, B)
    assert list(fl[:len(targets)]) == targets
    C, R = check_product(sg, A, B)
    assert np.array_equal(C.to_host()[2], R.val)


def test_single_huge_row(sg):
    # one row selecting every row of an R-MAT matrix: dense accumulator over
    # all chunks, streaming of long B rows
    B = inputs.rmat(13)
    A = inputs.CSR(1, B.nrows, np.array([0, B.nrows]), np.arange(B.nrows, dtype=np.int32),
                   np.random.default_rng(1).random(B.nrows))
    check_product(sg, A, B)


def test_hypersparse_int64_columns(sg):
    # n > 2^31 columns, few entries: int64 indices end to end (hash rows only)
    rng = np.random.default_rng(3)
    n = (1 << 33) + 7
    m, l = 50, 60
    rA = rng.integers(0, m, 200)
    cA = rng.integers(0, l, 200)
    A = inputs.coo_to_csr(m, l, rA, cA, rng.random(200), np.int64)
    rB = rng.integers(0, l, 300)
    cB = rng.integers(0, n, 300)
    B = inputs.coo_to_csr(l, n, rB, cB, rng.random(300), np.int64)
    C = run(sg, A, B)
    # the oracle's dense accumulator is O(n): relabel B's distinct columns
    # 0..u-1 (monotone, so every row stays sorted), multiply, map back
    uniq = np.unique(B.col)
    Bc = inputs.CSR(l, len(uniq), B.rowptr, np.searchsorted(uniq, B.col), B.val)
    Rc = oracle.spgemm(A, Bc)
    R = oracle.OCSR(Rc.nrows, n, Rc.rowptr, uniq[Rc.col], Rc.val)
    assert_pattern_equal(C, R)
    assert_values_close(C, R)
    assert C.col.dtype.itemsize == 8 and int(C.col.max()) > 2**31


def test_empty_operands(sg):
    A = inputs.CSR(5, 4, np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = inputs.random_csr(4, 7, 0.5, 1, index_dtype=np.int32)
    C = run(sg, A, B)
    assert C.nnz == 0 and np.array_equal(C.to_host()[0], np.zeros(6))
    Z = inputs.CSR(0, 4, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    C = run(sg, Z, B)
    assert C.nnz == 0 and C.nrows == 0


def test_determinism_bitwise(sg):
    A = inputs.rmat(13)
    dA = sg.to_device(A)
    C1 = sg.spgemm(dA, dA)
    C2 = sg.spgemm(dA, dA)
    assert bool((C1.val == C2.val).all()) and bool((C1.col == C2.col).all())


def test_checked_mode_rejects_invalid_csr(sg):
    A = inputs.random_csr(10, 10, 0.3, 2, index_dtype=np.int32)
    bad = A.col.copy()
    r = int(np.argmax(np.diff(A.rowptr) >= 2))
    bad[A.rowptr[r]], bad[A.rowptr[r] + 1] = bad[A.rowptr[r] + 1], bad[A.rowptr[r]]
    Abad = inputs.CSR(10, 10, A.rowptr, bad, A.val)
    with pytest.raises(sg.SpgemmError) as ei:
        run(sg, Abad, A, checked=True)
    assert ei.value.status == 2
    oob = A.col.copy()
    oob[-1] = 10
    with pytest.raises(sg.SpgemmError) as ei:
        run(sg, inputs.CSR(10, 10, A.rowptr, oob, A.val), A, checked=True)
    assert ei.value.status == 2


@pytest.mark.parametrize("c", [1, 2, 3, 4, 8, 16])
def test_kslice_merge(sg, c):
    A = inputs.rmat(12)
    dA = sg.to_device(A)
    C, parts = sg.spgemm_kslice(dA, dA, c, verify=True)
    ref_parts = [oracle.spgemm(As, Bs) for As, Bs in oracle.kslice(A, A, c)]
    for P, R in zip(parts, ref_parts):
        assert_pattern_equal(P, R)
        assert np.array_equal(P.to_host()[2], R.val)
    S = oracle.sum_partials(ref_parts)
    assert_pattern_equal(C, S)
    assert np.array_equal(C.to_host()[2], S.val)     # same order as the definition
    U = oracle.spgemm(A, A)
    assert_pattern_equal(C, U)
    assert_values_close(C, U, A, A)


def test_kslice_bounds_match_oracle(sg):
    A = inputs.rmat(11)
    dA = sg.to_device(A)
    for c in (1, 3, 4, 7):
        b = sg.kslice_bounds(dA, c).cpu().numpy()
        for s, (As, _) in enumerate(oracle.kslice(A, A, c)):
            assert np.array_equal(b[s + 1] - b[s], np.diff(As.rowptr))


def test_merge_integer_and_bool(sg):
    A = inputs.rmat(11, value="int")
    dA = sg.to_device(A)
    C, _ = sg.spgemm_kslice(dA, dA, 4, verify=True)
    R = oracle.spgemm(A, A)
    assert_pattern_equal(C, R)
    assert np.array_equal(C.to_host()[2], R.val)
    Cb, _ = sg.spgemm_kslice(sg.to_device(A.pattern()), sg.to_device(A.pattern()), 3,
                             semiring=1, verify=True)
    assert_pattern_equal(Cb, R)


def test_merge_unaligned_column_arrays(sg):
    """Partials whose int32 column arrays do not start on a 16-byte boundary
    are counted one column per lane (the four-column loads need aligned
    arrays); the merged product is still the oracle's sum of the partials."""
    import torch

    A = inputs.rmat(11)
    dA = sg.to_device(A)
    _, parts = sg.spgemm_kslice(dA, dA, 4, verify=True)
    shifted = []
    for P in parts:
        buf = torch.empty(P.col.numel() + 1, dtype=P.col.dtype, device=P.col.device)
        buf[1:] = P.col
        shifted.append(sg.DeviceCSR(P.nrows, P.ncols, P.rowptr, buf[1:], P.val))
    assert shifted[0].col.data_ptr() % 16 != 0
    C = sg.merge(shifted, verify=True)
    S = oracle.sum_partials([oracle.spgemm(As, Bs) for As, Bs in oracle.kslice(A, A, 4)])
    assert_pattern_equal(C, S)
    assert np.array_equal(C.to_host()[2], S.val)


@pytest.mark.parametrize("c,value,idx", [(2, "u01_f64", np.int32), (3, "u01_f64", np.int32),
                                         (4, "u01_f64", np.int32), (4, "int", np.int64),
                                         (4, "none", np.int32)])
def test_staged_merge_matches_oracle(sg, c, value, idx):
    """The numeric merge with every list staged in shared memory by bulk
    asynchronous copies (spgemm_opts.merge_staged) gives the oracle's sum of
    the partials bit for bit, for rows spanning many windows (R-MAT 13) and
    lists whose arrays end off a 16-byte boundary."""
    import torch
    A = inputs.rmat(13, index_dtype=idx, value=value)
    dA = sg.to_device(A)
    semiring = 1 if value == "none" else 0
    _, parts = sg.spgemm_kslice(dA, dA, c, semiring=semiring, verify=True)
    ws = sg.merge_workspace(c, A.nrows, A.ncols, dA.rowptr.device)
    rp, nnz = sg.merge_symbolic(parts, ws, semiring)
    col = torch.empty(nnz, dtype=dA.col.dtype, device="cuda")
    val = None if value == "none" else torch.empty(nnz, dtype=dA.val.dtype, device="cuda")
    sg.merge_numeric(parts, ws, rp, col, val, semiring, staged=True)
    sg.merge_check(ws)
    C = sg.DeviceCSR(A.nrows, A.ncols, rp, col, val)
    ref = [oracle.spgemm(As, Bs, semiring="or_and" if value == "none" else "plus_times")
           for As, Bs in oracle.kslice(A, A, c)]
    S = oracle.sum_partials(ref, semiring="or_and" if value == "none" else "plus_times")
    assert_pattern_equal(C, S)
    if val is not None:
        assert np.array_equal(C.to_host()[2], S.val)


def test_rmat_scale18_sampled_rows(sg):
    """The full R-MAT scale-18 squaring in the benchmark's launch
    configuration; a seeded sample of rows (including the largest-flops rows)
    is recomputed by the oracle row by row."""
    A = inputs.rmat(18)
    dA = sg.to_device(A)
    C = sg.spgemm(dA, dA, verify=True)
    fl = oracle.row_flops(A, A)
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([np.argsort(-fl)[:8], rng.choice(A.nrows, 400, replace=False)]))
    R = oracle.spgemm(rows_subset(A, rows), A)
    rp = C.rowptr.cpu().numpy()
    col = C.col.cpu().numpy()
    val = C.val.cpu().numpy()
    for t, i in enumerate(rows):
        a, b = rp[i], rp[i + 1]
        ra, rb = R.rowptr[t], R.rowptr[t + 1]
        assert b - a == rb - ra
        assert np.array_equal(col[a:b], R.col[ra:rb])
        assert np.array_equal(val[a:b], R.val[ra:rb])
    # global invariants at full size
    assert int(rp[-1]) <= int(fl.sum())
    assert np.all(np.diff(rp) <= np.minimum(fl, A.ncols))


@pytest.mark.parametrize("c", [1, 4, 16])
def test_hypersparse_kslices(sg, c):
    """k-slices multiplied as DCSR views of their nonempty rows (many rows of
    a slice are empty) give the same partials and the same merged product as
    the plain slices; row panels too."""
    A = inputs.rmat(12, seed=101)
    dA = sg.to_device(A)
    C1, P1 = sg.spgemm_kslice(dA, dA, c)
    C2, P2 = sg.spgemm_kslice(dA, dA, c, hypersparse=True)
    for a, b in zip(P1, P2):
        assert bool((a.rowptr == b.rowptr).all()) and bool((a.col == b.col).all())
        assert bool((a.val == b.val).all())
    assert bool((C1.rowptr == C2.rowptr).all()) and bool((C1.col == C2.col).all())
    assert bool((C1.val == C2.val).all())
    ids, v = sg.dcsr_view(dA)
    empty = np.diff(A.rowptr) == 0
    assert v.nrows == int((~empty).sum())
    assert np.array_equal(ids.cpu().numpy(), np.flatnonzero(~empty))
    R = oracle.spgemm(A, A)
    E = sg.dcsr_expand(sg.spgemm(v, dA), ids, A.nrows)
    assert_pattern_equal(E, R)
    assert np.array_equal(E.to_host()[2], R.val)


@pytest.mark.parametrize("idt", [np.int32, np.int64])
def test_short_rows_over_many_a_entries(sg, idt):
    """Rows of at most 32 products whose A entries are many, most of them
    pointing at empty rows of B (the table-free short-row path gathers their
    products over several batches of 32 A entries), rows of exactly 32
    products, and rows whose 32 products all land in one column."""
    rng = np.random.default_rng(41)
    n = 300
    # B rows 0..199 empty; 200..299 one entry in column 5; 300..399 one to
    # three entries in random columns
    rB, cB = [], []
    for k in range(200, 300):
        rB.append(k)
        cB.append(5)
    blen_r = rng.integers(1, 4, 100)
    for k, c in zip(range(300, 400), blen_r):
        cols = rng.choice(n, int(c), replace=False)
        rB += [k] * len(cols)
        cB += list(cols)
    B = inputs.coo_to_csr(400, n, np.array(rB), np.array(cB), rng.random(len(rB)), idt)
    blen = np.diff(B.rowptr)
    rows_A, cols_A = [], []

    def add(i, ks):
        ks = sorted(set(int(k) for k in ks))
        rows_A.extend([i] * len(ks))
        cols_A.extend(ks)

    for i in range(64):
        empty = rng.choice(200, 70, replace=False)
        if i < 16:          # a few products among many empty rows
            add(i, list(empty) + list(rng.choice(np.arange(300, 400), 6, replace=False)))
        elif i < 32:        # exactly 32 products
            ks, left = [], 32
            for k in rng.permutation(np.arange(300, 400)):
                if blen[k] <= left:
                    ks.append(k)
                    left -= blen[k]
                if left == 0:
                    break
            ks += list(range(200, 200 + left))      # one product each
            add(i, list(empty) + ks)
        elif i < 48:        # 32 products, all in column 5
            add(i, list(empty) + list(rng.choice(np.arange(200, 300), 32, replace=False)))
        else:               # half in column 5, half anywhere
            ks = list(rng.choice(np.arange(200, 300), 12, replace=False))
            ks += list(rng.choice(np.arange(300, 400), 5, replace=False))
            add(i, list(empty) + ks)
    A = inputs.coo_to_csr(64, 400, np.array(rows_A), np.array(cols_A), rng.random(len(rows_A)), idt)
    fl = oracle.row_flops(A, B)
    assert fl.max() <= 32 and (fl == 32).sum() >= 32 and np.diff(A.rowptr).min() > 32
    C, R = check_product(sg, A, B)
    assert np.array_equal(C.to_host()[2], R.val)
    assert np.all(np.diff(R.rowptr)[32:48] == 1)
    # the same rows in slot mode (learned sizing with an untrained predictor:
    # slots too small are re-run exactly)
    dA, dB = sg.to_device(A), sg.to_device(B)
    L, _ = sg.learned_multiply(dA, dB, sg.sizer_init(seed=9), 0.0)
    Lc = sg.compact(L)
    assert np.array_equal(Lc.rowptr.cpu().numpy(), R.rowptr)
    assert np.array_equal(Lc.col.cpu().numpy().astype(np.int64), R.col)
    assert np.array_equal(Lc.val.cpu().numpy(), R.val)
