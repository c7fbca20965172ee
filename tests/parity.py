"""Comparison helpers shared by the GPU parity tests.

Tolerances (stated once, used everywhere):
* pattern (rowptr, columns), integer and Boolean results: bit-exact;
* float64 values: |c - c_ref| <= 1e-12 * |c_ref|, or, for entries whose terms
  cancel, <= 1e-12 * sum_k |A(i,k)| |B(k,j)|;
* float32 values against the float64 oracle: |c - c_ref| <= gamma_q *
  sum_k |A(i,k)| |B(k,j)| with gamma_q = q u / (1 - q u), u = 2^-24, q the
  number of terms of the entry plus one (each product is rounded once and each
  of the q-1 additions once) -- the standard bound for recursive summation.
"""
import numpy as np

import oracle

RTOL_F64 = 1e-12
U_F32 = 2.0 ** -24


def gpu_to_host(C):
    return C.to_host()


def assert_pattern_equal(C, R):
    rp, col, _ = C.to_host() if hasattr(C, "to_host") else (C.rowptr, C.col, C.val)
    assert np.array_equal(np.asarray(rp), np.asarray(R.rowptr)), "row pointers differ"
    assert np.array_equal(np.asarray(col, dtype=np.int64), np.asarray(R.col, dtype=np.int64)), \
        "column indices differ"


def term_counts(A, B):
    """Number of products per entry of P(A.B) (an integer product over the
    patterns, computed by the oracle on all-ones values)."""
    ones = lambda M: oracle.OCSR(M.nrows, M.ncols, M.rowptr, M.col,
                                 np.ones(len(M.col), dtype=np.int64))
    return oracle.spgemm(ones(A), ones(B)).val


def assert_values_close(C, R, A=None, B=None, dtype="f64"):
    _, _, val = C.to_host() if hasattr(C, "to_host") else (C.rowptr, C.col, C.val)
    ref = np.asarray(R.val)
    if dtype in ("i64",):
        assert np.array_equal(np.asarray(val), ref)
        return
    got = np.asarray(val, dtype=np.float64)
    err = np.abs(got - ref)
    if dtype == "f64":
        ok = err <= RTOL_F64 * np.abs(ref)
        if not ok.all():
            assert A is not None, "values differ beyond 1e-12 relative"
            scale = oracle.abs_bound(A, B)
            ok = err <= RTOL_F64 * scale
        bad = np.flatnonzero(~ok)
        assert bad.size == 0, f"{bad.size} f64 entries beyond tolerance, first {bad[:5]}"
    elif dtype == "f32":
        scale = oracle.abs_bound(A, B)
        q = term_counts(A, B).astype(np.float64) + 1.0
        gamma = q * U_F32 / (1 - q * U_F32)
        bad = np.flatnonzero(err > gamma * scale)
        assert bad.size == 0, f"{bad.size} f32 entries beyond gamma_q bound"
    else:
        raise ValueError(dtype)


def rows_subset(M, rows):
    """Host CSR of the given rows of M (data movement only)."""
    rp = np.asarray(M.rowptr)
    col = np.asarray(M.col)
    val = None if M.val is None else np.asarray(M.val)
    lens = rp[rows + 1] - rp[rows]
    nrp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=nrp[1:])
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if len(rows) else \
        np.zeros(0, dtype=np.int64)
    return oracle.OCSR(len(rows), M.ncols, nrp, col[idx].astype(np.int64),
                       None if val is None else val[idx])
