"""ctypes front end of the C oracle plus the plain numpy parts.

TEST INFRASTRUCTURE ONLY (see the package docstring)."""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, NamedTuple, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

F64, I64, BOOL = 0, 1, 2
MINPLUS_F64, MINPLUS_I64, MINSEL_F64, MINSEL_I64 = 3, 4, 5, 6
SEMIRINGS = ("plus_times", "or_and", "min_plus", "min_select2nd")


class OCSR(NamedTuple):
    nrows: int
    ncols: int
    rowptr: np.ndarray   # int64
    col: np.ndarray      # int64
    val: Optional[np.ndarray]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile spa_oracle.c with gcc (OpenMP when available, never FMA)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int64
        lib.oracle_row_flops.restype = I
        lib.oracle_row_flops.argtypes = [I, P, P, P, P]
        lib.oracle_spgemm_count.restype = I
        lib.oracle_spgemm_count.argtypes = [I, I, P, P, P, P, P, ctypes.c_int]
        lib.oracle_spgemm_fill.restype = ctypes.c_int
        lib.oracle_spgemm_fill.argtypes = [I, I, P, P, P, P, P, P, ctypes.c_int, P, P, P,
                                           ctypes.c_int]
        lib.oracle_sum_count.restype = I
        lib.oracle_sum_count.argtypes = [ctypes.c_int, I, I, P, P, P, ctypes.c_int]
        lib.oracle_sum_fill.restype = ctypes.c_int
        lib.oracle_sum_fill.argtypes = [ctypes.c_int, I, I, P, P, P, ctypes.c_int, P, P, P,
                                        ctypes.c_int]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def num_threads(nthreads: int = 0) -> int:
    return int(_load().oracle_num_threads(nthreads))


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _vtype(val, semiring: str) -> int:
    if semiring not in SEMIRINGS:
        raise ValueError(f"unknown semiring {semiring}")
    if semiring == "or_and" or val is None:
        return BOOL
    integer = np.issubdtype(val.dtype, np.integer)
    if semiring == "min_plus":
        return MINPLUS_I64 if integer else MINPLUS_F64
    if semiring == "min_select2nd":
        return MINSEL_I64 if integer else MINSEL_F64
    return I64 if integer else F64


def _is_int(vt) -> bool:
    return vt in (I64, MINPLUS_I64, MINSEL_I64)


def _vals(val, vt):
    if vt == BOOL:
        return None
    if _is_int(vt):
        return np.ascontiguousarray(val, dtype=np.int64)
    return np.ascontiguousarray(val, dtype=np.float64)   # float32 inputs are upcast


def _idx(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


def row_flops(A, B) -> np.ndarray:
    """flops_i = sum over k in A(i,:) of nnz(B(k,:)) (Sec. 2)."""
    out = np.zeros(A.nrows, dtype=np.int64)
    rpA, ciA, rpB = _idx(A.rowptr), _idx(A.col), _idx(B.rowptr)
    _load().oracle_row_flops(A.nrows, _p(rpA), _p(ciA), _p(rpB), _p(out))
    return out


def spgemm(A, B, semiring: str = "plus_times", nthreads: int = 0) -> OCSR:
    """C = A.B by Gustavson with a dense accumulator (Alg. 1).  Values are
    float64 (float32 operands are upcast), int64 (wraparound) or none
    (semiring "or_and" or pattern-only operands)."""
    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    lib = _load()
    vt = _vtype(A.val, semiring)
    if vt != BOOL and B.val is None:
        vt = BOOL
    m, n = A.nrows, B.ncols
    rpA, ciA, rpB, ciB = _idx(A.rowptr), _idx(A.col), _idx(B.rowptr), _idx(B.col)
    vA, vB = _vals(A.val, vt), _vals(B.val, vt)
    cnt = np.zeros(m, dtype=np.int64)
    nnz = lib.oracle_spgemm_count(m, n, _p(rpA), _p(ciA), _p(rpB), _p(ciB), _p(cnt), nthreads)
    if nnz < 0:
        raise MemoryError("oracle: out of memory")
    rpC = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(cnt, out=rpC[1:])
    ciC = np.empty(nnz, dtype=np.int64)
    vC = None if vt == BOOL else np.empty(nnz, dtype=np.int64 if _is_int(vt) else np.float64)
    st = lib.oracle_spgemm_fill(m, n, _p(rpA), _p(ciA), _p(vA), _p(rpB), _p(ciB), _p(vB), vt,
                                _p(rpC), _p(ciC), _p(vC), nthreads)
    if st != 0:
        raise RuntimeError(f"oracle fill failed ({st})")
    return OCSR(m, n, rpC, ciC, vC)


def abs_bound(A, B, nthreads: int = 0) -> np.ndarray:
    """sum_k |A(i,k)| |B(k,j)| per entry of P(C): the scale of the rounding
    error bound for entries that cancel."""
    absA = OCSR(A.nrows, A.ncols, A.rowptr, A.col, np.abs(np.asarray(A.val, dtype=np.float64)))
    absB = OCSR(B.nrows, B.ncols, B.rowptr, B.col, np.abs(np.asarray(B.val, dtype=np.float64)))
    return spgemm(absA, absB, nthreads=nthreads).val


def sum_partials(parts: List, semiring: str = "plus_times", nthreads: int = 0) -> OCSR:
    """C = (+)_{s ascending} C_s entrywise: what the multiway merge with
    duplicate reduction (Sec. 4.3) returns."""
    c = len(parts)
    m, n = parts[0].nrows, parts[0].ncols
    vt = _vtype(parts[0].val, semiring)
    rps = [_idx(P.rowptr) for P in parts]
    cis = [_idx(P.col) for P in parts]
    vs = [_vals(P.val, vt) for P in parts]
    arr_p = ctypes.c_void_p * c
    rp_arr = arr_p(*[_p(a) for a in rps])
    ci_arr = arr_p(*[_p(a) for a in cis])
    v_arr = arr_p(*[_p(a) for a in vs]) if vt != BOOL else None
    lib = _load()
    cnt = np.zeros(m, dtype=np.int64)
    nnz = lib.oracle_sum_count(c, m, n, ctypes.cast(rp_arr, ctypes.c_void_p),
                               ctypes.cast(ci_arr, ctypes.c_void_p), _p(cnt), nthreads)
    if nnz < 0:
        raise MemoryError("oracle: out of memory")
    rpC = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(cnt, out=rpC[1:])
    ciC = np.empty(nnz, dtype=np.int64)
    vC = None if vt == BOOL else np.empty(nnz, dtype=np.int64 if _is_int(vt) else np.float64)
    st = lib.oracle_sum_fill(c, m, n, ctypes.cast(rp_arr, ctypes.c_void_p),
                             ctypes.cast(ci_arr, ctypes.c_void_p),
                             None if v_arr is None else ctypes.cast(v_arr, ctypes.c_void_p), vt,
                             _p(rpC), _p(ciC), _p(vC), nthreads)
    if st != 0:
        raise RuntimeError(f"oracle sum failed ({st})")
    return OCSR(m, n, rpC, ciC, vC)


def mask(C, M, complement: bool = False) -> OCSR:
    """Entries (i, j) of C with j in M(i,:) (or not in it, complement): the
    structural mask MIS-2 applies to its products (Alg. 3), as a set filter
    row by row."""
    rpC, ciC = _idx(C.rowptr), _idx(C.col)
    rpM, ciM = _idx(M.rowptr), _idx(M.col)
    keep = np.zeros(ciC.size, dtype=bool)
    for i in range(C.nrows):
        a, b = rpC[i], rpC[i + 1]
        keep[a:b] = np.isin(ciC[a:b], ciM[rpM[i]:rpM[i + 1]]) != complement
    rows = np.repeat(np.arange(C.nrows), np.diff(rpC))[keep]
    rp = np.zeros(C.nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=C.nrows), out=rp[1:])
    val = None if C.val is None else np.asarray(C.val)[keep]
    return OCSR(C.nrows, C.ncols, rp, ciC[keep], val)


def kslice_bounds(l: int, c: int) -> List[tuple]:
    """K_s = [floor(s l / c), floor((s+1) l / c)), s = 0..c-1: contiguous,
    equal-size ranges of the inner dimension (the split distribution of
    Sec. 4.1 / Alg. 2); empty ranges are allowed when c > l."""
    return [((s * l) // c, ((s + 1) * l) // c) for s in range(c)]


def kslice(A, B, c: int):
    """The c partial problems (A(:,K_s), B(K_s,:)) with original indices kept."""
    out = []
    rowsA = np.repeat(np.arange(A.nrows, dtype=np.int64), np.diff(_idx(A.rowptr)))
    colA = _idx(A.col)
    lenB = np.diff(_idx(B.rowptr))
    for lo, hi in kslice_bounds(A.ncols, c):
        keep = (colA >= lo) & (colA < hi)
        cnt = np.bincount(rowsA[keep], minlength=A.nrows)
        rp = np.zeros(A.nrows + 1, dtype=np.int64)
        np.cumsum(cnt, out=rp[1:])
        As = OCSR(A.nrows, A.ncols, rp, colA[keep], None if A.val is None else A.val[keep])
        bl = lenB.copy()
        bl[:lo] = 0
        bl[hi:] = 0
        rpb = np.zeros(B.nrows + 1, dtype=np.int64)
        np.cumsum(bl, out=rpb[1:])
        b0, b1 = int(B.rowptr[lo]), int(B.rowptr[hi])
        Bs = OCSR(B.nrows, B.ncols, rpb, _idx(B.col)[b0:b1],
                  None if B.val is None else B.val[b0:b1])
        out.append((As, Bs))
    return out


def transpose(A) -> OCSR:
    """A^T in CSR with sorted rows: entry (i, j, v) -> (j, i, v)."""
    rows = np.repeat(np.arange(A.nrows, dtype=np.int64), np.diff(_idx(A.rowptr)))
    cols = _idx(A.col)
    order = np.lexsort((rows, cols))
    cnt = np.bincount(cols, minlength=A.ncols)
    rp = np.zeros(A.ncols + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    return OCSR(A.ncols, A.nrows, rp, rows[order], None if A.val is None else A.val[order])


def mcl_prune_renorm(C, threshold: float = 1e-4) -> OCSR:
    """One Markov-clustering epilogue on M^T stored in CSR (rows of M^T are
    columns of M): drop entries strictly below ``threshold``, then divide each
    row by the sum of its kept entries (summed left to right)."""
    rp = _idx(C.rowptr)
    val = np.asarray(C.val, dtype=np.float64)
    keep = val >= threshold
    rows = np.repeat(np.arange(C.nrows, dtype=np.int64), np.diff(rp))
    cnt = np.bincount(rows[keep], minlength=C.nrows)
    rpo = np.zeros(C.nrows + 1, dtype=np.int64)
    np.cumsum(cnt, out=rpo[1:])
    kv = val[keep]
    col = _idx(C.col)[keep]
    out = np.empty_like(kv)
    for i in range(C.nrows):
        a, b = rpo[i], rpo[i + 1]
        s = 0.0
        for t in range(a, b):
            s = s + kv[t]
        for t in range(a, b):
            out[t] = kv[t] / s
    return OCSR(C.nrows, C.ncols, rpo, col, out)
