"""(min, +) and (min, select2nd) on the GPU against the oracle, bit for bit
(the min keeps the first of equal terms in ascending k on both sides): hash
and dense rows, k-slice merge, batches, learned sizing, and the NaN and
infinity cases of the min rule."""
import numpy as np
import pytest

import oracle
from paper_1510_00844_gb300 import inputs

pytestmark = pytest.mark.gpu

NAMES = {2: "min_plus", 3: "min_select2nd"}


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


def assert_equal_host(C, R):
    rp, col, val = C.to_host()
    assert np.array_equal(rp, R.rowptr)
    assert np.array_equal(col.astype(np.int64), R.col)
    assert np.array_equal(val, R.val, equal_nan=True)


@pytest.mark.parametrize("sr", [2, 3])
@pytest.mark.parametrize("value", ["u01_f64", "int"])
@pytest.mark.parametrize("gen", ["rmat12", "er", "rmat12_i64"])
def test_min_semiring_products(sg, sr, value, gen):
    A = (inputs.rmat(12, seed=81, value=value) if gen == "rmat12"
         else inputs.rmat(12, seed=81, value=value, index_dtype=np.int64) if gen == "rmat12_i64"
         else inputs.er_column_regular(4096, 12, 82, value=value))
    dA = sg.to_device(A)
    C = sg.spgemm(dA, dA, semiring=sr, verify=True)
    assert_equal_host(C, oracle.spgemm(A, A, semiring=NAMES[sr]))


@pytest.mark.parametrize("sr", [2, 3])
def test_min_semiring_kslice_merge_and_batch(sg, sr):
    A = inputs.rmat(11, seed=83)
    dA = sg.to_device(A)
    C, parts = sg.spgemm_kslice(dA, dA, 4, semiring=sr)
    assert_equal_host(C, oracle.spgemm(A, A, semiring=NAMES[sr]))
    Bs = [inputs.er_column_regular(n, d, 84 + n) for n, d in ((1000, 6), (3000, 20))]
    dBs = [sg.to_device(B) for B in Bs]
    for C, B in zip(sg.batch_spgemm(dBs, dBs, semiring=sr, verify=True), Bs):
        assert_equal_host(C, oracle.spgemm(B, B, semiring=NAMES[sr]))


def test_min_semiring_learned_sizing_is_bit_identical(sg):
    from tests.test_gpu_learned import train_small
    params = train_small(sg)[0]
    A = inputs.rmat(12, seed=85)
    dA = sg.to_device(A)
    L, _ = sg.learned_multiply(dA, dA, params, margin=0.2, semiring=2)
    P = sg.spgemm(dA, dA, semiring=2)
    Lc = sg.compact(L)
    assert bool((Lc.col == P.col).all()) and bool((Lc.val == P.val).all())


def test_min_rule_with_nan_and_infinity(sg):
    """Terms that are NaN never become the minimum; +inf terms leave the
    identity; an entry whose terms are all NaN stays +inf (same on both sides)."""
    A = inputs.random_csr(300, 300, 0.05, 86, value="u01_f64")
    B = inputs.random_csr(300, 300, 0.05, 87, value="u01_f64")
    rng = np.random.default_rng(88)
    vb = B.val.copy()
    vb[rng.random(vb.size) < 0.2] = np.nan
    vb[rng.random(vb.size) < 0.1] = np.inf
    B = inputs.CSR(B.nrows, B.ncols, B.rowptr, B.col, vb)
    dA, dB = sg.to_device(A), sg.to_device(B)
    for sr in (2, 3):
        assert_equal_host(sg.spgemm(dA, dB, semiring=sr), oracle.spgemm(A, B, semiring=NAMES[sr]))


def test_min_semiring_rejects_float32(sg):
    A = inputs.er_column_regular(512, 4, 89, value="u11_f32")
    dA = sg.to_device(A)
    with pytest.raises(sg.SpgemmError):
        sg.spgemm(dA, dA, semiring=2)


@pytest.mark.parametrize("complement", [False, True])
@pytest.mark.parametrize("sr", [0, 2, 3])
def test_masked_products(sg, complement, sr):
    """(A.B) restricted to the pattern of M or to its complement, against the
    oracle's set filter of the oracle's product."""
    A = inputs.rmat(11, seed=90, value="int" if sr == 0 else "u01_f64")
    M = inputs.random_csr(A.nrows, A.ncols, 0.02, 91, value="none", index_dtype=np.int32)
    dA, dM = sg.to_device(A), sg.to_device(M)
    C = sg.masked_spgemm(dA, dA, dM, semiring=sr, complement=complement)
    name = {0: "plus_times", 2: "min_plus", 3: "min_select2nd"}[sr]
    R = oracle.mask(oracle.spgemm(A, A, semiring=name), M, complement)
    assert_equal_host(C, R)
