"""MIS-2 aggregation on the GPU (Alg. 3) against the oracle: the same keys
(SplitMix64 on both sides) give the same set, the same number of rounds and
the same aggregates, so R matches exactly; the Galerkin product with that R
matches the oracle's."""
import numpy as np
import pytest

import oracle
from oracle import mis2 as omis2
from paper_1510_00844_gb300 import inputs
from tests.parity import assert_pattern_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


def symmetric_random(n, density, seed):
    R = inputs.random_csr(n, n, density, seed, value="u01_f64")
    rows = np.repeat(np.arange(n), np.diff(R.rowptr))
    return inputs.coo_to_csr(n, n, np.concatenate([rows, R.col]), np.concatenate([R.col, rows]),
                             np.ones(2 * R.nnz), index_dtype=np.int32)


GRAPHS = {
    "lap8": lambda: inputs.laplacian_7pt(8),
    "lap16": lambda: inputs.laplacian_7pt(16),
    "random": lambda: symmetric_random(2000, 0.003, 5),
    "rmat10": lambda: inputs.rmat(10, seed=7),
    "rmat10_i64": lambda: inputs.rmat(10, seed=7, index_dtype=np.int64),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("seed", [1, 12345])
def test_mis2_restriction_matches_oracle(sg, name, seed):
    A = GRAPHS[name]()
    R, rounds = sg.mis2_restriction(sg.to_device(A), seed)
    (rp, col, val), naggs, orounds = omis2.restriction(A, seed)
    assert rounds == orounds and R.ncols == naggs
    hrp, hcol, hval = R.to_host()
    assert np.array_equal(hrp, rp) and np.array_equal(hcol.astype(np.int64), col)
    assert np.array_equal(hval, val)


def test_galerkin_with_mis2_aggregates(sg):
    A = inputs.laplacian_7pt(16)
    dA = sg.to_device(A)
    R, _ = sg.mis2_restriction(dA, 99)
    Rt = sg.transpose(R)
    C = sg.spgemm(sg.spgemm(Rt, dA), R)
    (rp, col, val), naggs, _ = omis2.restriction(A, 99)
    Ro = inputs.CSR(A.nrows, naggs, rp, col, val)
    ref = oracle.spgemm(oracle.spgemm(oracle.transpose(Ro), A), Ro)
    assert_pattern_equal(C, ref)
    assert np.array_equal(C.to_host()[2], ref.val)     # integer-valued: exact
    assert C.nrows == C.ncols == naggs
