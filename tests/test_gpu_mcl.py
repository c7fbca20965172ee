"""MCL epilogue on the GPU against the oracle, step by step: each GPU step's
input is the previous GPU output, the oracle prunes and renormalises the same
product.  Entries within 1e-12 (relative) of the threshold could fall on
either side of it; none may differ otherwise."""
import numpy as np
import pytest

import oracle
from paper_1510_00844_gb300 import inputs
from tests.parity import assert_pattern_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


@pytest.mark.parametrize("scale,steps,thr", [(10, 3, 1e-4), (10, 3, 1e-2), (14, 2, 1e-4)])
def test_mcl_steps_match_oracle(sg, scale, steps, thr):
    M = inputs.mcl_transition(scale)
    dM = sg.to_device(M)
    for step in range(steps):
        hostM = oracle.OCSR(M.nrows, M.ncols, *dM.to_host())
        C = sg.spgemm(dM, dM)
        R = oracle.mcl_prune_renorm(oracle.spgemm(hostM, hostM), thr)
        dM = sg.mcl_prune(C, thr)
        rp, col, val = dM.to_host()
        assert np.array_equal(rp, R.rowptr) and np.array_equal(col.astype(np.int64), R.col)
        np.testing.assert_allclose(val, R.val, rtol=1e-12)
        nz = np.diff(rp) > 0
        sums = np.add.reduceat(val, rp[:-1][nz]) if nz.any() else np.zeros(0)
        np.testing.assert_allclose(sums, 1.0, rtol=1e-12)


def test_mcl_on_slot_view_and_learned(sg):
    import torch
    M = inputs.mcl_transition(9)
    dM = sg.to_device(M)
    params = sg.sizer_init(seed=5)      # an untrained predictor: slots miss often
    A = sg.mcl_step(dM, 1e-3)
    B = sg.mcl_step(dM, 1e-3, params=params, margin=0.0)
    assert bool((A.rowptr == B.rowptr).all()) and bool((A.col == B.col).all())
    assert bool((A.val == B.val).all())
