"""The full R-MAT scale-18 squaring (the benchmark's workload: Graph500
parameters, edge factor 16, f64, int32) checked against the oracle on EVERY
row, one row panel at a time.  Each panel is the library's row-panel view of
A times A; the oracle multiplies the same rows.  Columns must be equal and
values equal bit for bit (both sides add each output's products in
ascending k).  Working one panel at a time keeps host memory to a few GB
where the whole C is 35.5 GB."""
import numpy as np
import pytest

import oracle
from paper_1510_00844_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_rmat18_every_row_streamed_by_panel():
    import torch
    from paper_1510_00844_gb300 import spgemm as sg
    A = inputs.rmat(18)
    dA = sg.to_device(A)
    rp = np.asarray(A.rowptr)
    npan = 16
    total = 0
    for p in range(npan):
        a, b = (A.nrows * p) // npan, (A.nrows * (p + 1)) // npan
        view = sg.DeviceCSR(b - a, A.ncols, dA.rowptr[a:b], dA.col, dA.val,
                            rowend=dA.rowptr[a + 1:b + 1])
        C = sg.spgemm(view, dA, verify=True)
        sub = inputs.CSR(b - a, A.ncols, rp[a:b + 1] - rp[a], A.col[rp[a]:rp[b]],
                         A.val[rp[a]:rp[b]])
        R = oracle.spgemm(sub, A)
        crp = C.rowptr.cpu().numpy()
        assert np.array_equal(crp, R.rowptr), f"panel {p}: row counts differ"
        assert np.array_equal(C.col.cpu().numpy().astype(np.int64), R.col), f"panel {p}: columns"
        assert np.array_equal(C.val.cpu().numpy(), R.val), f"panel {p}: values"
        total += int(crp[-1])
        del C, R
        torch.cuda.empty_cache()
    assert total == 2_958_724_919
