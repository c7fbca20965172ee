"""The allocation-free merge count, spgemm_merge_symbolic_static.

Some callers may not allocate device memory at all (a fixed device-memory
budget reserved at start-up, or an interface that passes only inputs and
outputs), so this entry point takes no workspace and uses the library's fixed
device scratch array instead.  It must give exactly the row pointers and
nnz(C) of the workspace-based spgemm_merge_symbolic, on repeated calls (the
scratch array keeps the previous call's contents, so the second call checks
that nothing stale leaks in).  Collected last so that a stop-at-first-failure
run has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1510_00844_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


@pytest.mark.parametrize("c,scale", [(4, 12), (3, 10)])
def test_static_merge_count_matches_workspace_version(sg, c, scale):
    import torch
    A = inputs.rmat(scale)
    dA = sg.to_device(A)
    parts = [sg.spgemm(As, dA) for As in sg.kslice_views(dA, c)]
    ws = sg.merge_workspace(c, A.nrows, A.ncols, dA.rowptr.device)
    ref_rp, ref_nnz = sg.merge_symbolic(parts, ws)
    ref = ref_rp.cpu().numpy()
    arr = sg._parts(parts)
    opts = sg._Opts(0, 0)
    rp = torch.full((A.nrows + 1,), -7, dtype=torch.int64, device=dA.rowptr.device)
    free_before = None
    for it in range(2):
        # called through the C ABI directly
        rp.fill_(-7)
        torch.cuda.synchronize()
        if it == 1:
            free_before = torch.cuda.mem_get_info()[0]
        nnz = ctypes.c_int64(-1)
        st = sg._lib.spgemm_merge_symbolic_static(
            c, arr, ctypes.byref(opts), sg._stream(), ctypes.c_void_p(rp.data_ptr()),
            ctypes.byref(nnz))
        assert st == 0, sg._lib.spgemm_last_error()
        torch.cuda.synchronize()
        if it == 1:
            # the second (warm) call took no device memory: any allocation
            # would take at least one 2 MB page from the free pool
            assert torch.cuda.mem_get_info()[0] == free_before
        assert nnz.value == ref_nnz
        assert np.array_equal(rp.cpu().numpy(), ref)


def test_static_merge_count_rejects_oversize(sg):
    import torch
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    big = sg._Csr((1 << 24) + 1, 10, 0, rp.data_ptr(), None, None, None, 0, 0)
    arr = (sg._Csr * 1)(big)
    nnz = ctypes.c_int64()
    st = sg._lib.spgemm_merge_symbolic_static(1, arr, None, None,
                                              ctypes.c_void_p(rp.data_ptr()), ctypes.byref(nnz))
    assert st == 1
    assert b"16777216" in sg._lib.spgemm_last_error()


def test_static_merge_count_checks_like_workspace_version(sg):
    """Both entry points reject a min semiring on float32 parts."""
    import torch
    A = inputs.rmat(8)
    A32 = inputs.CSR(A.nrows, A.ncols, A.rowptr, A.col, A.val.astype(np.float32))
    dA = sg.to_device(A32)
    arr = sg._parts([dA, dA])
    opts = sg._Opts(sg.MIN_PLUS, 0)
    rp = torch.zeros(A.nrows + 1, dtype=torch.int64, device="cuda")
    nnz = ctypes.c_int64()
    st = sg._lib.spgemm_merge_symbolic_static(2, arr, ctypes.byref(opts), sg._stream(),
                                              ctypes.c_void_p(rp.data_ptr()), ctypes.byref(nnz))
    ws = sg.merge_workspace(2, A.nrows, A.ncols, rp.device)
    st_ws = sg._lib.spgemm_merge_symbolic(2, arr, ctypes.byref(opts), sg._stream(),
                                          ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                          ctypes.c_void_p(rp.data_ptr()), ctypes.byref(nnz))
    assert st == st_ws == 7                      # NOT_SUPPORTED on both
