"""Persistent chains (spgemm_chain_*): many device-sized products in one
kernel launch with device-side barriers between phases.

* A chain gives the same bits as spgemm_execute on each plan and as the
  oracle: single products with dense and hash rows, a batch of uneven
  products, Boolean products, and the AMG Galerkin hierarchy (products that
  read the previous product's output), which also meets its closed form.
* A chain captured in a CUDA graph replays correctly.
* Stage stamps (record_stages) cover every barrier, in order.
* The bounded wait: with one stage's completion withheld, every block gives
  up after the timeout, spgemm_chain_check reports TIMEOUT, and the context
  stays usable (the same chain then runs normally)."""
import time

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


def _outputs(sg, p, cap, idt, vdt):
    import torch
    rowptrC = torch.empty(p.R + 1, dtype=torch.int64, device="cuda")
    colC = torch.empty(max(cap, 1), dtype=idt, device="cuda")
    valC = None if vdt is None else torch.empty(max(cap, 1), dtype=vdt, device="cuda")
    return rowptrC, colC, valC


@pytest.mark.parametrize("scale,idt,threads", [(12, np.int32, 0), (11, np.int64, 0),
                                               (12, np.int32, 1024), (11, np.int64, 1024)])
def test_chain_single_product_with_dense_rows(sg, scale, idt, threads):
    import torch
    M = inputs.rmat(scale, seed=210 + scale, index_dtype=idt)
    dA = sg.to_device(M)
    p = sg.device_plan([dA], [dA], max_row_nnz=8192)
    assert sg.plan(dA, dA).info()["rows_dense"] > 0
    cap = int(oracle.row_flops(M, M).sum())
    rp, col, val = _outputs(sg, p, cap, dA.col.dtype, torch.float64)
    ch = sg.Chain([(p, rp, cap, col, val)], record_stages=True, block_threads=threads)
    R = oracle.spgemm(M, M)
    for _ in range(2):
        col.fill_(-1)
        ch.launch()
        ch.check()
        C = sg.split_batch(p, rp, col, val)[0]
        assert_pattern_equal(C, R)
        assert np.array_equal(C.to_host()[2], R.val)
    assert ch.grid() >= 1
    # stage stamps: every barrier passed, in order
    st = ch.stage_ms()
    assert [n for _, n, _ in st] == ["clear"] + list(sg.CHAIN_STAGES)
    assert all(ms >= 0.0 for _, _, ms in st)
    assert sum(ms for _, _, ms in st) > 0.0


@pytest.mark.parametrize("threads", [0, 1024])
def test_chain_batch_matches_execute(sg, threads):
    """A batch of uneven float32 products as one chain step and a Boolean
    copy as a second step: bit-identical to spgemm_execute, with either
    block size."""
    import torch
    pairs = inputs.batched_er(40, nmin=256, nmax=8192)
    As = [sg.to_device(a) for a, _ in pairs]
    Bs = [sg.to_device(b) for _, b in pairs]
    cap = int(sg.batch_plan(As, Bs).info()["flops"])
    p = sg.device_plan(As, Bs, max_row_nnz=4096)
    rp, col, val = _outputs(sg, p, cap, As[0].col.dtype, torch.float32)
    ch = sg.Chain([(p, rp, cap, col, val)], block_threads=threads)
    ch.launch()
    ch.check()
    q = sg.device_plan(As, Bs, max_row_nnz=4096)
    rp2, col2, val2 = _outputs(sg, q, cap, As[0].col.dtype, torch.float32)
    sg.execute(q, rp2, cap, col2, val2)
    sg.check(q)
    nnz = int(rp[-1].item())
    assert torch.equal(rp, rp2)
    assert torch.equal(col[:nnz], col2[:nnz])
    assert torch.equal(val[:nnz].view(torch.int32), val2[:nnz].view(torch.int32))
    # the pattern-only copy
    Ap = [sg.DeviceCSR(a.nrows, a.ncols, a.rowptr, a.col, None) for a in As]
    Bp = [sg.DeviceCSR(b.nrows, b.ncols, b.rowptr, b.col, None) for b in Bs]
    pb = sg.device_plan(Ap, Bp, semiring=sg.OR_AND, max_row_nnz=4096)
    rpb, colb, _ = _outputs(sg, pb, cap, As[0].col.dtype, None)
    chb = sg.Chain([(pb, rpb, cap, colb, None)], block_threads=threads)
    chb.launch()
    chb.check()
    assert torch.equal(rpb, rp) and torch.equal(colb[:nnz], col[:nnz])


@pytest.mark.parametrize("N,levels,threads", [(32, 3, 768), (128, 3, 1024)])
def test_chain_galerkin_hierarchy(sg, N, levels, threads):
    """R^T A then (R^T A) R on every level, six dependent products in one
    launch, replayed from a CUDA graph: the same bits as the launch-by-launch
    graph, and the closed form 4^l x Laplacian of the coarse grid."""
    import torch
    from paper_1510_00844_gb300 import amg
    A0 = inputs.laplacian_7pt(N)
    Rs = [inputs.aggregation_2x2x2(N >> l) for l in range(levels)]
    dA0 = sg.to_device(A0)
    dRs = [sg.to_device(R) for R in Rs]
    s = torch.cuda.Stream()
    pc = amg.GalerkinChain(dA0, dRs, s, persistent=True, block_threads=threads)
    pc.capture()
    ref = amg.GalerkinChain(dA0, dRs, s)
    ref.capture()
    ref.replay()
    torch.cuda.synchronize()
    ref.check()
    for _ in range(2):
        pc.replay()
        torch.cuda.synchronize()
        pc.check()
        for C, D in zip(pc.results() + pc.intermediates(), ref.results() + ref.intermediates()):
            assert torch.equal(C.rowptr, D.rowptr) and torch.equal(C.col, D.col)
            assert torch.equal(C.val, D.val)
        for l, C in enumerate(pc.results()):
            L = inputs.laplacian_7pt(N >> (l + 1))
            rp, col, val = C.to_host()
            assert np.array_equal(rp, L.rowptr) and np.array_equal(col, L.col)
            assert np.array_equal(val, L.val * 4.0 ** (l + 1))


def test_chain_timeout_when_a_stage_is_withheld(sg):
    """No block signals the end of stage 3 (the symbolic stage of the first
    product): the wait after it expires after the 0.2 s limit, the kernel
    returns, the check reports TIMEOUT; then the chain runs normally."""
    import torch
    M = inputs.rmat(10, seed=5)
    dA = sg.to_device(M)
    p = sg.device_plan([dA], [dA], max_row_nnz=8192)
    cap = int(oracle.row_flops(M, M).sum())
    rp, col, val = _outputs(sg, p, cap, dA.col.dtype, torch.float64)
    stuck = sg.Chain([(p, rp, cap, col, val)], timeout_s=0.2, withhold_stage=3)
    t0 = time.perf_counter()
    stuck.launch()
    with pytest.raises(sg.SpgemmError) as ei:
        stuck.check()
    assert ei.value.status == 5                     # SPGEMM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    ok = sg.Chain([(p, rp, cap, col, val)], timeout_s=5.0)
    ok.launch()
    ok.check()
    C = sg.split_batch(p, rp, col, val)[0]
    R = oracle.spgemm(M, M)
    assert_pattern_equal(C, R)
    assert np.array_equal(C.to_host()[2], R.val)


def test_chain_rejects_other_block_sizes(sg):
    import torch
    M = inputs.rmat(8, seed=3)
    dA = sg.to_device(M)
    p = sg.device_plan([dA], [dA], max_row_nnz=8192)
    cap = int(oracle.row_flops(M, M).sum())
    rp, col, val = _outputs(sg, p, cap, dA.col.dtype, torch.float64)
    with pytest.raises(sg.SpgemmError) as ei:
        sg.Chain([(p, rp, cap, col, val)], block_threads=512)
    assert ei.value.status == 1                     # SPGEMM_ERR_INVALID_ARG
