"""GPU parity of the batched, device-sized and transpose paths against the
oracle: a batch of uneven products in one plan, the same batch enqueued with
no host readback, the CSR transpose, and the AMG Galerkin hierarchy captured
in one CUDA graph (checked against its closed form)."""
import numpy as np
import pytest

import oracle
from paper_1510_00844_gb300 import inputs
from tests.parity import assert_pattern_equal, assert_values_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


@pytest.mark.parametrize("value,index", [("u01_f64", np.int32), ("u11_f32", np.int64),
                                         ("int", np.int32), ("none", np.int32)])
def test_transpose(sg, value, index):
    A = inputs.random_csr(300, 500, 0.02, 5, value=value, index_dtype=index, empty_rows=0.3)
    T = sg.transpose(sg.to_device(A))
    R = oracle.transpose(A)
    rp, col, val = T.to_host()
    assert np.array_equal(rp, R.rowptr) and np.array_equal(col.astype(np.int64), R.col)
    if value != "none":
        assert np.array_equal(val, R.val)


def test_transpose_long_columns(sg):
    # R-MAT scale 16 has columns with more than 8192 entries (rank path)
    A = inputs.rmat(16)
    T = sg.transpose(sg.to_device(A))
    R = oracle.transpose(A)
    rp, col, val = T.to_host()
    assert np.diff(R.rowptr).max() > 8192
    assert np.array_equal(rp, R.rowptr) and np.array_equal(col.astype(np.int64), R.col)
    assert np.array_equal(val, R.val)


def small_batch(value="u11_f32", count=24, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(np.exp(rng.uniform(np.log(64), np.log(4096))))
        d = int(rng.integers(4, 33))
        d = min(d, n)
        A = inputs.er_column_regular(n, d, int(rng.integers(1 << 30)), value=value)
        B = inputs.er_column_regular(n, d, int(rng.integers(1 << 30)), value=value)
        out.append((A, B))
    return out


def test_batch_f32(sg):
    pairs = small_batch()
    Cs = sg.batch_spgemm([sg.to_device(A) for A, _ in pairs], [sg.to_device(B) for _, B in pairs],
                         verify=True)
    for (A, B), C in zip(pairs, Cs):
        R = oracle.spgemm(A, B)
        assert_pattern_equal(C, R)
        assert_values_close(C, R, A, B, "f32")


def test_batch_bool_and_mixed_sizes(sg):
    pairs = small_batch("none", 16, seed=4)
    Cs = sg.batch_spgemm([sg.to_device(A) for A, _ in pairs], [sg.to_device(B) for _, B in pairs],
                         semiring=1, verify=True)
    for (A, B), C in zip(pairs, Cs):
        assert C.val is None
        assert_pattern_equal(C, oracle.spgemm(A, B, semiring="or_and"))


def test_batch_with_dense_rows_bitexact(sg):
    mats = [inputs.rmat(s, seed=100 + s) for s in (9, 12, 10, 13)]
    Cs = sg.batch_spgemm([sg.to_device(M) for M in mats], [sg.to_device(M) for M in mats],
                         verify=True)
    for M, C in zip(mats, Cs):
        R = oracle.spgemm(M, M)
        assert_pattern_equal(C, R)
        assert np.array_equal(C.to_host()[2], R.val)


def test_batch_equals_single_products(sg):
    pairs = small_batch("u01_f64", 8, seed=9)
    Cs = sg.batch_spgemm([sg.to_device(A) for A, _ in pairs], [sg.to_device(B) for _, B in pairs])
    for (A, B), C in zip(pairs, Cs):
        S = sg.spgemm(sg.to_device(A), sg.to_device(B))
        assert bool((C.rowptr == S.rowptr).all()) and bool((C.col == S.col).all())
        assert bool((C.val == S.val).all())


def test_device_sized_execute_matches_host_synced(sg):
    import torch
    mats = [inputs.rmat(s, seed=200 + s) for s in (11, 12)]
    dA = [sg.to_device(M) for M in mats]
    p = sg.device_plan(dA, dA, max_row_nnz=8192)
    cap = int(sum(oracle.row_flops(M, M).sum() for M in mats))
    rowptrC = torch.empty(p.R + 1, dtype=torch.int64, device="cuda")
    colC = torch.empty(cap, dtype=torch.int32, device="cuda")
    valC = torch.empty(cap, dtype=torch.float64, device="cuda")
    for _ in range(2):
        sg.execute(p, rowptrC, cap, colC, valC)
        sg.check(p)
        Cs = sg.split_batch(p, rowptrC, colC, valC)
        for M, C in zip(mats, Cs):
            R = oracle.spgemm(M, M)
            assert_pattern_equal(C, R)
            assert np.array_equal(C.to_host()[2], R.val)


def test_device_sized_capacity_overflow_is_reported(sg):
    import torch
    M = inputs.rmat(10)
    dA = sg.to_device(M)
    p = sg.device_plan([dA], [dA], max_row_nnz=8192)
    cap = 1000
    rowptrC = torch.empty(p.R + 1, dtype=torch.int64, device="cuda")
    colC = torch.empty(cap, dtype=torch.int32, device="cuda")
    valC = torch.empty(cap, dtype=torch.float64, device="cuda")
    sg.execute(p, rowptrC, cap, colC, valC)
    with pytest.raises(sg.SpgemmError) as ei:
        sg.check(p)
    assert ei.value.status == 4
    # nnz(C) is still reported exactly
    assert int(rowptrC[-1].item()) == oracle.spgemm(M, M).nnz


@pytest.mark.parametrize("N,levels", [(16, 2), (32, 3), (128, 3)])
def test_amg_hierarchy_in_one_graph(sg, N, levels):
    import torch
    from paper_1510_00844_gb300 import amg
    A0 = inputs.laplacian_7pt(N)
    Rs = [inputs.aggregation_2x2x2(N >> l) for l in range(levels)]
    s = torch.cuda.Stream()
    chain = amg.GalerkinChain(sg.to_device(A0), [sg.to_device(R) for R in Rs], s)
    chain.capture()
    for _ in range(2):
        chain.replay()
        torch.cuda.synchronize()
        chain.check()
        A = A0
        for l, (C, T) in enumerate(zip(chain.results(), chain.intermediates())):
            ref_T = oracle.spgemm(oracle.transpose(Rs[l]), A)
            assert_pattern_equal(T, ref_T)
            assert np.array_equal(T.to_host()[2], ref_T.val)
            L = inputs.laplacian_7pt(N >> (l + 1))
            rp, col, val = C.to_host()
            assert np.array_equal(rp, L.rowptr) and np.array_equal(col, L.col)
            assert np.array_equal(val, L.val * 4.0 ** (l + 1))   # Galerkin closed form
            A = inputs.CSR(C.nrows, C.ncols, rp, col, val)


def test_distributed_kslice_on_one_rank(sg, tmp_path):
    """The k-split path of the multi-GPU module with the library's kernels on
    a one-rank group: the exchange is empty, partial + merge give the product."""
    import torch
    import torch.distributed as dist
    from paper_1510_00844_gb300 import distributed
    store = dist.FileStore(str(tmp_path / "store"), 1)
    dist.init_process_group("gloo", store=store, rank=0, world_size=1)
    try:
        A = inputs.rmat(11, seed=61)
        dA = sg.to_device(A)
        r0, r1, (rp, col, val) = distributed.gpu_kslice_product(dA, dA)
        C = sg.spgemm(dA, dA)
        assert (r0, r1) == (0, A.nrows)
        assert bool((rp == C.rowptr).all()) and bool((col == C.col).all())
        assert bool((val == C.val).all())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("panels,semiring", [(1, 0), (3, 0), (8, 0), (5, 1)])
def test_product_to_host_in_panels(sg, panels, semiring):
    """Row panels computed one after another with the copy of each panel to
    pinned host memory overlapping the next one's numeric phase: the host
    arrays equal the device product."""
    from paper_1510_00844_gb300 import pipeline
    A = inputs.rmat(12, seed=71)
    dA = sg.to_device(A)
    H = pipeline.spgemm_to_host(dA, dA, semiring=semiring, panels=panels)
    C = sg.spgemm(dA, dA, semiring=semiring)
    assert np.array_equal(H.rowptr.numpy(), C.rowptr.cpu().numpy())
    assert np.array_equal(H.col[:H.nnz].numpy(), C.col.cpu().numpy())
    if semiring == 0:
        assert np.array_equal(H.val[:H.nnz].numpy(), C.val.cpu().numpy())
    H2 = pipeline.spgemm_to_host(dA, dA, semiring=semiring, panels=panels + 1, out=H)
    assert H2 is H and np.array_equal(H2.col[:H2.nnz].numpy(), C.col.cpu().numpy())


def test_pinned_host_arrays(sg):
    """pipeline.pinned_empty: page-locked (registered) host memory of the
    requested size and type, usable as a copy target, released when freed."""
    import gc
    import torch
    from paper_1510_00844_gb300 import pipeline
    for dtype, numel in ((torch.float64, 1000), (torch.int32, 3), (torch.int64, 0)):
        h = pipeline.pinned_empty(numel, dtype)
        assert h.dtype == dtype and h.numel() == numel and h.is_contiguous()
        assert numel == 0 or h.is_pinned()
        if numel:
            d = torch.arange(numel, device="cuda").to(dtype)
            h.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
            assert torch.equal(h, d.cpu())
        del h
        gc.collect()


def test_batch_captured_in_a_graph(sg):
    """A batch of uneven products as one device-sized plan captured in a CUDA
    graph: replays give the host-synced batch's result bit for bit."""
    import torch
    pairs = inputs.batched_er(24, nmin=256, nmax=4096)
    As = [sg.to_device(a) for a, _ in pairs]
    Bs = [sg.to_device(b) for _, b in pairs]
    cap = int(sg.batch_plan(As, Bs).info()["flops"])
    s = torch.cuda.Stream()
    p = sg.device_plan(As, Bs, stream=s, max_row_nnz=4096)
    rowptrC = torch.empty(p.R + 1, dtype=torch.int64, device="cuda")
    colC = torch.empty(cap, dtype=As[0].col.dtype, device="cuda")
    valC = torch.empty(cap, dtype=As[0].val.dtype, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sg.execute(p, rowptrC, cap, colC, valC)
    ref = sg.batch_spgemm(As, Bs)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        sg.check(p)
        for C, R in zip(sg.split_batch(p, rowptrC, colC, valC), ref):
            assert bool((C.col == R.col).all()) and bool((C.val == R.val).all())


def test_full_batch_of_512_products_sampled(sg):
    """The full batched workload (512 uneven ER products, f32) with one plan;
    a seeded sample of products, always including the largest, is checked
    against the oracle (pattern exact, values within the f32 summation
    bound)."""
    pairs = inputs.batched_er(512)
    As = [sg.to_device(a) for a, _ in pairs]
    Bs = [sg.to_device(b) for _, b in pairs]
    Cs = sg.batch_spgemm(As, Bs, verify=True)
    sizes = np.array([a.nrows for a, _ in pairs])
    rng = np.random.default_rng(11)
    pick = np.unique(np.concatenate([np.argsort(-sizes)[:2], rng.choice(512, 10, replace=False)]))
    for q in pick:
        a, b = pairs[q]
        R = oracle.spgemm(a, b)
        assert_pattern_equal(Cs[q], R)
        assert_values_close(Cs[q], R, a, b, dtype="f32")


def test_split3d_on_one_rank(sg, tmp_path):
    """Alg. 2 with the library's kernels on a 1 x 1 x 1 grid: the broadcasts
    and all-to-alls reach only this rank; the result is the product."""
    import torch
    import torch.distributed as dist
    from paper_1510_00844_gb300 import split3d as s3
    store = dist.FileStore(str(tmp_path / "store3d"), 1)
    dist.init_process_group("gloo", store=store, rank=0, world_size=1)
    try:
        A = inputs.rmat(10, seed=63)
        dA = sg.to_device(A)
        P = (A.nrows, A.ncols, dA.rowptr, dA.col, dA.val)
        multiply, merge = s3.gpu_ops()
        grid = s3.Grid(1, 1)
        m, n, rp, col, val = s3.split3d(grid, P, P, (A.nrows, A.ncols, A.ncols), multiply, merge,
                                        dA.col.dtype, dA.val.dtype, torch.device("cuda"))
        C = sg.spgemm(dA, dA)
        assert bool((rp == C.rowptr).all()) and bool((col == C.col).all())
        assert bool((val == C.val).all())
    finally:
        dist.destroy_process_group()
