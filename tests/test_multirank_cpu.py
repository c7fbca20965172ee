"""Host logic of the multi-GPU path on CPU ranks (gloo, world size 2): row
panels of A cover every row once, their products (computed here by the
oracle, one panel per rank) concatenate to the full product, and the timing
reductions the benchmark uses (max of times, sum of flops) behave."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_panels_partition_rows():
    for m in (0, 1, 7, 262144):
        for world in (1, 2, 3, 8):
            bounds = [bench.panel(m, world, r) for r in range(world)]
            assert bounds[0][0] == 0 and bounds[-1][1] == m
            assert all(bounds[r][1] == bounds[r + 1][0] for r in range(world - 1))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch
    import oracle
    from paper_1510_00844_gb300 import inputs
    from tests.parity import rows_subset
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = inputs.rmat(10)
    r0, r1 = bench.panel(A.nrows, world, rank)
    C = oracle.spgemm(rows_subset(A, np.arange(r0, r1)), A)
    parts = [None] * world
    dist.all_gather_object(parts, (r0, r1, C.rowptr, C.col, C.val))
    t = torch.tensor([float(10 + rank)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    f = torch.tensor([float(C.nnz)], dtype=torch.float64)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    if rank == 0:
        full = oracle.spgemm(A, A)
        rp = [np.zeros(1, dtype=np.int64)]
        cols, vals, off = [], [], 0
        for (a, b, prp, pc, pv) in sorted(parts, key=lambda x: x[0]):
            rp.append(prp[1:] + off)
            off += prp[-1]
            cols.append(pc)
            vals.append(pv)
        ok = (np.array_equal(np.concatenate(rp), full.rowptr)
              and np.array_equal(np.concatenate(cols), full.col)
              and np.array_equal(np.concatenate(vals), full.val)
              and t.item() == 10 + world - 1 and f.item() == full.nnz)
        with open(out_path, "w") as fh:
            fh.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_row_panels_over_gloo(tmp_path):
    out = tmp_path / "result.txt"
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(out)), nprocs=world,
                       start_method="spawn", join=True)
    assert out.read_text() == "ok"


def _kslice_worker(rank, world, port, out_path):
    import torch
    import oracle
    from paper_1510_00844_gb300 import distributed, inputs
    from tests.parity import rows_subset
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = inputs.rmat(10)
    slices = oracle.kslice(A, A, world)

    def partial(s, w):
        C = oracle.spgemm(*slices[s])          # the local multiply of slice s
        return (torch.from_numpy(C.rowptr.astype(np.int64)),
                torch.from_numpy(C.col.astype(A.col.dtype)), torch.from_numpy(C.val))

    def merge(pieces):
        rows = pieces[0][0].numel() - 1
        parts = [inputs.CSR(rows, A.ncols, p[0].numpy(), p[1].numpy(), p[2].numpy())
                 for p in pieces]
        C = oracle.sum_partials(parts)         # the merge, ascending s
        return (torch.from_numpy(C.rowptr.astype(np.int64)),
                torch.from_numpy(C.col.astype(A.col.dtype)), torch.from_numpy(C.val))

    col_dtype = torch.from_numpy(np.zeros(0, dtype=A.col.dtype)).dtype
    r0, r1, (rp, col, val) = distributed.kslice_product(A.nrows, partial, merge, col_dtype,
                                                        torch.float64, torch.device("cpu"))
    ref = oracle.sum_partials([oracle.spgemm(*ks) for ks in slices])
    mine = rows_subset(ref, np.arange(r0, r1))
    full = rows_subset(oracle.spgemm(A, A), np.arange(r0, r1))
    ok = ((r0, r1) == distributed.panel(A.nrows, world, rank)
          and np.array_equal(rp.numpy(), mine.rowptr) and np.array_equal(col.numpy(), mine.col)
          and np.array_equal(val.numpy(), mine.val)
          and np.array_equal(rp.numpy(), full.rowptr) and np.array_equal(col.numpy(), full.col)
          and np.allclose(val.numpy(), full.val, rtol=1e-12, atol=0))
    flags = [None] * world
    dist.all_gather_object(flags, bool(ok))
    if rank == 0:
        with open(out_path, "w") as fh:
            fh.write("ok" if all(flags) else f"mismatch {flags}")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_kslice_exchange_over_gloo(tmp_path, world):
    """The k-split across ranks: each rank multiplies one k-slice, one
    point-to-point exchange hands every rank the rows it owns from all
    partials, and the local merge gives exactly the rows of the merged
    product (pattern equal to the unsplit product, values within 1e-12)."""
    out = tmp_path / "result.txt"
    mp.start_processes(_kslice_worker, args=(world, _free_port(), str(out)), nprocs=world,
                       start_method="spawn", join=True)
    assert out.read_text() == "ok"


def _split3d_worker(rank, world, port, q, c, out_path):
    import torch
    import oracle
    from paper_1510_00844_gb300 import inputs, split3d as s3
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = inputs.random_csr(90, 70, 0.06, 21, value="int", index_dtype=np.int64)
    B = inputs.random_csr(70, 110, 0.06, 22, value="int", index_dtype=np.int64)
    m, l, n = A.nrows, A.ncols, B.ncols

    def piece(M):
        return (M.nrows, M.ncols, torch.from_numpy(np.asarray(M.rowptr, dtype=np.int64)),
                torch.from_numpy(np.asarray(M.col, dtype=np.int64)),
                torch.from_numpy(np.asarray(M.val, dtype=np.int64)))

    def owned(M, rows_parts, i, j, k):
        r0, r1 = s3.block(M.nrows, q, i)
        c0, c1 = s3.sub(M.ncols, q, c, j, k)
        return s3.cols_range(s3.rows_range(piece(M), r0, r1), c0, c1)

    def to_csr(P):
        m_, n_, rp, col, val = P
        return inputs.CSR(m_, n_, rp.numpy(), col.numpy(), val.numpy())

    def multiply(a, b):                       # the local multiply (HeapSpGEMM's role)
        C = oracle.spgemm(to_csr(a), to_csr(b))
        return piece(C)

    def merge(ps):                            # LocalMerge
        return piece(oracle.sum_partials([to_csr(P) for P in ps]))

    grid = s3.Grid(q, c)
    i, j, k = grid.i, grid.j, grid.k
    Cp = s3.split3d(grid, owned(A, q, i, j, k), owned(B, q, i, j, k), (m, l, n), multiply, merge,
                    torch.int64, torch.int64, torch.device("cpu"))
    parts = [None] * world
    dist.all_gather_object(parts, (i, j, k, Cp[2].numpy(), Cp[3].numpy(), Cp[4].numpy()))
    if rank == 0:
        full = oracle.spgemm(A, B)
        D = np.zeros((m, n), dtype=np.int64)
        P = np.zeros((m, n), dtype=bool)
        for (pi, pj, pk, rp, col, val) in parts:
            r0, _ = s3.block(m, q, pi)
            c0, _ = s3.sub(n, q, c, pj, pk)
            rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp)) + r0
            D[rows, col + c0] = val
            P[rows, col + c0] = True
        rows = np.repeat(np.arange(m), np.diff(full.rowptr))
        D2 = np.zeros((m, n), dtype=np.int64)
        P2 = np.zeros((m, n), dtype=bool)
        D2[rows, full.col] = full.val
        P2[rows, full.col] = True
        ok = np.array_equal(P, P2) and np.array_equal(D, D2)
        with open(out_path, "w") as fh:
            fh.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("q,c", [(2, 1), (2, 2), (1, 3)])
def test_split3d_over_gloo(tmp_path, q, c):
    """Alg. 2 on a q x q x c grid of CPU ranks: B's all-to-all across layers,
    the SUMMA broadcasts of A and B^, the local multiplies, C^int's
    all-to-all and the local merge give exactly the product (integer values,
    so any summation order is exact)."""
    out = tmp_path / "result.txt"
    world = q * q * c
    mp.start_processes(_split3d_worker, args=(world, _free_port(), q, c, str(out)), nprocs=world,
                       start_method="spawn", join=True)
    assert out.read_text() == "ok"
