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
