"""The multi-GPU forms of the product with the library's kernels inside,
checked against the oracle.  Each rank is a process on cuda:0; messages go
through host memory over gloo (NCCL needs one GPU per rank).  No kernel
waits on another rank: every exchange is a host-side collective between
launches.

* k-split (the layers of Alg. 2): rank s multiplies k-slice K_s with the
  CUDA path, one exchange hands every rank its rows of all partials, the CUDA
  multiway merge sums them; each rank's rows are compared with the oracle's
  product (pattern exact, values within 1e-12 relative) and with the oracle's
  sum of its slice products (exact).
* Split-3D (Alg. 2) on 2x2x1 and 2x2x2 grids with the CUDA multiply and
  merge as the local operations; every rank's block is compared with the
  same block of the oracle's product."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    return dist


def _finish(dist, ok, out_path, rank, world):
    flags = [None] * world
    dist.all_gather_object(flags, ok)
    if rank == 0:
        with open(out_path, "w") as fh:
            fh.write("ok" if all(f == "ok" for f in flags) else f"mismatch {flags}")
    dist.barrier()
    dist.destroy_process_group()


def _kslice_worker(rank, world, port, out_path):
    import torch
    import oracle
    from paper_1510_00844_gb300 import distributed, inputs, spgemm as sg
    from tests.parity import rows_subset
    dist = _init(rank, world, port)
    A = inputs.rmat(11)
    dA = sg.to_device(A, "cuda:0")
    r0, r1, (rp, col, val) = distributed.gpu_kslice_product(dA, dA,
                                                            comm_device=torch.device("cpu"))
    rp, col, val = rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    full = rows_subset(oracle.spgemm(A, A), np.arange(r0, r1))
    sums = rows_subset(oracle.sum_partials([oracle.spgemm(*ks) for ks in oracle.kslice(A, A, world)]),
                       np.arange(r0, r1))
    ok = "ok"
    if (r0, r1) != distributed.panel(A.nrows, world, rank):
        ok = "panel"
    elif not (np.array_equal(rp, full.rowptr) and np.array_equal(col.astype(np.int64), full.col)):
        ok = "pattern"
    elif not np.all(np.abs(val - full.val) <= 1e-12 * np.abs(full.val)):
        ok = "values vs product"
    elif not np.array_equal(val, sums.val):
        ok = "values vs slice sums"
    _finish(dist, ok, out_path, rank, world)


@pytest.mark.parametrize("world", [2, 3])
def test_kslice_product_with_cuda_kernels_matches_oracle(tmp_path, world):
    out = tmp_path / "result.txt"
    mp.start_processes(_kslice_worker, args=(world, _free_port(), str(out)), nprocs=world,
                       start_method="spawn", join=True)
    assert out.read_text() == "ok"


def _split3d_worker(rank, world, port, q, c, value, out_path):
    import torch
    import oracle
    from paper_1510_00844_gb300 import inputs, split3d as s3
    dist = _init(rank, world, port)
    A = inputs.random_csr(300, 260, 0.03, 31, value=value, index_dtype=np.int64)
    B = inputs.random_csr(260, 340, 0.03, 32, value=value, index_dtype=np.int64)
    m, l, n = A.nrows, A.ncols, B.ncols
    dev = torch.device("cuda:0")
    vdt = torch.float64 if value == "u01_f64" else torch.int64

    def piece(M):
        return (M.nrows, M.ncols, torch.from_numpy(np.asarray(M.rowptr, dtype=np.int64)).to(dev),
                torch.from_numpy(np.asarray(M.col, dtype=np.int64)).to(dev),
                torch.from_numpy(np.asarray(M.val)).to(dev))

    def owned(M, i, j, k):
        r0, r1 = s3.block(M.nrows, q, i)
        c0, c1 = s3.sub(M.ncols, q, c, j, k)
        return s3.cols_range(s3.rows_range(piece(M), r0, r1), c0, c1)

    grid = s3.Grid(q, c)
    i, j, k = grid.i, grid.j, grid.k
    multiply, merge = s3.gpu_ops()
    Cp = s3.split3d(grid, owned(A, i, j, k), owned(B, i, j, k), (m, l, n), multiply, merge,
                    torch.int64, vdt, dev, comm_device=torch.device("cpu"))
    ref = s3.cols_range(s3.rows_range(piece(oracle.spgemm(A, B)), *s3.block(m, q, i)),
                        *s3.sub(n, q, c, j, k))
    got = [t.cpu().numpy() for t in Cp[2:]]
    exp = [t.cpu().numpy() for t in ref[2:]]
    ok = "ok"
    if not (np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])):
        ok = "pattern"
    elif value == "int" and not np.array_equal(got[2], exp[2]):
        ok = "values"
    elif value != "int" and not np.all(np.abs(got[2] - exp[2]) <= 1e-12 * np.abs(exp[2])):
        ok = "values"
    _finish(dist, ok, out_path, rank, world)


@pytest.mark.parametrize("q,c,value", [(2, 1, "u01_f64"), (2, 2, "u01_f64"), (2, 2, "int")])
def test_split3d_with_cuda_kernels_matches_oracle(tmp_path, q, c, value):
    out = tmp_path / "result.txt"
    world = q * q * c
    mp.start_processes(_split3d_worker, args=(world, _free_port(), q, c, value, str(out)),
                       nprocs=world, start_method="spawn", join=True)
    assert out.read_text() == "ok"
