"""Multi-GPU forms of the product: one process per GPU over torch.distributed.

Row panels: rank r multiplies rows panel(m, W, r) of A by the whole of B.
Panels are independent, so there is no collective on the data path.

k-split (the layers of Alg. 2): rank s multiplies the k-slice K_s of A by B;
its partial C_s covers all rows.  One exchange then sends rows
panel(m, W, r) of every C_s to rank r.  Rank r merges its W partials in
ascending s (Sec. 4.3).  The exchange is point to point: for each
destination, the rows it owns go as row pointers, columns and values.
NCCL carries it between GPUs; gloo carries it between CPU processes.

Row pieces are (rowptr, col, val) triples of torch tensors.  rowptr is
rebased to start at 0; val is None for pattern-only products."""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import torch
import torch.distributed as dist

Piece = Tuple[torch.Tensor, torch.Tensor, Optional[torch.Tensor]]


def panel(m: int, world: int, rank: int) -> Tuple[int, int]:
    """Rows [r0, r1) owned by `rank`: equal contiguous panels."""
    return (m * rank) // world, (m * (rank + 1)) // world


def rows_of(rowptr: torch.Tensor, col: torch.Tensor, val: Optional[torch.Tensor],
            r0: int, r1: int) -> Piece:
    """Rows [r0, r1) of a CSR as a piece (views of col/val, rebased rowptr)."""
    a, b = int(rowptr[r0].item()), int(rowptr[r1].item())
    rp = rowptr[r0:r1 + 1] - a
    return rp, col[a:b], None if val is None else val[a:b]


def exchange(pieces: Sequence[Piece], rows_per_rank: Sequence[int],
             col_dtype: torch.dtype, val_dtype: Optional[torch.dtype],
             device: torch.device) -> List[Piece]:
    """pieces[d] goes to rank d; returns what every rank s sent here, in s
    order.  Sizes travel first, then the row pointers, columns and values.
    Sends and receives are posted together, so the exchange cannot
    deadlock."""
    world, rank = dist.get_world_size(), dist.get_rank()
    assert len(pieces) == world
    nnz_out = [torch.tensor([int(p[1].numel())], dtype=torch.int64, device=device)
               for p in pieces]
    nnz_in = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    ops = []
    for peer in range(world):
        if peer == rank:
            nnz_in[peer].copy_(nnz_out[peer])
            continue
        ops.append(dist.P2POp(dist.isend, nnz_out[peer], peer, tag=3))
        ops.append(dist.P2POp(dist.irecv, nnz_in[peer], peer, tag=3))
    for w in (dist.batch_isend_irecv(ops) if ops else []):
        w.wait()
    mine = rows_per_rank[rank]
    recv: List[Piece] = []
    ops = []
    for peer in range(world):
        if peer == rank:
            recv.append(pieces[peer])
            continue
        k = int(nnz_in[peer].item())
        rp = torch.empty(mine + 1, dtype=torch.int64, device=device)
        cl = torch.empty(k, dtype=col_dtype, device=device)
        vl = None if val_dtype is None else torch.empty(k, dtype=val_dtype, device=device)
        recv.append((rp, cl, vl))
        sp = pieces[peer]
        for tag, (t_out, t_in) in enumerate(((sp[0], rp), (sp[1], cl), (sp[2], vl))):
            if t_in is None:
                continue
            assert t_out.dtype == t_in.dtype, "pieces must use the announced dtypes"
            ops.append(dist.P2POp(dist.isend, t_out.contiguous(), peer, tag=tag))
            ops.append(dist.P2POp(dist.irecv, t_in, peer, tag=tag))
    for w in (dist.batch_isend_irecv(ops) if ops else []):
        w.wait()
    return recv


def kslice_product(m: int, partial: Callable[[int, int], Piece],
                   merge: Callable[[List[Piece]], Piece],
                   col_dtype: torch.dtype, val_dtype: Optional[torch.dtype],
                   device: torch.device) -> Tuple[int, int, Piece]:
    """The k-split product on W ranks.  partial(s, W) returns the full-row
    partial C_s of this rank's slice as (rowptr, col, val); merge(pieces)
    sums the W pieces of one row panel in ascending s.  Returns (r0, r1,
    C(r0:r1, :))."""
    world, rank = dist.get_world_size(), dist.get_rank()
    rp, col, val = partial(rank, world)
    bounds = [panel(m, world, r) for r in range(world)]
    pieces = [rows_of(rp, col, val, a, b) for a, b in bounds]
    recv = exchange(pieces, [b - a for a, b in bounds], col_dtype, val_dtype, device)
    r0, r1 = bounds[rank]
    return r0, r1, merge(recv)


def gpu_kslice_product(A, B, semiring: int = 0, stream=None):
    """kslice_product with the library's own kernels: the partial is the
    plain two-phase product of this rank's k-slice view of A, the merge is
    the multiway merge (A6)."""
    from . import spgemm as sg
    dev = A.rowptr.device

    def partial(s, world):
        view = sg.kslice_views(A, world, stream)[s]
        C = sg.spgemm(view, B, semiring, stream=stream)
        return C.rowptr, C.col, C.val

    def merge(pieces):
        rows = pieces[0][0].numel() - 1
        parts = [sg.DeviceCSR(rows, B.ncols, p[0], p[1], p[2]) for p in pieces]
        C = sg.merge(parts, semiring, stream)
        return C.rowptr, C.col, C.val

    vdt = None if (A.val is None or semiring == sg.OR_AND) else A.val.dtype
    return kslice_product(A.nrows, partial, merge, A.col.dtype, vdt, dev)
