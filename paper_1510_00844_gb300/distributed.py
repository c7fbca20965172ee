"""Multi-GPU forms of the product: one process per GPU over torch.distributed.

Row panels: rank r multiplies rows panel(m, W, r) of A by the whole of B.
Panels are independent, so there is no collective on the data path.

k-split (the layers of Alg. 2): rank s multiplies the k-slice K_s of A by B;
its partial C_s covers all rows.  One exchange then sends rows
panel(m, W, r) of every C_s to rank r.  Rank r merges its W partials in
ascending s (Sec. 4.3).  The exchange is point to point: for each
destination, the rows it owns go as row pointers, columns and values.
NCCL carries it between GPUs; gloo carries it between CPU processes (and
between GPU processes through host memory, for tests on one GPU).

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


def panel_pieces(rowptr: torch.Tensor, col: torch.Tensor, val: Optional[torch.Tensor],
                 bounds: Sequence[Tuple[int, int]]) -> List[Piece]:
    """Rows [a, b) of a CSR for every (a, b) in `bounds` (consecutive
    panels), as pieces: views of col/val and rebased row pointers.  The
    panels' entry offsets are read back in one copy."""
    cuts = [bounds[0][0]] + [b for _, b in bounds]
    offs = rowptr[torch.tensor(cuts, dtype=torch.int64, device=rowptr.device)].tolist()
    out = []
    for t, (a, b) in enumerate(bounds):
        lo, hi = offs[t], offs[t + 1]
        out.append((rowptr[a:b + 1] - lo, col[lo:hi], None if val is None else val[lo:hi]))
    return out


def rows_of(rowptr: torch.Tensor, col: torch.Tensor, val: Optional[torch.Tensor],
            r0: int, r1: int) -> Piece:
    """Rows [r0, r1) of a CSR as a piece (views of col/val, rebased rowptr)."""
    return panel_pieces(rowptr, col, val, [(r0, r1)])[0]


def exchange(pieces: Sequence[Piece], rows_per_rank: Sequence[int],
             col_dtype: torch.dtype, val_dtype: Optional[torch.dtype],
             device: torch.device, comm_device: Optional[torch.device] = None) -> List[Piece]:
    """pieces[d] goes to rank d; returns what every rank s sent here, in s
    order, on `device`.  Two grouped point-to-point rounds: the entry counts
    (the receiver reads them back in one copy to size its buffers), then the
    row pointers, columns and values of every piece.  Sends and receives are
    posted together, so the exchange cannot deadlock.  Messages travel
    through `comm_device` (default `device`): the GPU itself under NCCL, host
    memory under gloo, whose point-to-point operations take CPU tensors."""
    world, rank = dist.get_world_size(), dist.get_rank()
    assert len(pieces) == world
    comm = device if comm_device is None else comm_device
    nnz_out = torch.tensor([int(p[1].numel()) for p in pieces], dtype=torch.int64, device=comm)
    nnz_in = torch.zeros(world, dtype=torch.int64, device=comm)
    ops = []
    for peer in range(world):
        if peer == rank:
            continue
        ops.append(dist.P2POp(dist.isend, nnz_out[peer:peer + 1], peer, tag=3))
        ops.append(dist.P2POp(dist.irecv, nnz_in[peer:peer + 1], peer, tag=3))
    for w in (dist.batch_isend_irecv(ops) if ops else []):
        w.wait()
    sizes = nnz_in.tolist()
    mine = rows_per_rank[rank]
    recv: List[Optional[Piece]] = []
    ops = []
    keep = []
    for peer in range(world):
        if peer == rank:
            recv.append(None)
            continue
        k = sizes[peer]
        rp = torch.empty(mine + 1, dtype=torch.int64, device=comm)
        cl = torch.empty(k, dtype=col_dtype, device=comm)
        vl = None if val_dtype is None else torch.empty(k, dtype=val_dtype, device=comm)
        recv.append((rp, cl, vl))
        sp = pieces[peer]
        for tag, (t_out, t_in) in enumerate(((sp[0], rp), (sp[1], cl), (sp[2], vl))):
            if t_in is None:
                continue
            assert t_out.dtype == t_in.dtype, "pieces must use the announced dtypes"
            t_send = t_out.contiguous().to(comm)
            keep.append(t_send)
            ops.append(dist.P2POp(dist.isend, t_send, peer, tag=tag))
            ops.append(dist.P2POp(dist.irecv, t_in, peer, tag=tag))
    for w in (dist.batch_isend_irecv(ops) if ops else []):
        w.wait()
    out: List[Piece] = []
    for peer in range(world):
        if peer == rank:
            out.append(pieces[peer])
        else:
            rp, cl, vl = recv[peer]
            out.append((rp.to(device), cl.to(device), None if vl is None else vl.to(device)))
    return out


def kslice_product(m: int, partial: Callable[[int, int], Piece],
                   merge: Callable[[List[Piece]], Piece],
                   col_dtype: torch.dtype, val_dtype: Optional[torch.dtype],
                   device: torch.device,
                   comm_device: Optional[torch.device] = None) -> Tuple[int, int, Piece]:
    """The k-split product on W ranks.  partial(s, W) returns the full-row
    partial C_s of this rank's slice as (rowptr, col, val); merge(pieces)
    sums the W pieces of one row panel in ascending s.  Returns (r0, r1,
    C(r0:r1, :))."""
    world, rank = dist.get_world_size(), dist.get_rank()
    rp, col, val = partial(rank, world)
    bounds = [panel(m, world, r) for r in range(world)]
    pieces = panel_pieces(rp, col, val, bounds)
    recv = exchange(pieces, [b - a for a, b in bounds], col_dtype, val_dtype, device,
                    comm_device)
    r0, r1 = bounds[rank]
    return r0, r1, merge(recv)


def gpu_kslice_product(A, B, semiring: int = 0, stream=None, comm_device=None):
    """kslice_product with the library's own kernels: the partial is the
    plain two-phase product of this rank's k-slice view of A, the merge is
    the multiway merge (A6).  comm_device: where messages travel (the GPU
    under NCCL; the CPU under gloo)."""
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
    return kslice_product(A.nrows, partial, merge, A.col.dtype, vdt, dev, comm_device)
