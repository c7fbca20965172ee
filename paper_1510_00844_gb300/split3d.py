"""Split-3D-SpGEMM (Alg. 2) over torch.distributed: C = A.B on a
q x q x c process grid (p = q*q*c ranks, one GPU each; rank = (i*q + j)*c + k
for process P(i,j,k)).

Distribution (the memory-friendly split of Sec. 3): P(i,j,k) owns rows
block(m, q, i) of A and the columns sub(l, q, c, j, k), i.e. column block j
of the inner dimension cut into c layers; B and C are split the same way
(rows by i; columns by j then k).  Per process:

1. B^_ijk = AlltoAll(B_ij:, P(i,j,:)): the fiber exchanges B so that layer k
   holds the k-th sub-block of B's row block i, with all columns of block j.
2. For r = 0..q-1 (SUMMA stages, one blocking step b = locinndim):
   A^rem = Broadcast(A_irk, P(i,:,k)), B^rem = Broadcast(B^_rjk, P(:,j,k)),
   C^int_ij: += A^rem . B^rem (the local multiply; partials are kept).
3. C^int_ijk = AlltoAll(C^int_ij:, P(i,j,:)): layer k receives the columns of
   its sub-block from every partial of the fiber.
4. C_ijk = LocalMerge(C^int_ijk): the multiway merge of Sec. 4.3.

Pieces are (nrows, ncols, rowptr, col, val) with torch tensors and local
indices; `multiply(a, b)` and `merge(pieces)` are the local operations (the
library's kernels on GPUs, see gpu_ops).  Broadcasts send the piece's sizes
first, then its arrays; all-to-alls are point-to-point, as in
distributed.exchange."""
from __future__ import annotations

from typing import Callable, Dict, List, Optional, Tuple

import torch
import torch.distributed as dist

Piece = Tuple[int, int, torch.Tensor, torch.Tensor, Optional[torch.Tensor]]


def block(x: int, parts: int, idx: int) -> Tuple[int, int]:
    """[lo, hi) of block idx when 0..x-1 is cut into `parts` equal blocks."""
    return (x * idx) // parts, (x * (idx + 1)) // parts


def sub(x: int, q: int, c: int, j: int, k: int) -> Tuple[int, int]:
    """Layer k of block j: block j of q, cut again into c parts."""
    lo, hi = block(x, q, j)
    a, b = block(hi - lo, c, k)
    return lo + a, lo + b


def coords(rank: int, q: int, c: int) -> Tuple[int, int, int]:
    return rank // (q * c), (rank // c) % q, rank % c


def rank_of(i: int, j: int, k: int, q: int, c: int) -> int:
    return (i * q + j) * c + k


def cols_range(P: Piece, c0: int, c1: int) -> Piece:
    """Entries with c0 <= col < c1, columns shifted to start at 0."""
    m, n, rp, col, val = P
    keep = (col >= c0) & (col < c1)
    rows = torch.repeat_interleave(torch.arange(m, device=rp.device), rp[1:] - rp[:-1])
    counts = torch.bincount(rows[keep], minlength=m) if m > 0 else rp[:0]
    nrp = torch.zeros(m + 1, dtype=torch.int64, device=rp.device)
    if m > 0:
        nrp[1:] = torch.cumsum(counts, 0)
    return (m, c1 - c0, nrp, (col[keep] - c0).to(col.dtype),
            None if val is None else val[keep])


def rows_range(P: Piece, r0: int, r1: int) -> Piece:
    m, n, rp, col, val = P
    a, b = rp[[r0, r1]].tolist()
    return (r1 - r0, n, rp[r0:r1 + 1] - a, col[a:b], None if val is None else val[a:b])


def hcat(pieces: List[Piece], offsets: List[int], ncols: int) -> Piece:
    """Pieces with the same rows and disjoint column ranges (piece t shifted
    by offsets[t]) placed side by side; columns stay sorted in every row."""
    m = pieces[0][0]
    dev = pieces[0][2].device
    rows, cols, vals = [], [], []
    for (pm, pn, rp, col, val), off in zip(pieces, offsets):
        rows.append(torch.repeat_interleave(torch.arange(m, device=dev), rp[1:] - rp[:-1]))
        cols.append(col.to(torch.int64) + off)
        vals.append(val)
    r = torch.cat(rows)
    cl = torch.cat(cols)
    order = torch.argsort(r * max(ncols, 1) + cl, stable=True)
    counts = torch.bincount(r, minlength=m) if m > 0 else torch.zeros(0, dtype=torch.int64)
    rp = torch.zeros(m + 1, dtype=torch.int64, device=dev)
    if m > 0:
        rp[1:] = torch.cumsum(counts, 0)
    val = None if vals[0] is None else torch.cat(vals)[order]
    return (m, ncols, rp, cl[order].to(pieces[0][3].dtype), val)


def _send_piece(P: Piece, dst: int, tag: int, ops: list, keep: list, comm):
    m, n, rp, col, val = P
    for t, a in enumerate((rp, col, val)):
        if a is not None:
            a = a.contiguous().to(comm)
            keep.append(a)
            ops.append(dist.P2POp(dist.isend, a, dst, tag=tag + t))


def _alltoall(pieces: Dict[int, Piece], incoming: Dict[int, Tuple[int, int]], col_dtype,
              val_dtype, device, comm=None) -> Dict[int, Piece]:
    """pieces[dst] goes to rank dst; incoming[src] = (rows, cols) of the piece
    rank src sends here.  nnz values travel first (read back in one copy);
    messages go through `comm` (default `device`), results land on `device`."""
    me = dist.get_rank()
    comm = device if comm is None else comm
    nnz_out = {d: torch.tensor([int(P[3].numel())], dtype=torch.int64, device=comm)
               for d, P in pieces.items() if d != me}
    srcs = [s for s in incoming if s != me]
    nnz_in = torch.zeros(max(len(srcs), 1), dtype=torch.int64, device=comm)
    ops = [dist.P2POp(dist.isend, t, d, tag=7) for d, t in nnz_out.items()]
    ops += [dist.P2POp(dist.irecv, nnz_in[t:t + 1], s, tag=7) for t, s in enumerate(srcs)]
    for w in (dist.batch_isend_irecv(ops) if ops else []):
        w.wait()
    sizes = dict(zip(srcs, nnz_in.tolist()))
    got: Dict[int, Piece] = {}
    ops = []
    keep = []
    for s, (m, n) in incoming.items():
        if s == me:
            continue
        k = sizes[s]
        rp = torch.empty(m + 1, dtype=torch.int64, device=comm)
        cl = torch.empty(k, dtype=col_dtype, device=comm)
        vl = None if val_dtype is None else torch.empty(k, dtype=val_dtype, device=comm)
        got[s] = (m, n, rp, cl, vl)
        ops.append(dist.P2POp(dist.irecv, rp, s, tag=10))
        ops.append(dist.P2POp(dist.irecv, cl, s, tag=11))
        if vl is not None:
            ops.append(dist.P2POp(dist.irecv, vl, s, tag=12))
    for d, P in pieces.items():
        if d != me:
            _send_piece(P, d, 10, ops, keep, comm)
    for w in (dist.batch_isend_irecv(ops) if ops else []):
        w.wait()
    out: Dict[int, Piece] = {}
    for s in incoming:
        if s == me:
            out[s] = pieces[me]
        else:
            m, n, rp, cl, vl = got[s]
            out[s] = (m, n, rp.to(device), cl.to(device), None if vl is None else vl.to(device))
    return out


def _broadcast(P: Optional[Piece], root: int, group, col_dtype, val_dtype, device,
               comm=None) -> Piece:
    """The root's piece on every member of the group (sent through `comm`,
    default `device`; returned on `device`)."""
    me = dist.get_rank()
    comm = device if comm is None else comm
    hdr = torch.zeros(3, dtype=torch.int64, device=comm)
    if me == root:
        hdr[0], hdr[1], hdr[2] = P[0], P[1], P[3].numel()
    dist.broadcast(hdr, root, group=group)
    m, n, k = (int(x) for x in hdr.tolist())
    if me == root:
        rp, cl = P[2].contiguous().to(comm), P[3].contiguous().to(comm)
        vl = None if P[4] is None else P[4].contiguous().to(comm)
    else:
        rp = torch.empty(m + 1, dtype=torch.int64, device=comm)
        cl = torch.empty(k, dtype=col_dtype, device=comm)
        vl = None if val_dtype is None else torch.empty(k, dtype=val_dtype, device=comm)
    dist.broadcast(rp, root, group=group)
    dist.broadcast(cl, root, group=group)
    if vl is not None:
        dist.broadcast(vl, root, group=group)
    if me == root:
        return P
    return (m, n, rp.to(device), cl.to(device), None if vl is None else vl.to(device))


class Grid:
    """The q x q x c grid of the calling process with its row, column and
    fiber groups (every rank creates every group, in the same order)."""

    def __init__(self, q: int, c: int):
        world = dist.get_world_size()
        assert world == q * q * c, "world size must be q*q*c"
        self.q, self.c = q, c
        self.i, self.j, self.k = coords(dist.get_rank(), q, c)
        self.row = {}
        self.col = {}
        for i in range(q):
            for k in range(c):
                self.row[(i, k)] = dist.new_group([rank_of(i, j, k, q, c) for j in range(q)])
        for j in range(q):
            for k in range(c):
                self.col[(j, k)] = dist.new_group([rank_of(i, j, k, q, c) for i in range(q)])


def split3d(grid: Grid, A_ijk: Piece, B_ijk: Piece, dims: Tuple[int, int, int],
            multiply: Callable[[Piece, Piece], Piece],
            merge: Callable[[List[Piece]], Piece], col_dtype, val_dtype, device,
            comm_device=None) -> Piece:
    """Alg. 2 on this process: returns C_ijk (rows block(m, q, i), columns
    sub(n, q, c, j, k), local indices).  Pieces live on `device`; messages go
    through `comm_device` (default `device`: the GPU under NCCL; the CPU
    under gloo)."""
    comm = comm_device
    q, c, i, j, k = grid.q, grid.c, grid.i, grid.j, grid.k
    m, l, n = dims
    # 1. B^ across the fiber: layer k' gets rows sub-block k' of B's row block i
    bi0, bi1 = block(l, q, i)
    pieces = {}
    incoming = {}
    for kk in range(c):
        r0, r1 = sub(l, q, c, i, kk)
        pieces[rank_of(i, j, kk, q, c)] = rows_range(B_ijk, r0 - bi0, r1 - bi0)
        s0, s1 = sub(n, q, c, j, kk)
        mine0, mine1 = sub(l, q, c, i, k)
        incoming[rank_of(i, j, kk, q, c)] = (mine1 - mine0, s1 - s0)
    got = _alltoall(pieces, incoming, col_dtype, val_dtype, device, comm)
    j0, j1 = block(n, q, j)
    B_hat = hcat([got[rank_of(i, j, kk, q, c)] for kk in range(c)],
                 [sub(n, q, c, j, kk)[0] - j0 for kk in range(c)], j1 - j0)
    # 2. SUMMA stages
    partials = []
    for r in range(q):
        A_rem = _broadcast(A_ijk if j == r else None, rank_of(i, r, k, q, c), grid.row[(i, k)],
                           col_dtype, val_dtype, device, comm)
        B_rem = _broadcast(B_hat if i == r else None, rank_of(r, j, k, q, c), grid.col[(j, k)],
                           col_dtype, val_dtype, device, comm)
        partials.append(multiply(A_rem, B_rem))
    # 3. C^int across the fiber: layer k' gets the columns of its sub-block
    i0, i1 = block(m, q, i)
    pieces = {}
    incoming = {}
    for kk in range(c):
        s0, s1 = sub(n, q, c, j, kk)
        dst = rank_of(i, j, kk, q, c)
        # one piece per destination: the partials side by side in row order is
        # not a CSR, so they travel one after another as separate messages
        pieces[dst] = [cols_range(P, s0 - j0, s1 - j0) for P in partials]
    received: List[Piece] = []
    for t in range(q):
        send = {d: ps[t] for d, ps in pieces.items()}
        s0, s1 = sub(n, q, c, j, k)
        inc = {rank_of(i, j, kk, q, c): (i1 - i0, s1 - s0) for kk in range(c)}
        got = _alltoall(send, inc, col_dtype, val_dtype, device, comm)
        received += [got[rank_of(i, j, kk, q, c)] for kk in range(c)]
    # 4. local merge (partials in ascending stage, then layer)
    order = [received[t * c + kk] for t in range(q) for kk in range(c)]
    return merge(order)


def gpu_ops(semiring: int = 0):
    """multiply and merge with the library's kernels on device pieces."""
    from . import spgemm as sg

    def as_csr(P: Piece):
        return sg.DeviceCSR(P[0], P[1], P[2], P[3], P[4])

    def multiply(a: Piece, b: Piece) -> Piece:
        C = sg.spgemm(as_csr(a), as_csr(b), semiring)
        return (C.nrows, C.ncols, C.rowptr, C.col, C.val)

    def merge(pieces: List[Piece]) -> Piece:
        C = sg.merge([as_csr(P) for P in pieces], semiring)
        return (C.nrows, C.ncols, C.rowptr, C.col, C.val)

    return multiply, merge
