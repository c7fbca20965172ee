"""C = A.B delivered to pinned host memory, one row panel at a time.

A product whose C is read on the host pays for a device-to-host copy of
every column index and value.  Here the rows of A are cut into panels.  The
symbolic phase of all panels runs first, so that the host arrays can be
sized once.  Then the numeric phase of panel p+1 runs on the compute stream
while panel p's columns and values are copied to the host on copy streams.
Two device buffers alternate between the two.  Panels also bound the device
memory that C needs, so products whose C exceeds HBM can be formed (the row
panelling of the learned-sizing workload)."""
from __future__ import annotations

import mmap
import weakref
from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import torch

from . import spgemm as sg


def pinned_empty(numel: int, dtype: torch.dtype) -> torch.Tensor:
    """Page-locked host array for copies to and from the GPU.

    Anonymous memory advised for transparent huge pages, touched once and
    registered with the CUDA driver (cudaHostRegister), so that the copy
    engines see it through few large pages: device-to-host copies of C then
    run at the link's rate from the first copy on, where freshly pinned
    small pages were measured at a third of it.  Falls back to torch's
    pinned allocator when huge-page advice or registration is unavailable.
    The registration is dropped when the last tensor viewing the memory is
    freed."""
    n = max(int(numel), 1)
    elem = torch.empty(0, dtype=dtype).element_size()
    try:
        mm = mmap.mmap(-1, n * elem, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        mm.madvise(mmap.MADV_HUGEPAGE)
        arr = np.frombuffer(mm, dtype=np.uint8)
        torch.from_numpy(arr).zero_()     # first touch, on all host threads
        ptr = int(arr.ctypes.data)
        cudart = torch.cuda.cudart()
        if int(cudart.cudaHostRegister(ptr, n * elem, 0)) != 0:
            raise OSError("cudaHostRegister failed")
    except (AssertionError, AttributeError, OSError, ValueError, RuntimeError):
        return torch.empty(numel, dtype=dtype, pin_memory=True)
    weakref.finalize(arr, cudart.cudaHostUnregister, ptr)
    return torch.from_numpy(arr).view(dtype)[:numel]


@dataclass
class HostCSR:
    nrows: int
    ncols: int
    rowptr: torch.Tensor          # int64 [nrows + 1], pinned host memory
    col: torch.Tensor             # pinned host memory
    val: Optional[torch.Tensor]   # pinned host memory, None for pattern-only

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def host_buffers(nrows: int, nnz: int, col_dtype, val_dtype) -> HostCSR:
    """Pinned host arrays for a result (pinned_empty); pass them back as
    `out` to reuse."""
    return HostCSR(nrows, 0, pinned_empty(nrows + 1, torch.int64),
                   pinned_empty(nnz, col_dtype),
                   None if val_dtype is None else pinned_empty(nnz, val_dtype))


def spgemm_to_host(A: sg.DeviceCSR, B: sg.DeviceCSR, semiring: int = sg.PLUS_TIMES,
                   panels: int = 8, copy_streams: int = 2, out: Optional[HostCSR] = None,
                   tuning: Optional[sg.Tuning] = None, timing: Optional[dict] = None) -> HostCSR:
    """C = A.B into pinned host memory (see the module docstring).  `out`
    is reused when it is large enough; otherwise new buffers are pinned.
    With `timing` (a dict), CUDA events record where the time goes; the
    dict receives milliseconds for the plans and symbolic phases, the
    numeric phases, the copies, the copy tail after the last numeric phase,
    and the bytes copied to the host."""
    dev = A.rowptr.device
    ev_t0 = None
    if timing is not None:
        ev_t0 = torch.cuda.Event(enable_timing=True)
        ev_t0.record(torch.cuda.current_stream(dev))
    m = A.nrows
    panels = max(1, min(int(panels), max(m, 1)))
    bounds = [((m * p) // panels, (m * (p + 1)) // panels) for p in range(panels)]
    compute = torch.cuda.current_stream(dev)
    plans: List[sg.Plan] = []
    rowptrs: List[torch.Tensor] = []
    counts: List[int] = []
    for a, b in bounds:
        end = A.rowend[a:b] if A.rowend is not None else A.rowptr[a + 1:b + 1]
        view = sg.DeviceCSR(b - a, A.ncols, A.rowptr[a:b], A.col, A.val, rowend=end)
        p = sg.plan(view, B, semiring, stream=compute, tuning=tuning)
        rp, nnz = sg.symbolic(p)
        plans.append(p)
        rowptrs.append(rp)
        counts.append(int(nnz))
    ev_sym = None
    if timing is not None:
        ev_sym = torch.cuda.Event(enable_timing=True)
        ev_sym.record(compute)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    total = int(offs[-1])
    pattern = plans[0].pattern_only
    col_dtype = A.col.dtype
    val_dtype = None if pattern else A.val.dtype
    if (out is None or out.col.numel() < total or out.rowptr.numel() < m + 1
            or (val_dtype is not None and (out.val is None or out.val.numel() < total))):
        out = host_buffers(m, total, col_dtype, val_dtype)
    out.ncols = B.ncols
    cap = max(counts) if counts else 0
    bufs = []
    for _ in range(min(2, panels)):
        bufs.append((torch.empty(max(cap, 1), dtype=col_dtype, device=dev),
                     None if pattern else torch.empty(max(cap, 1), dtype=val_dtype, device=dev)))
    copiers = [torch.cuda.Stream(dev) for _ in range(max(1, copy_streams))]
    free = [None] * len(bufs)            # event: the buffer's last copy finished
    num_ev, copy_ev = [], []
    for p, (a, b) in enumerate(bounds):
        k = p % len(bufs)
        colb, valb = bufs[k]
        if free[k] is not None:
            compute.wait_event(free[k])
        if timing is not None:
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(compute)
        sg.numeric(plans[p], rowptrs[p], colb, valb)
        if timing is not None:
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record(compute)
            num_ev.append((e0, e1))
        rp_glob = rowptrs[p][1:] + int(offs[p])
        ready = torch.cuda.Event()
        ready.record(compute)
        n = counts[p]
        o = int(offs[p])
        done = []
        for j, s in enumerate(copiers):
            s.wait_event(ready)
            lo, hi = (n * j) // len(copiers), (n * (j + 1)) // len(copiers)
            if timing is not None and j == 0:
                c0 = torch.cuda.Event(enable_timing=True)
                c0.record(s)
            with torch.cuda.stream(s):
                if hi > lo:
                    out.col[o + lo:o + hi].copy_(colb[lo:hi], non_blocking=True)
                    if valb is not None:
                        out.val[o + lo:o + hi].copy_(valb[lo:hi], non_blocking=True)
                if j == 0:
                    out.rowptr[a + 1:b + 1].copy_(rp_glob, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s)
                done.append(ev)
        for ev in done[1:]:
            copiers[0].wait_event(ev)
        fin = torch.cuda.Event(enable_timing=timing is not None)
        fin.record(copiers[0])
        free[k] = fin
        if timing is not None:
            copy_ev.append((c0, fin))
        rp_glob.record_stream(copiers[0])
    out.rowptr[0] = 0
    for s in copiers:
        s.synchronize()
    if timing is not None:
        compute.synchronize()
        timing["plans_symbolic_ms"] = ev_t0.elapsed_time(ev_sym)
        timing["numeric_ms"] = sum(x.elapsed_time(y) for x, y in num_ev)
        timing["copy_ms"] = sum(x.elapsed_time(y) for x, y in copy_ev)
        timing["copy_tail_ms"] = num_ev[-1][1].elapsed_time(copy_ev[-1][1]) if num_ev else 0.0
        timing["first_numeric_to_last_copy_ms"] = (num_ev[0][0].elapsed_time(copy_ev[-1][1])
                                                   if num_ev else 0.0)
        elem = col_dtype.itemsize + (0 if val_dtype is None else val_dtype.itemsize)
        timing["d2h_bytes"] = int(total) * elem + (m + 1) * 8
    for p in plans:
        p.close()
    return out
