"""Galerkin hierarchy A_{l+1} = R_l^T A_l R_l on the GPU, all levels in one
CUDA graph, or in one persistent kernel launch.

The paper multiplies a matrix by its restriction operator to coarsen it
(Sec. 5.4: R^T A, then (R^T A) R).  Here every level's transpose and both
products are device-sized library calls (no host readback), so the whole
hierarchy is captured once in a CUDA graph and replayed; the product order
follows the paper (R^T A first).  Output capacities are upper bounds: with
one nonzero per row of R, flops(R^T A) = nnz(A) and flops((R^T A) R) =
nnz(R^T A), so nnz(A_l) bounds both products of level l."""
from __future__ import annotations

import ctypes
from typing import List, Optional

import torch

from . import spgemm as sg


class GalerkinChain:
    """persistent=False: every level's transpose and both products as
    device-sized library calls (about 140 launches, captured in one graph).
    persistent=True: the transposes R_l^T (which depend only on the given
    R_l) are formed once here, and the six products run as one persistent
    chain launch (spgemm_chain_launch): a graph of two nodes; block_threads
    is the chain's block size (1024 by default, for these short rows)."""

    def __init__(self, A0: sg.DeviceCSR, Rs: List[sg.DeviceCSR], stream: torch.cuda.Stream,
                 max_row_nnz: int = 64, tuning: Optional[sg.Tuning] = None,
                 persistent: bool = False, timeout_s: float = 0.0,
                 record_stages: bool = False, block_threads: int = 1024):
        self.stream = stream
        self.persistent = persistent
        self.Rs = Rs
        dev = A0.rowptr.device
        cap = A0.nnz
        vdt = A0.val.dtype
        idt = A0.col.dtype
        self.levels = []
        self._keep = []
        A = A0
        for R in Rs:
            n_f, n_c = R.nrows, R.ncols
            # R^T output (exact size: nnz(R))
            cR = sg._csr(R)
            tws = sg._workspace(sg._lib.spgemm_transpose_workspace_size(ctypes.byref(cR)), dev)
            Rt = sg.DeviceCSR(n_c, n_f, torch.empty(n_c + 1, dtype=torch.int64, device=dev),
                              torch.empty(R.nnz, dtype=idt, device=dev),
                              torch.empty(R.nnz, dtype=vdt, device=dev))
            T = sg.DeviceCSR(n_c, A.ncols, torch.empty(n_c + 1, dtype=torch.int64, device=dev),
                             torch.empty(cap, dtype=idt, device=dev),
                             torch.empty(cap, dtype=vdt, device=dev))
            An = sg.DeviceCSR(n_c, n_c, torch.empty(n_c + 1, dtype=torch.int64, device=dev),
                              torch.empty(cap, dtype=idt, device=dev),
                              torch.empty(cap, dtype=vdt, device=dev))
            p1 = sg.device_plan([Rt], [A], stream=stream, max_row_nnz=max_row_nnz, tuning=tuning)
            p2 = sg.device_plan([T], [R], stream=stream, max_row_nnz=max_row_nnz, tuning=tuning)
            self.levels.append(dict(R=R, cR=cR, tws=tws, Rt=Rt, T=T, A=An, p1=p1, p2=p2, cap=cap))
            A = An
        self.graph = None
        self.chain = None
        if persistent:
            with torch.cuda.stream(stream):
                for lv in self.levels:
                    self._transpose(lv)
            stream.synchronize()
            steps = []
            for lv in self.levels:
                steps.append((lv["p1"], lv["T"].rowptr, lv["cap"], lv["T"].col, lv["T"].val))
                steps.append((lv["p2"], lv["A"].rowptr, lv["cap"], lv["A"].col, lv["A"].val))
            # the hierarchy's rows are short (at most 56 products on a 7-point
            # stencil): 1024-thread blocks keep more of them in flight
            self.chain = sg.Chain(steps, timeout_s=timeout_s, record_stages=record_stages,
                                  block_threads=block_threads)

    def _transpose(self, lv):
        Rt = lv["Rt"]
        sg._check(sg._lib.spgemm_transpose(
            ctypes.byref(lv["cR"]), sg._stream(self.stream),
            ctypes.c_void_p(lv["tws"].data_ptr()), lv["tws"].numel(),
            ctypes.c_void_p(Rt.rowptr.data_ptr()), ctypes.c_void_p(Rt.col.data_ptr()),
            ctypes.c_void_p(Rt.val.data_ptr())))

    def _enqueue(self):
        if self.chain is not None:
            self.chain.launch(self.stream)
            return
        for lv in self.levels:
            self._transpose(lv)
            sg.execute(lv["p1"], lv["T"].rowptr, lv["cap"], lv["T"].col, lv["T"].val)
            sg.execute(lv["p2"], lv["A"].rowptr, lv["cap"], lv["A"].col, lv["A"].val)

    def run_eager(self):
        with torch.cuda.stream(self.stream):
            self._enqueue()

    def capture(self):
        """Records the whole hierarchy into one CUDA graph."""
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._enqueue()
        return self.graph

    def replay(self):
        self.graph.replay()

    def check(self):
        if self.chain is not None:
            self.chain.check(self.stream)
        for lv in self.levels:
            sg.check(lv["p1"])
            sg.check(lv["p2"])

    def results(self) -> List[sg.DeviceCSR]:
        """Coarse operators A_1..A_L (views trimmed to their nnz)."""
        out = []
        for lv in self.levels:
            A = lv["A"]
            nnz = int(A.rowptr[-1].item())
            out.append(sg.DeviceCSR(A.nrows, A.ncols, A.rowptr, A.col[:nnz], A.val[:nnz]))
        return out

    def intermediates(self) -> List[sg.DeviceCSR]:
        out = []
        for lv in self.levels:
            T = lv["T"]
            nnz = int(T.rowptr[-1].item())
            out.append(sg.DeviceCSR(T.nrows, T.ncols, T.rowptr, T.col[:nnz], T.val[:nnz]))
        return out
