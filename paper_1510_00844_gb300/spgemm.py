"""Python binding of the C ABI in include/spgemm.h (ctypes).

Argument marshalling only: every step of the product runs in the CUDA
library.  PyTorch supplies device memory (outputs and workspaces are torch
tensors) and the stream (the current torch stream).  If the library cannot
be loaded the import fails; there is no CPU fallback.

Names follow the C entry points: ``plan``, ``symbolic``, ``numeric``,
``kslice_bounds``, ``merge_symbolic``, ``merge_numeric``; ``spgemm`` and
``spgemm_kslice`` chain them for the common case."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

F64, F32, I64, BOOL = 0, 1, 2, 3
INDEX_I32, INDEX_I64 = 0, 1
PLUS_TIMES, OR_AND, MIN_PLUS, MIN_SELECT2ND = 0, 1, 2, 3

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "INVALID_CSR", 3: "INDEX_OVERFLOW", 4: "OUT_OF_MEMORY",
          5: "TIMEOUT", 6: "CUDA", 7: "NOT_SUPPORTED", 8: "INTERNAL"}


class SpgemmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("rowend", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("index_type", ctypes.c_int32), ("value_type", ctypes.c_int32)]


class _Opts(ctypes.Structure):
    _fields_ = [("semiring", ctypes.c_int32), ("checked", ctypes.c_int32),
                ("dense_chunk", ctypes.c_int32), ("dense_min_flops", ctypes.c_int32),
                ("max_row_nnz", ctypes.c_int32), ("hash_shift", ctypes.c_int32),
                ("seg_log2", ctypes.c_int32), ("merge_staged", ctypes.c_int32)]


@dataclass(frozen=True)
class Tuning:
    """Runtime knobs of a plan (spgemm_opts): dense-row chunk width (0, 1024
    or 2048), dense threshold in products (0 = 1024, else 32..1024), hash
    table sizing shift (0..2) and dense work-unit size log2 (0 = per plan, else
    10..22).  The autotuner (autotune.py) searches them."""
    dense_chunk: int = 0
    dense_min_flops: int = 0
    hash_shift: int = 0
    seg_log2: int = 0


def _make_opts(semiring: int, checked: bool = False, tuning: Optional[Tuning] = None,
               dense_chunk: int = 0, dense_min_flops: int = 0, max_row_nnz: int = 0) -> "_Opts":
    t = tuning or Tuning()
    return _Opts(semiring, 1 if checked else 0, t.dense_chunk or dense_chunk,
                 t.dense_min_flops or dense_min_flops, max_row_nnz, t.hash_shift, t.seg_log2)


class _Info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in
                ("m", "l", "n", "flops", "max_row_flops", "rows_empty", "rows_hash",
                 "rows_dense", "chunk_width", "chunks_per_row", "nnz_c")]


def _load():
    path = _build.LIB
    if not _build.up_to_date():
        path = _build.build()
    lib = ctypes.CDLL(path)
    P, S, I64_, I32_ = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int32
    st = ctypes.c_int
    sig = {
        "spgemm_version": (ctypes.c_char_p, []),
        "spgemm_kernel_launches": (I64_, []),
        "spgemm_last_error": (ctypes.c_char_p, []),
        "spgemm_plan_workspace_size": (S, [I64_]),
        "spgemm_plan": (st, [P, P, P, P, P, S, P]),
        "spgemm_batch_plan_workspace_size": (S, [I32_, P]),
        "spgemm_batch_plan": (st, [I32_, P, P, P, P, P, S, P]),
        "spgemm_plan_device": (st, [I32_, P, P, P, P, P, S, P]),
        "spgemm_execute": (st, [P, P, S, P, I64_, P, P]),
        "spgemm_batch_rowptrs": (st, [P, P, P]),
        "spgemm_transpose_workspace_size": (S, [P]),
        "spgemm_sizer_param_count": (I32_, [I32_]),
        "spgemm_mcl_workspace_size": (S, [I64_]),
        "spgemm_mask_workspace_size": (S, [I64_]),
        "spgemm_mis2_workspace_size": (S, [I64_]),
        "spgemm_dcsr_workspace_size": (S, [I64_]),
        "spgemm_dcsr_view": (st, [P, P, P, S, P, P, P, P]),
        "spgemm_dcsr_expand": (st, [I64_, I64_, P, P, P, P]),
        "spgemm_mis2_restriction": (st, [P, ctypes.c_uint64, P, P, S, P, P, P, P, P]),
        "spgemm_mask_count": (st, [P, P, I32_, P, P, S, P, P]),
        "spgemm_mask_fill": (st, [P, P, I32_, P, P, P, P]),
        "spgemm_mcl_prune_count": (st, [P, ctypes.c_double, P, P, S, P, P]),
        "spgemm_mcl_prune_fill": (st, [P, ctypes.c_double, P, P, S, P, P, P]),
        "spgemm_sizer_forward": (st, [P, I64_, I32_, P, P, P]),
        "spgemm_sizer_grad": (st, [P, P, I64_, I32_, P, P, P, P]),
        "spgemm_sizer_train": (st, [P, P, P, I64_, I32_, P, P, P, P, I32_, I32_, ctypes.c_float, P, P]),
        "spgemm_row_features": (st, [P, P]),
        "spgemm_sizer_targets": (st, [P, I64_, P, P]),
        "spgemm_sizer_save": (st, [P, I32_, P, P, S, P]),
        "spgemm_sizer_load": (st, [P, S, I32_, P, P]),
        "spgemm_learned_multiply": (st, [P, P, P, P, ctypes.c_float, P, P, P, P]),
        "spgemm_transpose": (st, [P, P, P, S, P, P, P]),
        "spgemm_plan_info": (st, [P, P]),
        "spgemm_workspace_size": (st, [P, P]),
        "spgemm_symbolic": (st, [P, P, S, P, P]),
        "spgemm_numeric": (st, [P, P, S, P, P, P]),
        "spgemm_check": (st, [P]),
        "spgemm_plan_destroy": (None, [P]),
        "spgemm_kslice_bounds": (st, [P, I32_, P, P]),
        "spgemm_merge_workspace_size": (S, [I32_, I64_, I64_]),
        "spgemm_merge_symbolic": (st, [I32_, P, P, P, P, S, P, P]),
        "spgemm_merge_numeric": (st, [I32_, P, P, P, P, S, P, P, P]),
        "spgemm_merge_check": (st, [P, P]),
        "spgemm_merge_symbolic_static": (st, [I32_, P, P, P, P, P]),
        "spgemm_chain_workspace_size": (S, [I32_]),
        "spgemm_chain_create": (st, [I32_, P, P, P, S, P]),
        "spgemm_chain_launch": (st, [P, P]),
        "spgemm_chain_check": (st, [P, P]),
        "spgemm_chain_grid": (I32_, [P]),
        "spgemm_chain_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
LIBRARY_PATH = _build.LIB


def version() -> str:
    return _lib.spgemm_version().decode()


def kernel_launches() -> int:
    """Kernels this library has launched in this process."""
    return int(_lib.spgemm_kernel_launches())


def _check(status: int):
    if status != 0:
        raise SpgemmError(status, _lib.spgemm_last_error().decode())


@dataclasses.dataclass
class DeviceCSR:
    """CSR on the GPU: rowptr int64 [nrows+1] (or per-row starts when rowend
    is given), col int32/int64, val float64/float32/int64 or None."""

    nrows: int
    ncols: int
    rowptr: torch.Tensor
    col: torch.Tensor
    val: Optional[torch.Tensor]
    rowend: Optional[torch.Tensor] = None

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def index_type(self) -> int:
        return INDEX_I32 if self.col.dtype == torch.int32 else INDEX_I64

    @property
    def value_type(self) -> int:
        if self.val is None:
            return BOOL
        return {torch.float64: F64, torch.float32: F32, torch.int64: I64}[self.val.dtype]

    def to_host(self):
        """Returns (rowptr, col, val) numpy arrays (rowptr always plain CSR)."""
        rp = self.rowptr.cpu().numpy()
        col = self.col.cpu().numpy()
        val = None if self.val is None else self.val.cpu().numpy()
        return rp, col, val


def to_device(M, device="cuda") -> DeviceCSR:
    """Copies a host CSR (any object with nrows, ncols, rowptr, col, val)."""
    val = None if M.val is None else torch.from_numpy(np.ascontiguousarray(M.val)).to(device)
    return DeviceCSR(int(M.nrows), int(M.ncols),
                     torch.from_numpy(np.ascontiguousarray(M.rowptr, dtype=np.int64)).to(device),
                     torch.from_numpy(np.ascontiguousarray(M.col)).to(device), val)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None or t.numel() == 0 and t.data_ptr() == 0 else ctypes.c_void_p(t.data_ptr())


def _csr(M: DeviceCSR, value_type: Optional[int] = None) -> _Csr:
    for t in (M.rowptr, M.col, M.val, M.rowend):
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("CSR arrays must be contiguous CUDA tensors")
    return _Csr(M.nrows, M.ncols, M.nnz if M.rowend is None else int(M.col.numel()),
                M.rowptr.data_ptr(), None if M.rowend is None else M.rowend.data_ptr(),
                M.col.data_ptr() if M.col.numel() else None,
                None if M.val is None or M.val.numel() == 0 else M.val.data_ptr(),
                M.index_type, M.value_type if value_type is None else value_type)


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


class Plan:
    """A planned product C = A.B (spgemm_plan); keeps A, B and its
    workspaces alive until closed."""

    def __init__(self, A: DeviceCSR, B: DeviceCSR, semiring: int = PLUS_TIMES,
                 checked: bool = False, stream=None, dense_chunk: int = 0,
                 tuning: Optional[Tuning] = None):
        self.A, self.B = A, B
        self.device = A.rowptr.device
        self._cA, self._cB = _csr(A), _csr(B)
        self._opts = _make_opts(semiring, checked, tuning, dense_chunk)
        self.pattern_only = semiring == OR_AND or A.val is None
        self.stream = stream
        self._plan_ws = _workspace(_lib.spgemm_plan_workspace_size(A.nrows), self.device)
        h = ctypes.c_void_p()
        _check(_lib.spgemm_plan(ctypes.byref(self._cA), ctypes.byref(self._cB),
                                ctypes.byref(self._opts), _stream(stream),
                                ctypes.c_void_p(self._plan_ws.data_ptr()),
                                self._plan_ws.numel(), ctypes.byref(h)))
        self._h = h
        nb = ctypes.c_size_t()
        _check(_lib.spgemm_workspace_size(self._h, ctypes.byref(nb)))
        self.ws = _workspace(nb.value, self.device)

    def info(self) -> dict:
        inf = _Info()
        _check(_lib.spgemm_plan_info(self._h, ctypes.byref(inf)))
        return {name: getattr(inf, name) for name, _ in _Info._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.spgemm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan(A: DeviceCSR, B: DeviceCSR, semiring: int = PLUS_TIMES, checked: bool = False,
         stream=None, dense_chunk: int = 0, tuning: Optional[Tuning] = None) -> Plan:
    return Plan(A, B, semiring, checked, stream, dense_chunk, tuning)


class BatchPlan(Plan):
    """spgemm_batch_plan (device_sized=False) or spgemm_plan_device
    (device_sized=True) over products C_p = As[p] . Bs[p]."""

    def __init__(self, As: Sequence[DeviceCSR], Bs: Sequence[DeviceCSR], semiring: int = PLUS_TIMES,
                 checked: bool = False, stream=None, dense_chunk: int = 0,
                 dense_min_flops: int = 0, device_sized: bool = False, max_row_nnz: int = 0,
                 tuning: Optional[Tuning] = None):
        self.As, self.Bs = list(As), list(Bs)
        self.A, self.B = self.As[0], self.Bs[0]
        self.device = self.A.rowptr.device
        self.count = len(self.As)
        self._cAs = (_Csr * self.count)(*[_csr(M) for M in self.As])
        self._cBs = (_Csr * self.count)(*[_csr(M) for M in self.Bs])
        self._opts = _make_opts(semiring, checked, tuning, dense_chunk, dense_min_flops,
                                max_row_nnz)
        self.pattern_only = semiring == OR_AND or self.A.val is None
        self.stream = stream
        self.device_sized = device_sized
        self.rows = [M.nrows for M in self.As]
        self.row_base = np.concatenate([[0], np.cumsum(self.rows)]).astype(np.int64)
        self.R = int(self.row_base[-1])
        nbytes = _lib.spgemm_batch_plan_workspace_size(self.count, self._cAs)
        self._plan_ws = _workspace(nbytes, self.device)
        h = ctypes.c_void_p()
        fn = _lib.spgemm_plan_device if device_sized else _lib.spgemm_batch_plan
        _check(fn(self.count, self._cAs, self._cBs, ctypes.byref(self._opts), _stream(stream),
                  ctypes.c_void_p(self._plan_ws.data_ptr()), self._plan_ws.numel(),
                  ctypes.byref(h)))
        self._h = h
        nb = ctypes.c_size_t()
        _check(_lib.spgemm_workspace_size(self._h, ctypes.byref(nb)))
        self.ws = _workspace(nb.value, self.device)


def batch_plan(As, Bs, semiring: int = PLUS_TIMES, checked: bool = False, stream=None,
               dense_chunk: int = 0, dense_min_flops: int = 0,
               tuning: Optional[Tuning] = None) -> BatchPlan:
    return BatchPlan(As, Bs, semiring, checked, stream, dense_chunk, dense_min_flops,
                     tuning=tuning)


def device_plan(As, Bs, semiring: int = PLUS_TIMES, stream=None, dense_chunk: int = 0,
                dense_min_flops: int = 0, max_row_nnz: int = 0,
                tuning: Optional[Tuning] = None) -> BatchPlan:
    return BatchPlan(As, Bs, semiring, False, stream, dense_chunk, dense_min_flops,
                     device_sized=True, max_row_nnz=max_row_nnz, tuning=tuning)


def execute(p: BatchPlan, rowptrC: torch.Tensor, capacity: int, colC: torch.Tensor,
            valC: Optional[torch.Tensor]) -> None:
    """spgemm_execute: the whole batch enqueued with no host readback."""
    _check(_lib.spgemm_execute(p._h, ctypes.c_void_p(p.ws.data_ptr()), p.ws.numel(),
                               ctypes.c_void_p(rowptrC.data_ptr()), int(capacity),
                               ctypes.c_void_p(colC.data_ptr()) if colC.numel() else None,
                               None if valC is None or valC.numel() == 0
                               else ctypes.c_void_p(valC.data_ptr())))


class _ChainStep(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t),
                ("rowptrC", ctypes.c_void_p), ("capacity", ctypes.c_int64),
                ("colC", ctypes.c_void_p), ("valC", ctypes.c_void_p)]


class _ChainOpts(ctypes.Structure):
    _fields_ = [("timeout_s", ctypes.c_double), ("withhold_stage", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("stage_ns", ctypes.c_void_p)]


CHAIN_STAGES = ("analysis", "binning", "symbolic", "scan sums", "scan apply", "numeric")


class Chain:
    """spgemm_chain_*: device-sized products run in ONE persistent kernel
    launch.  steps: (plan from device_plan, rowptrC, capacity, colC, valC); a
    step may read an earlier step's outputs.  launch() enqueues (capturable
    in a CUDA graph), check() waits and raises SpgemmError(TIMEOUT) when a
    barrier wait expired.  With record_stages, every launch records when
    block 0 passed each barrier; stage_ms() returns the stage durations.
    block_threads: 0 (768) or 1024 (spgemm_chain_opts.block_threads)."""

    def __init__(self, steps, timeout_s: float = 0.0, withhold_stage: int = -1,
                 record_stages: bool = False, block_threads: int = 0):
        self._steps = list(steps)
        dev = self._steps[0][1].device
        arr = (_ChainStep * len(self._steps))()
        for t, (p, rp, cap, col, val) in enumerate(self._steps):
            arr[t] = _ChainStep(p._h.value, p.ws.data_ptr(), p.ws.numel(), rp.data_ptr(), int(cap),
                                col.data_ptr() if col is not None and col.numel() else None,
                                None if val is None or val.numel() == 0 else val.data_ptr())
        self.ws = _workspace(_lib.spgemm_chain_workspace_size(len(self._steps)), dev)
        self.stamps = (torch.zeros(2 + 6 * len(self._steps), dtype=torch.int64, device=dev)
                       if record_stages else None)
        opts = _ChainOpts(float(timeout_s), int(withhold_stage), int(block_threads),
                          None if self.stamps is None else self.stamps.data_ptr())
        h = ctypes.c_void_p()
        _check(_lib.spgemm_chain_create(len(self._steps), arr, ctypes.byref(opts),
                                        ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                        ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(_lib.spgemm_chain_launch(self._h, _stream(stream)))

    def check(self, stream=None):
        _check(_lib.spgemm_chain_check(self._h, _stream(stream)))
        for p, *_ in self._steps:
            check(p)

    def grid(self) -> int:
        return int(_lib.spgemm_chain_grid(self._h))

    def stage_ms(self):
        """[(step, stage name, ms)] of the last launch (record_stages), the
        counter-clearing stage as step -1."""
        if self.stamps is None:
            raise ValueError("chain created without record_stages")
        t = self.stamps.cpu().tolist()
        out = [(-1, "clear", (t[1] - t[0]) * 1e-6)]
        for q in range(len(self._steps)):
            for j, name in enumerate(CHAIN_STAGES):
                k = 1 + 6 * q + j
                out.append((q, name, (t[k + 1] - t[k]) * 1e-6))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.spgemm_chain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_rowptrs(p: BatchPlan, rowptrC: torch.Tensor) -> torch.Tensor:
    """Per-product row pointers (each m_p + 1 entries, one after the other)."""
    out = torch.empty(p.R + p.count, dtype=torch.int64, device=p.device)
    _check(_lib.spgemm_batch_rowptrs(p._h, ctypes.c_void_p(rowptrC.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr())))
    return out


def split_batch(p: BatchPlan, rowptrC: torch.Tensor, colC: torch.Tensor,
                valC: Optional[torch.Tensor]) -> List[DeviceCSR]:
    """Views of the products of a batch result (no copy of columns/values)."""
    rps = batch_rowptrs(p, rowptrC)
    starts = rowptrC[torch.as_tensor(p.row_base, device=p.device)].cpu().numpy()
    out = []
    for q in range(p.count):
        m = p.rows[q]
        rp = rps[p.row_base[q] + q: p.row_base[q] + q + m + 1]
        a, b = int(starts[q]), int(starts[q + 1])
        out.append(DeviceCSR(m, p.Bs[q].ncols, rp, colC[a:b],
                             None if valC is None else valC[a:b]))
    return out


def batch_spgemm(As, Bs, semiring: int = PLUS_TIMES, checked: bool = False, stream=None,
                 verify: bool = False, dense_chunk: int = 0,
                 dense_min_flops: int = 0, tuning: Optional[Tuning] = None) -> List[DeviceCSR]:
    """All products C_p = As[p] . Bs[p] with one plan (one launch per phase)."""
    p = batch_plan(As, Bs, semiring, checked, stream, dense_chunk, dense_min_flops, tuning)
    rowptrC, nnz = symbolic(p)
    colC, valC = alloc_output(p, nnz)
    numeric(p, rowptrC, colC, valC)
    if verify:
        check(p)
    res = split_batch(p, rowptrC, colC, valC)
    p.close()
    return res


def symbolic(p: Plan, rowptrC: Optional[torch.Tensor] = None):
    """Row pointers of C and nnz(C) (waits for the stream)."""
    if rowptrC is None:
        rowptrC = torch.empty(getattr(p, "R", p.A.nrows) + 1, dtype=torch.int64, device=p.device)
    nnz = ctypes.c_int64()
    _check(_lib.spgemm_symbolic(p._h, ctypes.c_void_p(p.ws.data_ptr()), p.ws.numel(),
                                ctypes.c_void_p(rowptrC.data_ptr()), ctypes.byref(nnz)))
    return rowptrC, int(nnz.value)


def numeric(p: Plan, rowptrC: torch.Tensor, colC: torch.Tensor,
            valC: Optional[torch.Tensor]) -> None:
    _check(_lib.spgemm_numeric(p._h, ctypes.c_void_p(p.ws.data_ptr()), p.ws.numel(),
                               ctypes.c_void_p(rowptrC.data_ptr()),
                               ctypes.c_void_p(colC.data_ptr()) if colC.numel() else None,
                               None if valC is None or valC.numel() == 0
                               else ctypes.c_void_p(valC.data_ptr())))


def check(p: Plan) -> None:
    _check(_lib.spgemm_check(p._h))


def alloc_output(p: Plan, nnz: int):
    colC = torch.empty(nnz, dtype=p.A.col.dtype, device=p.device)
    valC = None if p.pattern_only else torch.empty(nnz, dtype=p.A.val.dtype, device=p.device)
    return colC, valC


def spgemm(A: DeviceCSR, B: DeviceCSR, semiring: int = PLUS_TIMES, checked: bool = False,
           stream=None, verify: bool = False, dense_chunk: int = 0,
           tuning: Optional[Tuning] = None) -> DeviceCSR:
    """C = A.B: plan, symbolic, allocate C, numeric."""
    p = plan(A, B, semiring, checked, stream, dense_chunk, tuning)
    rowptrC, nnz = symbolic(p)
    colC, valC = alloc_output(p, nnz)
    numeric(p, rowptrC, colC, valC)
    if verify:
        check(p)
    p.close()
    return DeviceCSR(A.nrows, B.ncols, rowptrC, colC, valC)


def transpose(A: DeviceCSR, stream=None) -> DeviceCSR:
    """A^T with ascending columns (spgemm_transpose)."""
    cA = _csr(A)
    ws = _workspace(_lib.spgemm_transpose_workspace_size(ctypes.byref(cA)), A.rowptr.device)
    rp = torch.empty(A.ncols + 1, dtype=torch.int64, device=A.rowptr.device)
    col = torch.empty(A.nnz, dtype=A.col.dtype, device=A.rowptr.device)
    val = None if A.val is None else torch.empty(A.nnz, dtype=A.val.dtype, device=A.rowptr.device)
    _check(_lib.spgemm_transpose(ctypes.byref(cA), _stream(stream), ctypes.c_void_p(ws.data_ptr()),
                                 ws.numel(), ctypes.c_void_p(rp.data_ptr()),
                                 ctypes.c_void_p(col.data_ptr()) if A.nnz else None,
                                 None if val is None or A.nnz == 0 else ctypes.c_void_p(val.data_ptr())))
    return DeviceCSR(A.ncols, A.nrows, rp, col, val)


# ------------------------------------------------------------ MCL epilogue
def mcl_prune(C: DeviceCSR, threshold: float = 1e-4, stream=None) -> DeviceCSR:
    """Drop entries below threshold, renormalise rows (float64)."""
    cC = _csr(C)
    dev = C.rowptr.device
    ws = _workspace(_lib.spgemm_mcl_workspace_size(C.nrows), dev)
    rp = torch.empty(C.nrows + 1, dtype=torch.int64, device=dev)
    nnz = ctypes.c_int64()
    _check(_lib.spgemm_mcl_prune_count(ctypes.byref(cC), ctypes.c_double(threshold), _stream(stream),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       ctypes.c_void_p(rp.data_ptr()), ctypes.byref(nnz)))
    col = torch.empty(nnz.value, dtype=C.col.dtype, device=dev)
    val = torch.empty(nnz.value, dtype=torch.float64, device=dev)
    _check(_lib.spgemm_mcl_prune_fill(ctypes.byref(cC), ctypes.c_double(threshold), _stream(stream),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      ctypes.c_void_p(rp.data_ptr()),
                                      ctypes.c_void_p(col.data_ptr()) if nnz.value else None,
                                      ctypes.c_void_p(val.data_ptr()) if nnz.value else None))
    return DeviceCSR(C.nrows, C.ncols, rp, col, val)


def mask(C: DeviceCSR, M: DeviceCSR, complement: bool = False, stream=None) -> DeviceCSR:
    """Entries of C inside the pattern of M (or outside it with complement)."""
    dev = C.rowptr.device
    cC, cM = _csr(C), _csr(M)
    ws = _workspace(_lib.spgemm_mask_workspace_size(C.nrows), dev)
    rp = torch.empty(C.nrows + 1, dtype=torch.int64, device=dev)
    nnz = ctypes.c_int64()
    _check(_lib.spgemm_mask_count(ctypes.byref(cC), ctypes.byref(cM), 1 if complement else 0,
                                  _stream(stream), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  ctypes.c_void_p(rp.data_ptr()), ctypes.byref(nnz)))
    col = torch.empty(nnz.value, dtype=C.col.dtype, device=dev)
    val = None if C.val is None else torch.empty(nnz.value, dtype=C.val.dtype, device=dev)
    _check(_lib.spgemm_mask_fill(ctypes.byref(cC), ctypes.byref(cM), 1 if complement else 0,
                                 _stream(stream), ctypes.c_void_p(rp.data_ptr()),
                                 ctypes.c_void_p(col.data_ptr()) if col.numel() else None,
                                 _ptr(val) if val is not None and val.numel() else None))
    return DeviceCSR(C.nrows, C.ncols, rp, col, val)


def dcsr_view(A: DeviceCSR, stream=None):
    """The nonempty rows of A (spgemm_dcsr_view): returns (rowids, view)."""
    dev = A.rowptr.device
    m = A.nrows
    ws = _workspace(_lib.spgemm_dcsr_workspace_size(m), dev)
    ids = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
    rp = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
    re = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
    nzr = ctypes.c_int64()
    _check(_lib.spgemm_dcsr_view(ctypes.byref(_csr(A)), _stream(stream),
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(rp.data_ptr()),
                                 ctypes.c_void_p(re.data_ptr()), ctypes.byref(nzr)))
    k = int(nzr.value)
    return ids[:k], DeviceCSR(k, A.ncols, rp[:k], A.col, A.val, rowend=re[:k])


def dcsr_expand(C: DeviceCSR, rowids: torch.Tensor, m: int, stream=None) -> DeviceCSR:
    """The product of a DCSR view with its row pointers expanded to all m rows."""
    full = torch.empty(m + 1, dtype=torch.int64, device=C.rowptr.device)
    _check(_lib.spgemm_dcsr_expand(m, C.nrows, ctypes.c_void_p(rowids.data_ptr()) if C.nrows else None,
                                   ctypes.c_void_p(C.rowptr.data_ptr()), _stream(stream),
                                   ctypes.c_void_p(full.data_ptr())))
    return DeviceCSR(m, C.ncols, full, C.col, C.val)


def mis2_restriction(A: DeviceCSR, seed: int, stream=None):
    """MIS-2 aggregation of the graph of A (spgemm_mis2_restriction): returns
    (R as a DeviceCSR n x naggs with values 1.0, rounds)."""
    dev = A.rowptr.device
    n = A.nrows
    ws = _workspace(_lib.spgemm_mis2_workspace_size(n), dev)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(n, 1), dtype=A.col.dtype, device=dev)
    val = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    naggs = ctypes.c_int64()
    rounds = ctypes.c_int32()
    _check(_lib.spgemm_mis2_restriction(ctypes.byref(_csr(A)), ctypes.c_uint64(seed),
                                        _stream(stream), ctypes.c_void_p(ws.data_ptr()),
                                        ws.numel(), ctypes.c_void_p(rp.data_ptr()),
                                        ctypes.c_void_p(col.data_ptr()),
                                        ctypes.c_void_p(val.data_ptr()), ctypes.byref(naggs),
                                        ctypes.byref(rounds)))
    return DeviceCSR(n, int(naggs.value), rp, col[:n], val[:n]), int(rounds.value)


def masked_spgemm(A: DeviceCSR, B: DeviceCSR, M: DeviceCSR, semiring: int = PLUS_TIMES,
                  complement: bool = False, stream=None) -> DeviceCSR:
    """(A.B) restricted to the pattern of M (or to its complement)."""
    return mask(spgemm(A, B, semiring, stream=stream), M, complement, stream)


def mcl_step(M: DeviceCSR, threshold: float = 1e-4, params: Optional[torch.Tensor] = None,
             margin: float = 0.25, stream=None, panel_bytes: float = 32e9,
             stats: Optional[dict] = None, compare_every: int = 0) -> DeviceCSR:
    """One MCL expansion on M^T in CSR: (M M)^T = M^T M^T, then the epilogue.
    With params the product uses learned sizing.  When the unpruned product
    could exceed panel_bytes (flops bound x 12 bytes), rows are processed in
    panels, each pruned before the next is formed.  With `stats` (a dict),
    the step records its flops, panels, nnz before and after pruning and the
    product / prune times (CUDA events, milliseconds).  With params and
    compare_every = k > 0, every k-th panel is also formed by the exact
    two-phase product; stats then records both paths' times on those panels
    and whether their pruned outputs are identical."""
    fl = plan(M, M, stream=stream).info()["flops"]
    npan = max(1, int(np.ceil(fl * (M.col.element_size() + 8) / panel_bytes)))
    parts = []
    if stats is not None:
        stats.update(flops=int(fl), panels=npan, nnz_product=0, product_ms=0.0, prune_ms=0.0)
        if params is not None and compare_every > 0:
            stats.update(compared_panels=0, compared_identical=True, compared_learned_ms=0.0,
                         compared_plain_ms=0.0)
        s_ = torch.cuda.current_stream() if stream is None else stream
    for p in range(npan):
        a, b = (M.nrows * p) // npan, (M.nrows * (p + 1)) // npan
        V = M if npan == 1 else DeviceCSR(b - a, M.ncols, M.rowptr[a:b], M.col, M.val,
                                          rowend=M.rowptr[a + 1:b + 1])
        if stats is not None:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(s_)
        if params is None:
            C = spgemm(V, M, stream=stream)
        else:
            C, _ = learned_multiply(V, M, params, margin, stream=stream)
        if stats is not None:
            ev[1].record(s_)
        parts.append(mcl_prune(C, threshold, stream))
        if stats is not None:
            ev[2].record(s_)
            ev[2].synchronize()
            stats["product_ms"] += ev[0].elapsed_time(ev[1])
            stats["prune_ms"] += ev[1].elapsed_time(ev[2])
            stats["nnz_product"] += int(C.rowend.sum() - C.rowptr[:-1].sum()) \
                if C.rowend is not None else int(C.nnz)
            if params is not None and compare_every > 0 and p % compare_every == 0:
                ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev2[0].record(s_)
                Cp = spgemm(V, M, stream=stream)
                Pp = mcl_prune(Cp, threshold, stream)
                ev2[1].record(s_)
                ev2[1].synchronize()
                L = parts[-1]
                stats["compared_panels"] += 1
                stats["compared_learned_ms"] += ev[0].elapsed_time(ev[2])
                stats["compared_plain_ms"] += ev2[0].elapsed_time(ev2[1])
                stats["compared_identical"] = bool(
                    stats["compared_identical"] and torch.equal(Pp.rowptr, L.rowptr)
                    and torch.equal(Pp.col, L.col)
                    and torch.equal(Pp.val.view(torch.int64), L.val.view(torch.int64)))
                del Cp, Pp
        del C
    if stats is not None:
        stats["nnz_pruned"] = int(sum(P.nnz for P in parts))
    if npan == 1:
        return parts[0]
    offs = np.cumsum([0] + [P.nnz for P in parts])
    rowptr = torch.cat([parts[0].rowptr[:1]] + [P.rowptr[1:] + int(o) for P, o in zip(parts, offs)])
    return DeviceCSR(M.nrows, M.ncols, rowptr, torch.cat([P.col for P in parts]),
                     torch.cat([P.val for P in parts]))


# ------------------------------------------------------------ learned sizing
SIZER_F = 6
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class _LearnedResult(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("rowend", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("slot_total", ctypes.c_int64), ("overflow_rows", ctypes.c_int64),
                ("total_flops", ctypes.c_int64)]


def sizer_param_count(F: int = SIZER_F) -> int:
    return int(_lib.spgemm_sizer_param_count(F))


def sizer_forward(X: torch.Tensor, params: torch.Tensor, stream=None) -> torch.Tensor:
    N, F = X.shape
    y = torch.empty(N, dtype=torch.float32, device=X.device)
    _check(_lib.spgemm_sizer_forward(ctypes.c_void_p(X.data_ptr()), N, F,
                                     ctypes.c_void_p(params.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), _stream(stream)))
    return y


def sizer_grad(X: torch.Tensor, T: torch.Tensor, params: torch.Tensor, stream=None):
    N, F = X.shape
    g = torch.empty(sizer_param_count(F), dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(_lib.spgemm_sizer_grad(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                  N, F, ctypes.c_void_p(params.data_ptr()),
                                  ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                  _stream(stream)))
    return g, loss


def sizer_init(F: int = SIZER_F, seed: int = 0, device="cuda") -> torch.Tensor:
    """He-style random initial parameters (seeded, drawn on the host)."""
    rng = np.random.default_rng(seed)
    H = 32
    parts = [rng.normal(0, np.sqrt(2.0 / F), H * F), np.zeros(H),
             rng.normal(0, np.sqrt(2.0 / H), H * H), np.zeros(H),
             rng.normal(0, np.sqrt(1.0 / H), H), np.zeros(1)]
    return torch.tensor(np.concatenate(parts), dtype=torch.float32, device=device)


def sizer_train(X: torch.Tensor, T: torch.Tensor, params: torch.Tensor, steps: int, batch: int,
                lr: float, seed: int = 0, stream=None) -> torch.Tensor:
    """Adam steps on (X, T) in place on params; returns the per-step loss."""
    N, F = X.shape
    order = torch.from_numpy(np.random.default_rng(seed).permutation(N).astype(np.int64)).to(X.device)
    P = sizer_param_count(F)
    m = torch.zeros(P, dtype=torch.float32, device=X.device)
    v = torch.zeros(P, dtype=torch.float32, device=X.device)
    g = torch.empty(P, dtype=torch.float32, device=X.device)
    trace = torch.empty(max(steps, 1), dtype=torch.float32, device=X.device)
    _check(_lib.spgemm_sizer_train(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                   ctypes.c_void_p(order.data_ptr()), N, F,
                                   ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                                   ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                   steps, batch, ctypes.c_float(lr),
                                   ctypes.c_void_p(trace.data_ptr()), _stream(stream)))
    return trace[:steps]


def row_features(p: Plan) -> torch.Tensor:
    X = torch.empty((getattr(p, "R", p.A.nrows), SIZER_F), dtype=torch.float32, device=p.device)
    _check(_lib.spgemm_row_features(p._h, ctypes.c_void_p(X.data_ptr())))
    return X


def sizer_targets(rowptrC: torch.Tensor, stream=None) -> torch.Tensor:
    """spgemm_sizer_targets: log2(1 + nnz(C(i,:))) per row."""
    m = rowptrC.numel() - 1
    T = torch.empty(max(m, 0), dtype=torch.float32, device=rowptrC.device)
    _check(_lib.spgemm_sizer_targets(ctypes.c_void_p(rowptrC.data_ptr()), m,
                                     ctypes.c_void_p(T.data_ptr()) if m > 0 else None,
                                     _stream(stream)))
    return T


def sizer_training_set(pairs, stream=None):
    """(features, targets) of every row with products (first feature
    log2(1 + flops) > 0) of the given products; the targets come from the
    exact symbolic phase (spgemm_sizer_targets)."""
    Xs, Ts = [], []
    for A, B in pairs:
        p = plan(A, B, stream=stream)
        X = row_features(p)
        rp, _ = symbolic(p)
        T = sizer_targets(rp, stream)
        keep = X[:, 0] > 0
        Xs.append(X[keep])
        Ts.append(T[keep])
        p.close()
    return torch.cat(Xs), torch.cat(Ts)


def sizer_save(params: torch.Tensor, F: int = SIZER_F, stream=None) -> bytes:
    """spgemm_sizer_save: the trained predictor as a versioned byte record."""
    need = ctypes.c_size_t()
    _check(_lib.spgemm_sizer_save(None, F, None, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(_lib.spgemm_sizer_save(ctypes.c_void_p(params.data_ptr()), F, _stream(stream), buf,
                                  need.value, ctypes.byref(need)))
    return buf.raw[: need.value]


def sizer_load(record: bytes, F: int = SIZER_F, device="cuda", stream=None) -> torch.Tensor:
    """spgemm_sizer_load: parameters from a record written by sizer_save."""
    params = torch.empty(sizer_param_count(F), dtype=torch.float32, device=device)
    _check(_lib.spgemm_sizer_load(record, len(record), F, ctypes.c_void_p(params.data_ptr()),
                                  _stream(stream)))
    return params


def learned_multiply(A: DeviceCSR, B: DeviceCSR, params: torch.Tensor, margin: float = 0.25,
                     semiring: int = PLUS_TIMES, stream=None, dense_min_flops: int = 0,
                     tuning: Optional[Tuning] = None):
    """C = A.B with learned sizing (spgemm_learned_multiply).  Returns
    (C, stats); C carries rowend when it is returned as slots."""
    keep = []
    dev = A.rowptr.device

    def alloc(nbytes, ctx):
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=dev)
        keep.append(t)
        return t.data_ptr()

    cb = _ALLOC_FN(alloc)
    cA, cB = _csr(A), _csr(B)
    opts = _make_opts(semiring, False, tuning, 0, dense_min_flops)
    res = _LearnedResult()
    _check(_lib.spgemm_learned_multiply(ctypes.byref(cA), ctypes.byref(cB), ctypes.byref(opts),
                                        ctypes.c_void_p(params.data_ptr()), ctypes.c_float(margin),
                                        _stream(stream), cb, None, ctypes.byref(res)))
    by_ptr = {t.data_ptr(): t for t in keep}

    def view(ptr, dtype, count):
        if count == 0:
            return torch.empty(0, dtype=dtype, device=dev)
        t = by_ptr[ptr]
        return t[: count * torch.empty(0, dtype=dtype).element_size()].view(dtype)

    m = res.nrows
    rowptr = view(res.rowptr, torch.int64, m + 1)
    rowend = view(res.rowend, torch.int64, m) if res.rowend else None
    col = view(res.col, A.col.dtype, res.nnz)
    pattern = semiring == OR_AND or A.val is None
    val = None if pattern else view(res.val, A.val.dtype, res.nnz)
    C = DeviceCSR(m, res.ncols, rowptr, col, val, rowend=rowend)
    stats = {"slot_total": res.slot_total, "overflow_rows": res.overflow_rows,
             "flops": res.total_flops, "slots": res.rowend is not None}
    C._keep = keep
    return C, stats


def compact(C: DeviceCSR) -> DeviceCSR:
    """A plain CSR copy of a CSR view (rowend given): rows packed."""
    if C.rowend is None:
        return C
    return merge([DeviceCSR(C.nrows, C.ncols, C.rowptr, C.col, C.val, rowend=C.rowend)])


def kslice_bounds(A: DeviceCSR, c: int, stream=None) -> torch.Tensor:
    """(c+1) x m int64: slice s of row i is [b[s, i], b[s+1, i])."""
    b = torch.empty((c + 1, A.nrows), dtype=torch.int64, device=A.rowptr.device)
    cA = _csr(A)
    _check(_lib.spgemm_kslice_bounds(ctypes.byref(cA), c, _stream(stream),
                                     ctypes.c_void_p(b.data_ptr()) if b.numel() else None))
    return b


def kslice_views(A: DeviceCSR, c: int, stream=None) -> List[DeviceCSR]:
    b = kslice_bounds(A, c, stream)
    return [DeviceCSR(A.nrows, A.ncols, b[s], A.col, A.val, rowend=b[s + 1]) for s in range(c)]


def _parts(parts: Sequence[DeviceCSR]):
    arr = (_Csr * len(parts))(*[_csr(P) for P in parts])
    return arr


def merge_workspace(c: int, m: int, n: int, device) -> torch.Tensor:
    return _workspace(_lib.spgemm_merge_workspace_size(c, m, n), device)


def merge_symbolic(parts: Sequence[DeviceCSR], ws: torch.Tensor, semiring: int = PLUS_TIMES,
                   stream=None, rowptrC: Optional[torch.Tensor] = None):
    m = parts[0].nrows
    if rowptrC is None:
        rowptrC = torch.empty(m + 1, dtype=torch.int64, device=ws.device)
    arr = _parts(parts)
    opts = _Opts(semiring, 0)
    nnz = ctypes.c_int64()
    _check(_lib.spgemm_merge_symbolic(len(parts), arr, ctypes.byref(opts), _stream(stream),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      ctypes.c_void_p(rowptrC.data_ptr()), ctypes.byref(nnz)))
    return rowptrC, int(nnz.value)


def merge_symbolic_static(parts: Sequence[DeviceCSR], semiring: int = PLUS_TIMES, stream=None,
                          rowptrC: Optional[torch.Tensor] = None):
    """spgemm_merge_symbolic_static: the merge count with no workspace (the
    library's fixed device scratch array is used instead)."""
    m = parts[0].nrows
    if rowptrC is None:
        rowptrC = torch.empty(m + 1, dtype=torch.int64, device=parts[0].rowptr.device)
    arr = _parts(parts)
    opts = _Opts(semiring, 0)
    nnz = ctypes.c_int64()
    _check(_lib.spgemm_merge_symbolic_static(len(parts), arr, ctypes.byref(opts),
                                             _stream(stream),
                                             ctypes.c_void_p(rowptrC.data_ptr()),
                                             ctypes.byref(nnz)))
    return rowptrC, int(nnz.value)


def merge_numeric(parts: Sequence[DeviceCSR], ws: torch.Tensor, rowptrC: torch.Tensor,
                  colC: torch.Tensor, valC: Optional[torch.Tensor], semiring: int = PLUS_TIMES,
                  stream=None, staged: bool = False) -> None:
    """spgemm_merge_numeric; staged: entries staged in shared memory by bulk
    asynchronous copies (spgemm_opts.merge_staged)."""
    arr = _parts(parts)
    opts = _Opts(semiring, 0)
    opts.merge_staged = 1 if staged else 0
    _check(_lib.spgemm_merge_numeric(len(parts), arr, ctypes.byref(opts), _stream(stream),
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                     ctypes.c_void_p(rowptrC.data_ptr()),
                                     ctypes.c_void_p(colC.data_ptr()) if colC.numel() else None,
                                     None if valC is None or valC.numel() == 0
                                     else ctypes.c_void_p(valC.data_ptr())))


def merge_check(ws: torch.Tensor, stream=None) -> None:
    _check(_lib.spgemm_merge_check(_stream(stream), ctypes.c_void_p(ws.data_ptr())))


def merge(parts: Sequence[DeviceCSR], semiring: int = PLUS_TIMES, stream=None,
          verify: bool = False, staged: bool = False) -> DeviceCSR:
    m, n = parts[0].nrows, parts[0].ncols
    ws = merge_workspace(len(parts), m, n, parts[0].rowptr.device)
    rowptrC, nnz = merge_symbolic(parts, ws, semiring, stream)
    pattern = semiring == OR_AND or parts[0].val is None
    colC = torch.empty(nnz, dtype=parts[0].col.dtype, device=ws.device)
    valC = None if pattern else torch.empty(nnz, dtype=parts[0].val.dtype, device=ws.device)
    merge_numeric(parts, ws, rowptrC, colC, valC, semiring, stream, staged=staged)
    if verify:
        merge_check(ws, stream)
    return DeviceCSR(m, n, rowptrC, colC, valC)


def spgemm_kslice(A: DeviceCSR, B: DeviceCSR, c: int, semiring: int = PLUS_TIMES,
                  stream=None, verify: bool = False, hypersparse: bool = False):
    """The k-split product: C_s = A(:,K_s).B for the c contiguous slices K_s
    of the inner dimension, then C = sum_s C_s by the merge.  With
    hypersparse, each slice is multiplied as a DCSR view of its nonempty rows
    and its row pointers are expanded afterwards.  Returns (C, partials)."""
    parts = []
    for As in kslice_views(A, c, stream):
        if hypersparse:
            ids, v = dcsr_view(As, stream)
            Cv = spgemm(v, B, semiring, stream=stream, verify=verify)
            parts.append(dcsr_expand(Cv, ids, A.nrows, stream))
        else:
            parts.append(spgemm(As, B, semiring, stream=stream, verify=verify))
    return merge(parts, semiring, stream, verify), parts
