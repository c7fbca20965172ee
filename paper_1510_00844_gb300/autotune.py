"""Autotuner of the runtime knobs of a plan (spgemm.Tuning).

Coordinate descent over the dense threshold (which rows use a dense
accumulator instead of a hash table), the hash-table sizing shift, the dense
chunk width and the dense work-unit size (how many warps share a dense row).
Every candidate is timed with CUDA events on the caller's own workload:
plan + symbolic + numeric for a product or a batch, one replay of the
captured graph for a Galerkin chain.  The paper's local multiply has fixed
parameters; this is an addition, and no knob changes the arithmetic: every
row is still accumulated over ascending k, so results are identical for all
candidates."""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import torch

from . import spgemm as sg
from .spgemm import Tuning

SPACE: Dict[str, Tuple[int, ...]] = {
    "dense_min_flops": (1024, 512, 256),
    "hash_shift": (0, 1),
    "dense_chunk": (1024, 2048),
    "seg_log2": (16, 18, 20, 22),
}


def _normal(t: Tuning) -> Tuning:
    """Spells out the library defaults (0 = default) so that equal settings
    are measured once."""
    return dataclasses.replace(t, dense_min_flops=t.dense_min_flops or 1024)


def descend(measure: Callable[[Tuning], float], space: Dict[str, Iterable[int]] = SPACE,
            base: Tuning = Tuning(), min_gain: float = 0.02):
    """Coordinate descent: for each knob in turn keep the value whose
    measured time beats the best so far by more than min_gain (relative).
    Returns (best tuning, {tuning: time}) with every measured candidate."""
    table: Dict[Tuning, float] = {}
    seen: Dict[Tuning, float] = {}

    def cost(t: Tuning) -> float:
        key = _normal(t)
        if key not in seen:
            seen[key] = float(measure(t))
        table[t] = seen[key]
        return seen[key]

    best = base
    best_ms = cost(best)
    for knob, values in space.items():
        for v in values:
            cand = dataclasses.replace(best, **{knob: v})
            ms = cost(cand)
            if ms < best_ms * (1.0 - min_gain):
                best, best_ms = cand, ms
    return best, table


def time_ms(step: Callable[[], None], repeats: int = 3, warmup: int = 1) -> float:
    """Median device time of step() on the current stream (synchronised)."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ts: List[float] = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def product(A: sg.DeviceCSR, B: sg.DeviceCSR, semiring: int = sg.PLUS_TIMES,
            space: Dict[str, Iterable[int]] = SPACE, repeats: int = 3):
    """Tuning for C = A.B (plan + symbolic + numeric timed per candidate)."""
    def measure(t: Tuning) -> float:
        return time_ms(lambda: sg.spgemm(A, B, semiring, tuning=t), repeats)
    return descend(measure, space)


def batch(As: Sequence[sg.DeviceCSR], Bs: Sequence[sg.DeviceCSR], semiring: int = sg.PLUS_TIMES,
          space: Dict[str, Iterable[int]] = SPACE, repeats: int = 3):
    """Tuning for a batch of products run with one plan."""
    def measure(t: Tuning) -> float:
        return time_ms(lambda: sg.batch_spgemm(As, Bs, semiring, tuning=t), repeats)
    return descend(measure, space)


def galerkin(A0: sg.DeviceCSR, Rs: Sequence[sg.DeviceCSR], stream: torch.cuda.Stream,
             space: Dict[str, Iterable[int]] = SPACE, repeats: int = 5,
             max_row_nnz: int = 64):
    """Tuning for a Galerkin hierarchy: one captured graph per candidate,
    timed by replay."""
    from .amg import GalerkinChain

    def measure(t: Tuning) -> float:
        chain = GalerkinChain(A0, list(Rs), stream, max_row_nnz=max_row_nnz, tuning=t)
        chain.capture()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ms = time_ms(chain.replay, repeats)
        del chain
        return ms
    return descend(measure, space)
