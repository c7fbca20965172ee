"""Benchmark of the sparse product C = A.A on R-MAT scale 18 (Graph500
parameters a=.57, b=c=.19, d=.05, edge factor 16, symmetrised, duplicates
summed, randomly permuted, float64 values U(0,1), int32 column indices).

One step = the whole plain two-phase path through the library: row analysis
and binning (spgemm_plan), symbolic phase and row pointers (spgemm_symbolic),
allocation of C, numeric phase (spgemm_numeric).  Inputs are resident in HBM
when the timed region starts; L2 is flushed (a 256 MiB write) between steps,
outside the timed events.  value = 2 * flops / time (GFLOP/s).

--impl reference times the CPU oracle (plain Gustavson with a dense
accumulator, all host cores) on a bounded sample of rows of the same
workload, with the same metric.

Multi-GPU (torchrun, N ranks): each rank multiplies a contiguous row panel of
A by the full A (rows are independent; no collective on the data path);
value = total flops of all ranks / max rank time ("scaling": "strong")."""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpGEMM GFLOP/s + HBM-roofline %, learned/batched vs plain 2-phase, 1 GB300"
UNIT = "GFLOP/s"
SCALE = 18
L2_FLUSH_BYTES = 256 << 20
FP64_LANES_PER_SM_CLK = 2
SMS = 152
SM_MAX_MHZ = 2070.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def algorithmic_bytes(A, nnz_c: int):
    """Bytes the plain two-phase method must move (symbolic + numeric):
    symbolic reads rowptr/col of A and B and writes rowptr(C); numeric reads
    rowptr/col/val of A and B and rowptr(C) and writes col/val of C."""
    m, nnzA = A.nrows, A.nnz
    idx, v, r = A.col.dtype.itemsize, 8, 8
    a_idx = r * (m + 1) + idx * nnzA
    sym = 2 * a_idx + 8 * (m + 1)
    num = 2 * (a_idx + v * nnzA) + 8 * (m + 1) + (idx + v) * nnz_c
    return sym, num


def dense_kernel_digest():
    """sha256 (first 16 hex) of the numeric_dense_kernel source: from its
    section comment of kernels.cuh to the end of its kernel wrapper (the
    learned path's packing kernel that follows is not part of it)."""
    import hashlib
    src = os.path.join(ROOT, "paper_1510_00844_gb300", "csrc", "kernels.cuh")
    text = open(src).read()
    a = text.index("// --------------------------------------------------- numeric: dense rows")
    b = text.index("// Learned sizing: close the gaps a slot-mode dense row leaves", a)
    return hashlib.sha256(text[a:b].encode()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of numeric_dense_kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "numeric_dense_rmat18.md")
    try:
        text = open(path).read()
        digest = dense_kernel_digest()
    except (OSError, ValueError):
        return None
    if f"`{digest}`" not in text:
        return None
    for ln in text.splitlines():
        if ln.startswith("traffic_bytes_per_launch_rmat18:"):
            return int(ln.split(":")[1])
    return None


def panel(m: int, world: int, rank: int):
    return (m * rank) // world, (m * (rank + 1)) // world


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1510_00844_gb300 import inputs
    from paper_1510_00844_gb300 import spgemm as sg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    A = inputs.rmat(SCALE)
    dA = sg.to_device(A, dev)
    r0, r1 = panel(A.nrows, world, rank)
    # row panel of A as a view on its own arrays (rowptr slice + rowend)
    dP = sg.DeviceCSR(r1 - r0, A.ncols, dA.rowptr[r0:r1], dA.col, dA.val,
                      rowend=dA.rowptr[r0 + 1:r1 + 1]) if world > 1 else dA
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        p = sg.plan(dP, dA)
        rowptrC, nnz = sg.symbolic(p)
        colC, valC = sg.alloc_output(p, nnz)
        if ev is not None:
            ev[0].record(stream)
        sg.numeric(p, rowptrC, colC, valC)
        if ev is not None:
            ev[1].record(stream)
        return p, rowptrC, colC, valC, nnz

    for _ in range(args.warmup):
        out = step()
        del out
    torch.cuda.synchronize()
    info = None
    step_ms, num_ms = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = sg.kernel_launches()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        e0.record(stream)
        p, rowptrC, colC, valC, nnz = step(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        num_ms.append(ev[0].elapsed_time(ev[1]))
        info = p.info()
        del p, rowptrC, colC, valC
    torch.cuda.synchronize()
    launches = sg.kernel_launches() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    total_ms = float(np.sum(step_ms))
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    fl = torch.tensor([float(info["flops"])], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(fl, op=dist.ReduceOp.SUM)
    total_ms = float(t.item())
    flops_all = float(fl.item())
    ms_per_step = total_ms / args.steps
    value = 2.0 * flops_all / (ms_per_step * 1e-3) / 1e9

    # roofline of the numeric phase (numeric_dense_kernel is ~99% of it)
    nnz_c = int(info["nnz_c"])
    _, num_bytes = algorithmic_bytes(A, nnz_c)
    num_avg = float(np.mean(num_ms))
    hbm, peak_src = peaks()
    achieved = num_bytes / (num_avg * 1e-3) / 1e9
    traffic = profiled_traffic()
    # the FP64 pipe: every product is one multiply and one add; GB300 issues
    # 2 FP64 lanes per clock per SM (ncu peak_sustained of the FP64 pipe)
    fp64_peak = FP64_LANES_PER_SM_CLK * SMS * SM_MAX_MHZ * 1e6 / 1e9
    fp64_achieved = 2.0 * flops_all / (num_avg * 1e-3) / 1e9 / world

    # the end-to-end leg runs first, before the other legs fill the allocator's
    # cache, and from an empty cache: the timed steps leave tens of GB of
    # output blocks cached, which a user's call would not find
    torch.cuda.empty_cache()
    e2e = (run_e2e(args, A, sg, torch, dev, dP if world == 1 else None)
           if rank == 0 and not args.no_e2e else None)
    torch.cuda.empty_cache()
    paths = run_paths(args, A, dA, sg, torch) if (rank == 0 and world == 1 and not args.no_paths) else None
    if paths is not None:
        paths["er16384_f64"] = run_config_er16384(sg, torch)
    if paths is not None and not args.no_learned:
        paths["learned"] = run_learned(args, sg, torch)
    cpu = run_cpu_baseline(A) if (rank == 0 and world == 1 and not args.no_cpu) else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded R-MAT generator; no dataset)",
            "config": {"workload": "rmat18_g500_squared", "scale": SCALE, "edge_factor": 16,
                       "n": A.nrows, "nnz_A": A.nnz, "flops": int(flops_all // 1),
                       "nnz_C": nnz_c, "index": "int32", "values": "f64",
                       "path": "plain two-phase", "l2": "flushed between steps",
                       "parallelism": f"row panels x{world}"},
            "phases_ms": {"numeric": round(num_avg, 3), "step": round(ms_per_step, 3)},
            "roofline": {"bound": "hbm", "kernel": "numeric phase (numeric_dense_kernel)",
                         "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "peak_source": peak_src,
                         "algorithmic_bytes": num_bytes, "traffic": traffic},
            "fp64_roofline": {"bound": "alu", "kernel": "numeric phase (numeric_dense_kernel)",
                              "achieved": round(fp64_achieved, 1), "peak": round(fp64_peak, 1),
                              "unit": "G FP64 lane-ops/s (one mul + one add per product)",
                              "frac": round(fp64_achieved / fp64_peak, 4),
                              "peak_source": "2 FP64 lanes/clk/SM x 152 SMs x 2070 MHz"},
            "paths": paths,
            "gpu_launches": int(launches),
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed(torch, fn, reps):
    """Wall time of fn() with a device synchronize on both sides (best of reps)."""
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        del out
        best = dt if best is None else min(best, dt)
    return best


def merge_roofline(sg, torch, dA, c=4, reps=3):
    """The multiway merge alone on the 4 k-slice partials of the product
    (count + scan + numeric, then the numeric pass by itself), register
    windows against lists staged in shared memory by bulk asynchronous
    copies.  Algorithmic bytes of the numeric pass: every partial entry read
    once and every entry of C written once (index + value each), plus the c
    partial row-pointer arrays and rowptr(C)."""
    _, parts = sg.spgemm_kslice(dA, dA, c)
    torch.cuda.synchronize()
    m = dA.nrows
    ws = sg.merge_workspace(len(parts), m, dA.ncols, dA.rowptr.device)
    rowptrC, nnz = sg.merge_symbolic(parts, ws)
    colC = torch.empty(nnz, dtype=parts[0].col.dtype, device="cuda")
    valC = torch.empty(nnz, dtype=parts[0].val.dtype, device="cuda")
    ent = parts[0].col.element_size() + parts[0].val.element_size()
    nparts = sum(int(p.nnz) for p in parts)
    nbytes = ent * (nparts + int(nnz)) + 8 * (m + 1) * (len(parts) + 1)
    stream = torch.cuda.current_stream()
    hbm, _ = peaks()
    res = {"partial_entries": nparts, "nnz_C": int(nnz), "algorithmic_bytes": int(nbytes)}
    for name, staged in (("windows", False), ("staged", True)):
        sg.merge_numeric(parts, ws, rowptrC, colC, valC, staged=staged)
        sg.merge_check(ws)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sg.merge_numeric(parts, ws, rowptrC, colC, valC, staged=staged)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        avg = float(np.mean(ms))
        res[name] = {"numeric_ms": round(avg, 3),
                     "gbs": round(nbytes / (avg * 1e-3) / 1e9, 1),
                     "frac_of_measured_hbm": round(nbytes / (avg * 1e-3) / 1e9 / hbm, 4)}
    del parts, colC, valC, ws
    return res


def _stage_report(stages):
    """Stage times of a persistent chain's last launch (block 0's
    %globaltimer at every barrier): totals per stage kind over the products,
    and per product."""
    by_stage, by_step = {}, {}
    for q, name, ms in stages:
        by_stage[name] = round(by_stage.get(name, 0.0) + ms, 4)
        if q >= 0:
            by_step[str(q)] = round(by_step.get(str(q), 0.0) + ms, 4)
    return {"by_stage": by_stage, "by_product": by_step}


def run_paths(args, A, dA, sg, torch):
    """The other rows of the path, each against its plain counterpart:
    k=4 split + merge on the same product, 512 uneven ER products batched vs
    one by one, and the AMG Galerkin hierarchy in one CUDA graph vs the
    host-synced chain."""
    from paper_1510_00844_gb300 import amg, autotune, inputs
    out = {}
    reps = 2
    flops = sg.plan(dA, dA).info()["flops"]
    _timed(torch, lambda: sg.spgemm_kslice(dA, dA, 4), 1)
    t = _timed(torch, lambda: sg.spgemm_kslice(dA, dA, 4), reps)
    _timed(torch, lambda: sg.spgemm_kslice(dA, dA, 4, hypersparse=True), 1)
    th = _timed(torch, lambda: sg.spgemm_kslice(dA, dA, 4, hypersparse=True), reps)
    out["kslice4_merge_rmat18"] = {"ms": round(t * 1e3, 3),
                                   "gflops": round(2 * flops / t / 1e9, 3),
                                   "hypersparse_slices_ms": round(th * 1e3, 3),
                                   "merge": merge_roofline(sg, torch, dA),
                                   "note": "4 k-slice partial products + multiway merge; "
                                           "hypersparse: slices as DCSR views"}
    pairs = inputs.batched_er(512)
    As = [sg.to_device(a) for a, _ in pairs]
    Bs = [sg.to_device(b) for _, b in pairs]
    bflops = sg.batch_plan(As, Bs).info()["flops"]
    _timed(torch, lambda: sg.batch_spgemm(As, Bs), 1)
    tb = _timed(torch, lambda: sg.batch_spgemm(As, Bs), reps)
    ts = _timed(torch, lambda: [sg.spgemm(a, b) for a, b in zip(As, Bs)], reps)
    best, table = autotune.batch(As, Bs, repeats=2)
    # the same batch as one device-sized plan captured in a CUDA graph (no
    # host readback; output capacity = the flops bound)
    gs = torch.cuda.Stream()
    dp = sg.device_plan(As, Bs, stream=gs, max_row_nnz=4096)
    rowptrC = torch.empty(dp.R + 1, dtype=torch.int64, device="cuda")
    colC = torch.empty(int(bflops), dtype=As[0].col.dtype, device="cuda")
    valC = torch.empty(int(bflops), dtype=As[0].val.dtype, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        sg.execute(dp, rowptrC, int(bflops), colC, valC)
    graph.replay()
    torch.cuda.synchronize()
    sg.check(dp)
    tgb = _timed(torch, graph.replay, reps)
    ref = sg.batch_spgemm(As, Bs)
    nnz = int(rowptrC[-1].item())
    same = (nnz == sum(C.nnz for C in ref)
            and bool((colC[:nnz] == torch.cat([C.col for C in ref])).all())
            and bool((valC[:nnz] == torch.cat([C.val for C in ref])).all()))
    # the same device-sized plan as one persistent chain launch
    colC.fill_(-1)
    chain = sg.Chain([(dp, rowptrC, int(bflops), colC, valC)], record_stages=True)
    with torch.cuda.stream(gs):
        chain.launch(gs)
    chain.check(gs)
    tpc = _timed(torch, lambda: chain.launch(gs), reps)
    chain.check(gs)
    batch_stages = _stage_report(chain.stage_ms())
    same_chain = (int(rowptrC[-1].item()) == nnz
                  and bool((colC[:nnz] == torch.cat([C.col for C in ref])).all())
                  and bool((valC[:nnz] == torch.cat([C.val for C in ref])).all()))
    f32_error = batch_f32_error(sg, torch, pairs, ref)
    del ref, graph, dp, rowptrC, colC, valC, chain
    out["batched_er512_f32"] = {"batched_ms": round(tb * 1e3, 3), "sequential_ms": round(ts * 1e3, 3),
                                "speedup": round(ts / tb, 3), "flops": int(bflops),
                                "gflops_batched": round(2 * bflops / tb / 1e9, 3),
                                "graph_ms": round(tgb * 1e3, 3),
                                "graph_speedup_vs_sequential": round(ts / tgb, 3),
                                "graph_bit_identical": bool(same),
                                "persistent_ms": round(tpc * 1e3, 3),
                                "persistent_launches": 1,
                                "persistent_bit_identical": bool(same_chain),
                                "persistent_speedup_vs_sequential": round(ts / tpc, 3),
                                "persistent_stage_ms": batch_stages,
                                "f32_error": f32_error,
                                "autotune": _tuning_report(best, table)}
    del As, Bs, pairs
    N = 128
    A0 = inputs.laplacian_7pt(N)
    Rs = [inputs.aggregation_2x2x2(N >> l) for l in range(3)]
    dA0 = sg.to_device(A0)
    dRs = [sg.to_device(R) for R in Rs]
    s = torch.cuda.Stream()
    chain = amg.GalerkinChain(dA0, dRs, s)
    chain.capture()
    tg = _timed(torch, chain.replay, 5)
    chain.check()
    # the six products of the hierarchy in one persistent launch (the
    # transposes R_l^T depend only on the given R_l and are formed once)
    pchain = amg.GalerkinChain(dA0, dRs, s, persistent=True, record_stages=True)
    pchain.capture()
    pchain.replay()
    torch.cuda.synchronize()
    pchain.check()
    tpg = _timed(torch, pchain.replay, 5)
    pchain.check()
    amg_stages = _stage_report(pchain.chain.stage_ms())
    same_p = all(bool(torch.equal(C.col, D.col)) and bool(torch.equal(C.val, D.val))
                 for C, D in zip(pchain.results(), chain.results()))
    tr_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(tr_graph, stream=s):
        for lv in chain.levels:
            chain._transpose(lv)
    ttr = _timed(torch, tr_graph.replay, 5)
    del pchain, tr_graph

    def plain_chain():
        A_ = dA0
        for R in dRs:
            A_ = sg.spgemm(sg.spgemm(sg.transpose(R), A_), R)
        return A_
    plain_chain()
    tp = _timed(torch, plain_chain, 5)
    gflops = 0
    A_ = dA0
    for R in dRs:
        Rt = sg.transpose(R)
        gflops += sg.plan(Rt, A_).info()["flops"]
        T = sg.spgemm(Rt, A_)
        gflops += sg.plan(T, R).info()["flops"]
        A_ = sg.spgemm(T, R)
    out["amg_mis2_128cubed_3levels"] = run_mis2_hierarchy(sg, torch, dA0, 3)
    best, table = autotune.galerkin(dA0, dRs, s, repeats=5)
    out["amg_galerkin_128cubed_3levels"] = {"graph_ms": round(tg * 1e3, 3), "plain_ms": round(tp * 1e3, 3),
                                            "speedup": round(tp / tg, 3), "flops": int(gflops),
                                            "gflops_graph": round(2 * gflops / tg / 1e9, 3),
                                            "persistent_ms": round(tpg * 1e3, 3),
                                            "persistent_launches": 1,
                                            "persistent_bit_identical": bool(same_p),
                                            "persistent_stage_ms": amg_stages,
                                            "transposes_ms": round(ttr * 1e3, 3),
                                            "note": "graph_ms: transposes and both products of "
                                                    "every level as one captured graph of "
                                                    "library launches; persistent_ms: the six "
                                                    "products in one persistent launch (a graph "
                                                    "of a memset and the kernel), transposes "
                                                    "(transposes_ms) formed once beforehand",
                                            "autotune": _tuning_report(best, table)}
    return out


def run_mis2_hierarchy(sg, torch, dA0, levels, seed=20151004):
    """The paper's own coarsening (Sec. 5.4): at every level, MIS-2
    aggregation of the current matrix builds R on the GPU (Alg. 3), then
    A_{l+1} = R^T A_l R.  Times the aggregation and the products apart."""
    def build():
        A = dA0
        t_mis = t_gal = 0.0
        sizes, rounds = [], []
        for _ in range(levels):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            R, r = sg.mis2_restriction(A, seed)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            A = sg.spgemm(sg.spgemm(sg.transpose(R), A), R)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            t_mis += t1 - t0
            t_gal += t2 - t1
            sizes.append(int(R.ncols))
            rounds.append(r)
        return t_mis, t_gal, sizes, rounds
    build()
    t_mis, t_gal, sizes, rounds = build()
    return {"mis2_ms": round(t_mis * 1e3, 3), "galerkin_ms": round(t_gal * 1e3, 3),
            "coarse_sizes": sizes, "mis2_rounds": rounds,
            "note": "R from MIS-2 aggregation on the GPU at every level (not graph-captured)"}


def _tuning_report(best, table):
    """Chosen knobs, their time and the library default's (milliseconds)."""
    from paper_1510_00844_gb300.spgemm import Tuning
    return {"best": {k: v for k, v in vars(best).items() if v}, "best_ms": round(table[best], 3),
            "default_ms": round(table[Tuning()], 3), "candidates": len(table)}


def _checksum(torch, C):
    """Order-sensitive int64 digest of a CSR (rows, columns, value bits)."""
    rp = C.rowptr[: C.nrows + 1]
    cnt = (rp[1:] - rp[:-1]).to(torch.int64)
    h = int((cnt * torch.arange(1, C.nrows + 1, device=cnt.device)).sum().item())
    pos = torch.arange(C.col.numel(), device=cnt.device, dtype=torch.int64)
    h ^= int(((C.col.to(torch.int64) + 7) * (pos % 1000003 + 1)).sum().item())
    if C.val is not None:
        bits = C.val.view(torch.int64) if C.val.dtype == torch.float64 else C.val.to(torch.int64)
        h ^= int((bits * (pos % 999983 + 3)).sum().item())
    return h


def train_sizer(sg, torch, inputs):
    """Predictor trained on the GPU on exact symbolic outputs of R-MAT scales
    14-18 and ER matrices (the training recipe of the learned-sizing row)."""
    pairs = [inputs.rmat(s, seed=500 + s) for s in (14, 15, 16, 17, 18)]
    pairs += [inputs.er_column_regular(1 << 15, d, 600 + d) for d in (8, 16)]
    dev = [(sg.to_device(A), sg.to_device(A)) for A in pairs]
    X, T = sg.sizer_training_set(dev)
    params = sg.sizer_init(seed=7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trace = sg.sizer_train(X, T, params, steps=1500, batch=4096, lr=3e-3, seed=8)
    torch.cuda.synchronize()
    tt = time.perf_counter() - t0
    y = sg.sizer_forward(X, params)
    rmse = float(((y - T) ** 2).mean().sqrt())
    return params, {"samples": int(X.shape[0]), "steps": 1500, "train_s": round(tt, 3),
                    "final_loss": round(float(trace[-50:].mean()), 5), "rmse_log2": round(rmse, 4)}


def run_learned(args, sg, torch):
    """Learned sizing vs the exact two-phase path: R-MAT scale 20 squaring in
    row panels (C does not fit HBM; each panel is reduced to a checksum), and
    five MCL steps on a column-stochastic R-MAT scale 20 matrix."""
    from paper_1510_00844_gb300 import inputs
    params, train = train_sizer(sg, torch, inputs)
    out = {"sizer": train}
    margin = 0.35
    A = inputs.rmat(20)
    dA = sg.to_device(A)
    npan = 16
    bounds = [((A.nrows * p) // npan, (A.nrows * (p + 1)) // npan) for p in range(npan)]
    views = [sg.DeviceCSR(b - a, A.ncols, dA.rowptr[a:b], dA.col, dA.val, rowend=dA.rowptr[a + 1:b + 1])
             for a, b in bounds]
    fl = sum(sg.plan(v, dA).info()["flops"] for v in views)
    times = {"plain": 0.0, "learned": 0.0}
    same = True
    overflow = 0
    for v in views:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C = sg.spgemm(v, dA)
        torch.cuda.synchronize()
        times["plain"] += time.perf_counter() - t0
        h1 = _checksum(torch, C)
        del C
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        L, st = sg.learned_multiply(v, dA, params, margin)
        torch.cuda.synchronize()
        times["learned"] += time.perf_counter() - t0
        overflow += st["overflow_rows"]
        Lc = sg.compact(L)
        same = same and _checksum(torch, Lc) == h1
        del L, Lc
        torch.cuda.empty_cache()
    out["rmat20_squared_panels16"] = {
        "plain_ms": round(times["plain"] * 1e3, 1), "learned_ms": round(times["learned"] * 1e3, 1),
        "speedup": round(times["plain"] / times["learned"], 3), "flops": int(fl),
        "gflops_plain": round(2 * fl / times["plain"] / 1e9, 2),
        "gflops_learned": round(2 * fl / times["learned"] / 1e9, 2),
        "overflow_rows": int(overflow), "bit_identical": bool(same)}
    del views, dA, A
    torch.cuda.empty_cache()
    print("learned rmat20:", json.dumps(out), flush=True, file=sys.stderr)
    if args.no_mcl:
        return out
    out["mcl5_rmat20"] = run_mcl(args, sg, torch, params, margin)
    return out


def run_mcl(args, sg, torch, params, margin):
    """Five MCL expansions (M^T M^T, prune < 1e-4, renormalise) on a
    column-stochastic R-MAT scale 20 matrix with learned sizing, per step
    flops, panels, nnz before and after pruning, product and prune times;
    the exact two-phase path runs on every `--mcl-compare`-th panel of every
    step (and on all panels with --mcl), on the same input, with the pruned
    panels compared bit for bit."""
    from paper_1510_00844_gb300 import inputs
    M = inputs.mcl_transition(20)
    X = sg.to_device(M)
    every = 1 if args.mcl else max(1, args.mcl_compare)
    steps = []
    total_ms = 0.0
    same = True
    lt = pt = 0.0
    for _ in range(5):
        st = {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X = sg.mcl_step(X, 1e-4, params=params, margin=margin, stats=st, compare_every=every)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        total_ms += ms
        same = same and st["compared_identical"]
        lt += st["compared_learned_ms"]
        pt += st["compared_plain_ms"]
        steps.append({"flops": st["flops"], "panels": st["panels"],
                      "nnz_before_prune": st["nnz_product"], "nnz_after_prune": st["nnz_pruned"],
                      "product_ms": round(st["product_ms"], 1), "prune_ms": round(st["prune_ms"], 1),
                      "gflops": round(2 * st["flops"] / (st["product_ms"] * 1e-3) / 1e9, 2),
                      "compared_panels": st["compared_panels"]})
        torch.cuda.empty_cache()
    return {"steps": steps, "learned_step_total_ms": round(total_ms, 1), "nnz_final": int(X.nnz),
            "compared_every": every, "compared_learned_ms": round(lt, 1),
            "compared_plain_ms": round(pt, 1), "speedup_on_compared": round(pt / lt, 3) if lt else None,
            "bit_identical": bool(same),
            "note": "learned sizing on every panel; the exact two-phase product and prune on the "
                    "compared panels of each step, same input; wall time of a step includes the "
                    "compared panels' plain products"}


def _anon_huge_bytes():
    """Bytes of this process's anonymous memory held in transparent huge
    pages (the pinned host buffers of the end-to-end leg ask for them)."""
    try:
        for ln in open("/proc/self/smaps_rollup"):
            if ln.startswith("AnonHugePages:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def run_e2e(args, A, sg, torch, dev, dP):
    """Same metric through the public API from pinned host buffers: H2D of
    A, then C = A.A delivered to pinned host memory by row panels whose
    device-to-host copies overlap the next panel's numeric phase
    (pipeline.spgemm_to_host)."""
    from paper_1510_00844_gb300 import pipeline
    if dP is None:
        return None
    hr = pipeline.pinned_empty(A.rowptr.size, torch.int64)
    hc = pipeline.pinned_empty(A.col.size, torch.int32 if A.col.dtype == np.int32 else torch.int64)
    hv = pipeline.pinned_empty(A.val.size, torch.float64)
    hr.copy_(torch.from_numpy(A.rowptr))
    hc.copy_(torch.from_numpy(A.col))
    hv.copy_(torch.from_numpy(A.val))
    dr = torch.empty_like(hr, device=dev)
    dc = torch.empty_like(hc, device=dev)
    dv = torch.empty_like(hv, device=dev)
    out_host = None
    times = []
    h2d = hr.numel() * 8 + hc.numel() * hc.element_size() + hv.numel() * 8
    d2h = 0
    nsteps = max(1, min(args.steps, 2))
    warm = 2     # the first copies into freshly registered pages run slow
    splits = []
    for it in range(warm + nsteps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        dr.copy_(hr, non_blocking=True)
        dc.copy_(hc, non_blocking=True)
        dv.copy_(hv, non_blocking=True)
        e1.record()
        M = sg.DeviceCSR(A.nrows, A.ncols, dr, dc, dv)
        tm = {}
        out_host = pipeline.spgemm_to_host(M, M, panels=8, out=out_host, timing=tm)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tm["h2d_ms"] = e0.elapsed_time(e1)
        tm["wall_ms"] = (t1 - t0) * 1e3
        nnz = out_host.nnz
        d2h = (A.nrows + 1) * 8 + nnz * (out_host.col.element_size() + 8)
        if it >= warm:
            times.append(t1 - t0)
            splits.append(tm)
        del M
    fl = sg.plan(sg.DeviceCSR(A.nrows, A.ncols, dr, dc, dv),
                 sg.DeviceCSR(A.nrows, A.ncols, dr, dc, dv)).info()["flops"]
    # the link by itself at this moment: one 2 GiB device-to-host copy into
    # the same host buffer, outside the timed steps
    probe = torch.empty(1 << 28, dtype=torch.float64, device=dev)
    probe.fill_(1.0)
    ms_link = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out_host.val[:probe.numel()].copy_(probe, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        ms_link.append(a.elapsed_time(b))
    del probe
    sec = float(np.mean(times))
    last = splits[-1]
    split = {k: round(float(np.mean([t[k] for t in splits])), 3)
             for k in ("h2d_ms", "plans_symbolic_ms", "numeric_ms", "copy_ms", "copy_tail_ms",
                       "first_numeric_to_last_copy_ms", "wall_ms")}
    split["h2d_gbs"] = round(h2d / (split["h2d_ms"] * 1e-3) / 1e9, 1)
    split["d2h_gbs"] = round(last["d2h_bytes"] / (split["copy_ms"] * 1e-3) / 1e9, 1)
    split["link_d2h_gbs"] = round((1 << 31) / (min(ms_link) * 1e-3) / 1e9, 1)
    split["host_huge_page_bytes"] = _anon_huge_bytes()
    split["host_buffer_bytes"] = int(h2d + d2h)
    split["per_step_wall_ms"] = [round(t["wall_ms"], 1) for t in splits]
    split["per_step_plans_symbolic_ms"] = [round(t["plans_symbolic_ms"], 1) for t in splits]
    split["per_step_copy_ms"] = [round(t["copy_ms"], 1) for t in splits]
    return {"value": round(2.0 * fl / sec / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(sec * 1e3, 3), "steps": nsteps, "split": split,
            "note": "8 row panels, copies overlapped with the next panel's numeric phase; "
                    "split: CUDA-event times of the H2D copy, plans + symbolic phases, "
                    "numeric phases, device-to-host copies and the copy tail after the "
                    "last numeric phase"}


def oracle_sample(A, target_flops):
    """Rows of A chosen by a seeded permutation until their flops reach
    target_flops (a bounded sample with the workload's row mix)."""
    import oracle
    fl = oracle.row_flops(A, A)
    order = np.random.default_rng(11).permutation(A.nrows)
    cum = np.cumsum(fl[order])
    k = int(np.searchsorted(cum, target_flops)) + 1
    rows = np.sort(order[:k])
    lens = A.rowptr[rows + 1] - A.rowptr[rows]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows])
    sub = oracle.OCSR(len(rows), A.ncols, rp, A.col[idx].astype(np.int64), A.val[idx])
    return sub, int(fl[rows].sum()), len(rows)


def run_cpu_baseline(A, target_flops=3e9, reps=1, one_thread_flops=3e8):
    import oracle
    sub, sflops, nrows = oracle_sample(A, target_flops)
    threads = len(os.sched_getaffinity(0))
    oracle.spgemm(oracle.OCSR(1, A.ncols, sub.rowptr[:2], sub.col, sub.val), A,
                  nthreads=threads)   # warm the library
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.spgemm(sub, A, nthreads=threads)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    sub1, sflops1, nrows1 = oracle_sample(A, one_thread_flops)
    t0 = time.perf_counter()
    oracle.spgemm(sub1, A, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": round(2.0 * sflops / best / 1e9, 4), "unit": UNIT,
            "cores": oracle.num_threads(threads), "kind": "oracle",
            "sample": f"{nrows} seeded random rows of A (flops {sflops}) times A; "
                      f"{best:.2f} s wall",
            "one_thread": {"value": round(2.0 * sflops1 / dt1 / 1e9, 4), "unit": UNIT,
                           "sample": f"{nrows1} seeded random rows (flops {sflops1}); "
                                     f"{dt1:.2f} s wall"}}


def run_config_er16384(sg, torch):
    """The small configuration: C = A.A, A Erdos-Renyi n = 16384 with exactly
    8 nonzeros per column, float64.  GPU: the plain two-phase path (plan,
    symbolic, numeric), CUDA events, best of 10 after 3 warm-ups.  Oracle:
    the whole product on all host cores and on one core (best of 3), with
    the GPU result compared to it entry by entry."""
    import oracle
    from paper_1510_00844_gb300 import inputs
    A = inputs.er_column_regular(16384, 8, inputs.BASE_SEED + 1)
    dA = sg.to_device(A)
    s = torch.cuda.current_stream()
    best = None
    for it in range(13):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        C = sg.spgemm(dA, dA)
        e1.record(s)
        torch.cuda.synchronize()
        if it >= 3:
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    flops = int(sg.plan(dA, dA).info()["flops"])
    threads = len(os.sched_getaffinity(0))
    times = {}
    for nt in (threads, 1):
        bt = None
        for _ in range(3):
            t0 = time.perf_counter()
            R = oracle.spgemm(A, A, nthreads=nt)
            dt = time.perf_counter() - t0
            bt = dt if bt is None else min(bt, dt)
        times[nt] = bt
    rp, col, val = C.to_host()
    same = (np.array_equal(rp, R.rowptr) and np.array_equal(col.astype(np.int64), R.col)
            and bool(np.all(np.abs(val - R.val) <= 1e-12 * np.abs(R.val))))
    return {"flops": flops, "nnz_C": int(C.nnz), "gpu_ms": round(best, 4),
            "gpu_gflops": round(2 * flops / (best * 1e-3) / 1e9, 3),
            "oracle_s": round(times[threads], 4), "oracle_cores": oracle.num_threads(threads),
            "oracle_1thread_s": round(times[1], 4), "matches_oracle": bool(same),
            "note": "plan + symbolic + numeric on the GPU; the whole product on the host"}


def batch_f32_error(sg, torch, pairs, Cs, sample=24):
    """Error of float32 accumulation against the float64 oracle on a seeded
    sample of the batched products: per entry |c32 - c64| / sum_k |a||b|,
    its maximum, and its maximum relative to gamma_q = q u / (1 - q u)
    (u = 2^-24, q = the entry's number of terms), the recursive-summation
    bound the tests assert."""
    import oracle
    from paper_1510_00844_gb300 import inputs
    rng = np.random.default_rng(17)
    pick = rng.choice(len(pairs), min(sample, len(pairs)), replace=False)
    u = 2.0 ** -24
    worst, worst_ratio, entries = 0.0, 0.0, 0
    for q in pick:
        a, b = pairs[q]
        a64 = inputs.CSR(a.nrows, a.ncols, a.rowptr, a.col, a.val.astype(np.float64))
        b64 = inputs.CSR(b.nrows, b.ncols, b.rowptr, b.col, b.val.astype(np.float64))
        R = oracle.spgemm(a64, b64)
        S = oracle.spgemm(a64.with_values(np.abs(a64.val)), b64.with_values(np.abs(b64.val)))
        Q = oracle.spgemm(a64.with_values(np.ones(a.nnz)), b64.with_values(np.ones(b.nnz)))
        c32 = Cs[q].val.cpu().numpy().astype(np.float64)
        err = np.abs(c32 - R.val) / np.where(S.val > 0, S.val, 1.0)
        gq = Q.val * u / (1 - Q.val * u)
        worst = max(worst, float(err.max(initial=0.0)))
        worst_ratio = max(worst_ratio, float((err / gq).max(initial=0.0)))
        entries += int(R.nnz)
    return {"products_sampled": int(len(pick)), "entries": entries,
            "max_err_over_sum_abs": worst, "max_err_over_gamma_q": round(worst_ratio, 4),
            "u": u}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1510_00844_gb300 import inputs
    import oracle
    A = inputs.rmat(SCALE)
    threads = len(os.sched_getaffinity(0))
    sub, sflops, nrows = oracle_sample(A, 1e9)
    for _ in range(args.warmup):
        oracle.spgemm(sub, A, nthreads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.spgemm(sub, A, nthreads=threads)
        times.append(time.perf_counter() - t0)
    ms = float(np.mean(times)) * 1e3
    value = 2.0 * sflops / (ms * 1e-3) / 1e9
    cores = oracle.num_threads(threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded R-MAT generator; no dataset)",
        "config": {"workload": "rmat18_g500_squared", "scale": SCALE, "edge_factor": 16,
                   "index": "int32", "values": "f64", "path": "CPU oracle (dense-accumulator Gustavson)"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{nrows} seeded random rows of A (flops {sflops}) times A per step"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_leg(args):
    """One workload run `--reps` times with no timing and no JSON line: the
    command the ncu summaries under profiles/ profile (the first run warms
    up, so a capture skips its launches)."""
    import torch
    from paper_1510_00844_gb300 import amg, inputs, spgemm as sg
    leg, reps = args.profile_leg, max(1, args.reps)
    if leg in ("product", "kslice"):
        dA = sg.to_device(inputs.rmat(args.scale))
        for _ in range(reps):
            if leg == "product":
                nnz = sg.spgemm(dA, dA).nnz
            else:
                nnz = sg.spgemm_kslice(dA, dA, 4)[0].nnz
            torch.cuda.synchronize()
        print(f"{leg} R-MAT {args.scale}: nnz(C) {nnz}", flush=True)
    elif leg == "batched":
        pairs = inputs.batched_er(512)[: max(1, min(512, args.products))]
        As = [sg.to_device(a) for a, _ in pairs]
        Bs = [sg.to_device(b) for _, b in pairs]
        for _ in range(reps):
            nnz = sum(C.nnz for C in sg.batch_spgemm(As, Bs))
            torch.cuda.synchronize()
        print(f"batched {len(pairs)} ER products: nnz {nnz}", flush=True)
    elif leg == "batched-chain":
        pairs = inputs.batched_er(512)[: max(1, min(512, args.products))]
        As = [sg.to_device(a) for a, _ in pairs]
        Bs = [sg.to_device(b) for _, b in pairs]
        cap = int(sg.batch_plan(As, Bs).info()["flops"])
        dp = sg.device_plan(As, Bs, max_row_nnz=4096)
        rp = torch.empty(dp.R + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(cap, dtype=As[0].col.dtype, device="cuda")
        val = torch.empty(cap, dtype=As[0].val.dtype, device="cuda")
        ch = sg.Chain([(dp, rp, cap, col, val)])
        for _ in range(reps):
            ch.launch()
            ch.check()
        print(f"batched chain {len(pairs)} ER products: nnz {int(rp[-1].item())}", flush=True)
    elif leg == "learned":
        # one 1/16 row panel of the R-MAT 20 squaring, exact two-phase then
        # learned sizing (the panels of the learned-sizing leg)
        params, _ = train_sizer(sg, torch, inputs)
        A = inputs.rmat(20)
        dA = sg.to_device(A)
        a, b = 0, A.nrows // 16
        v = sg.DeviceCSR(b - a, A.ncols, dA.rowptr[a:b], dA.col, dA.val,
                         rowend=dA.rowptr[a + 1:b + 1])
        for _ in range(reps):
            C = sg.spgemm(v, dA)
            torch.cuda.synchronize()
            nnz = C.nnz
            del C
            L, st = sg.learned_multiply(v, dA, params, 0.35)
            torch.cuda.synchronize()
            del L
        print(f"learned panel of R-MAT 20: nnz {nnz}, overflow rows {st['overflow_rows']}", flush=True)
    elif leg in ("amg", "amg-chain", "mis2"):
        N = 128
        dA0 = sg.to_device(inputs.laplacian_7pt(N))
        if leg in ("amg", "amg-chain"):
            dRs = [sg.to_device(inputs.aggregation_2x2x2(N >> l)) for l in range(3)]
            chain = amg.GalerkinChain(dA0, dRs, torch.cuda.Stream(), persistent=leg == "amg-chain")
            chain.capture()
            for _ in range(reps):
                chain.replay()
                torch.cuda.synchronize()
            chain.check()
            print("amg: 3-level Galerkin hierarchy of the 128^3 Laplacian, graph replays", reps,
                  flush=True)
        else:
            for _ in range(reps):
                R, rounds = sg.mis2_restriction(dA0, 20151004)
                torch.cuda.synchronize()
            print(f"mis2: {R.ncols} aggregates in {rounds} rounds", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-sizing comparison (R-MAT 20 squaring)")
    ap.add_argument("--mcl", action="store_true",
                    help="compare the MCL steps against the exact path on every panel (slow)")
    ap.add_argument("--no-mcl", action="store_true", help="skip the five MCL steps")
    ap.add_argument("--mcl-compare", type=int, default=16,
                    help="compare every k-th MCL panel against the exact two-phase path")
    ap.add_argument("--no-paths", action="store_true",
                    help="skip the split / batched / AMG comparisons")
    ap.add_argument("--profile-leg", choices=["product", "kslice", "batched", "batched-chain",
                                              "amg", "amg-chain", "mis2", "learned"],
                    help="run one workload --reps times without timing (for ncu captures)")
    ap.add_argument("--scale", type=int, default=18, help="R-MAT scale of --profile-leg")
    ap.add_argument("--reps", type=int, default=2, help="runs of --profile-leg")
    ap.add_argument("--products", type=int, default=512,
                    help="first N of the 512 batched products for --profile-leg batched")
    args = ap.parse_args()
    if args.profile_leg:
        run_profile_leg(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
