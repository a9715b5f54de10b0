"""Benchmark of the REFINE importance / prune / compact pass on GB300.

One step = refine_score + refine_select + refine_compact (every hot-path
step) over one resident synthetic scene.  The default workload is the
3.5M-primitive core-shell scene with 250 views at 1600x1063, plain FP32,
prune ratio 0.5.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c2|c1|c0]

Under torchrun each rank scores its own replica scene (weak scaling, no
data-path collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic FP32 work of the score kernel, counted only for the stages a
# (primitive, view) pair needed (the kernel's diagnostic counters say which),
# an FMA as 2 FLOPs and a compare, max or MUFU reciprocal as 1:
FLOP_COSTS = {
    "tile_view": 118,     # interval classification of one view for one tile: z, U, V, U - w z,
                          # V - h z over the tile box (22 each) and the six range tests
    "in_pair": 10,        # tile entirely visible: depth z (3 FMA), z^2 + eta (FMA), reciprocal, add
    "mixed_pair": 6,      # decided pair by pair: depth z (3 FMA)
    "open_axis": 10,      # per open u or v axis: U (3 FMA), d = max(-U, U - w z) (FMA, max), compare
    "open_depth": 2,      # open depth range: two compares
    "visible_mixed": 4,   # visible pair decided one by one: z^2 + eta, reciprocal, add
    "bound_pair": 1,      # z^2 of a centre outside the image
    "bound_axis": 10,     # per open axis: e = max(d, 0) z, e^2, t = U - c z, t^2, f^2 z^2 + t^2,
                          # times 9 s_max^2, compare
    "exact_axis": 30,     # per needed extent: g = z P - U P2 (3 MUL, 3 FMA), L g (3 MUL, 6 FMA),
                          # |L g|^2 (MUL, 2 FMA), compare
    "kahan_block": 4,     # per primitive and 32-view block: compensated add of the block sum
    "epilogue": 8,        # per primitive: Eq. 7 coupling and the Eq. 20 scaling
}
FP32_LANES_PER_SM = 128
METRIC = "Gaussian×view pairs/s"


def workload(name: str, rank: int = 0, storage: str = "f32"):
    from paper_2606_09074_gb300 import synth
    if name == "c2":
        w = synth.config2(seed=replica_seed(2, rank), dtype=storage)
        w.name = f"core-shell N=3.5M V=250 1600x1063, {storage.upper()} storage, ratio 0.5"
    elif name == "c1":
        w = synth.config1(seed=replica_seed(1, rank))
        w.ratios = (0.5,)
        w.name = "core-shell N=1M V=150 1297x840, FP32, ratio 0.5"
    elif name == "c0":
        w = synth.config0(seed=replica_seed(0, rank))
        w.name = "normal N=10k V=16 640x480, FP32, ratio 0.5"
    else:
        raise ValueError(name)
    return w


def cell_bits_for(n: int) -> int:
    """Resolution of the processing-order grid the library picks for n
    primitives (2^(3b) Morton cells, b in 4..7, about 0.5 or more per cell)."""
    b = 4
    while b < 7 and (1 << (3 * (b + 1))) <= 2 * n:
        b += 1
    return b


def stream_bytes(n: int, n_keep: int, storage: str) -> dict:
    """Algorithmic DRAM bytes of one plain step, per kernel class: what each
    kernel must read and write at least once (row bytes by storage type;
    the processing-order keys are cells and size classes, 2 x 8^b)."""
    col = {"f32": 224, "bf16": 112, "bf16s": 118}[storage]  # the 56 attribute rows
    es = 2 if storage == "bf16" else 4       # bytes of a log-scale element
    row = 12 + col                           # pos (FP32) + 56 attribute rows
    keys = 2 * (1 << (3 * cell_bits_for(n)))
    return {
        "features": n * row + 64 * n,        # all rows in, one 64-B record out
        "cells": n * (12 + 3 * es) + 8 * n,  # pos and log-scales in, (cell, slot) out
        "cell_scan": 8 * keys,               # counts in, offsets out
        "cell_scatter": 16 * n,              # (cell, slot) and the cell's offset in, order out
        "score": 72 * n,                     # record and order entry in, score out
        "select_pass": 12 * n,               # three passes over the scores
        "select_mask": 4 * n + n // 8,       # scores in, keep bits out
        "compact_count": n // 8,             # keep bits in
        "compact_scatter": n * row + n_keep * (row + 4),  # all rows in, kept rows and indices out
    }


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2606_09074_gb300", "csrc")
    for f in ("kernels_score.cu", "common.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_profile(kernel: str, workload_name: str):
    """The committed ncu record of a kernel on a workload (DRAM bytes and
    pipe figures per launch), or None when the kernel source has changed
    since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload_name}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    return rec


def score_work_flops(st: dict, n: int, views: int) -> float:
    """Algorithmic FP32 FLOPs of one score launch over all views, from the
    kernel's own counts of how each (primitive, view) pair was decided
    (refine_scene_stats): tiles found invisible cost nothing, tiles found
    visible only the weight, and pairs decided one by one the stages they
    entered (FLOP_COSTS)."""
    c = FLOP_COSTS
    return float(st["tile_views"] * c["tile_view"] + st["in_pairs"] * c["in_pair"]
                 + st["mixed_pairs"] * c["mixed_pair"]
                 + (st["open_u_pairs"] + st["open_v_pairs"]) * c["open_axis"]
                 + st["open_z_pairs"] * c["open_depth"] + st["visible_mixed_pairs"] * c["visible_mixed"]
                 + st["bound_pairs"] * c["bound_pair"] + (st["bound_u_pairs"] + st["bound_v_pairs"]) * c["bound_axis"]
                 + (st["exact_u_pairs"] + st["exact_v_pairs"]) * c["exact_axis"]
                 + n * ((views + 31) // 32) * c["kahan_block"] + n * c["epilogue"])


class ClockSampler:
    """SM clock, power and clock-event reasons of the benchmarked GPU, read
    through NVML (read-only queries; libnvidia-ml is loaded with ctypes):
    one sample at the start and one at the end of the timed region
    (sample()) and one every ~2 ms in between from a background thread."""
    # nvmlClocksEventReason* bits of the public NVML header
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    NVML_CLOCK_SM = 1

    def __init__(self, props, index: int, period_s: float = 0.002):
        import ctypes
        self.C = ctypes
        self.period = period_s
        self.samples = []  # (time, sm MHz, reasons bitmask, power W)
        self.max_mhz = None
        self.dev = None
        self._stop = threading.Event()
        self.th = None
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit_v2 failed")
            h = ctypes.c_void_p()
            ok = False
            dom, bus, devn = (getattr(props, k, None) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id"))
            if None not in (dom, bus, devn):
                bid = f"{dom:08X}:{bus:02X}:{devn:02X}.0".encode()
                ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bid), ctypes.byref(h)) == 0
            if not ok:
                ok = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) == 0
            if not ok:
                raise OSError("no NVML handle")
            self.dev = h
            mx = ctypes.c_uint()
            if self.lib.nvmlDeviceGetMaxClockInfo(self.dev, self.NVML_CLOCK_SM, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self._reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError):
            self.dev = None

    def sample(self):
        if self.dev is None:
            return
        C = self.C
        mhz, rs, mw = C.c_uint(), C.c_ulonglong(), C.c_uint()
        if self.lib.nvmlDeviceGetClockInfo(self.dev, self.NVML_CLOCK_SM, C.byref(mhz)) != 0:
            return
        if self._reasons(self.dev, C.byref(rs)) != 0:
            rs.value = 0
        power = mw.value / 1000.0 if self.lib.nvmlDeviceGetPowerUsage(self.dev, C.byref(mw)) == 0 else None
        self.samples.append((time.time(), float(mhz.value), int(rs.value), power))

    def _run(self):
        while not self._stop.is_set():
            self.sample()
            time.sleep(self.period)

    def start(self):
        if self.dev is not None:
            self.th = threading.Thread(target=self._run, daemon=True)
            self.th.start()

    def stop(self):
        self._stop.set()
        if self.th is not None:
            self.th.join(timeout=5)

    def summary(self, t0, t1):
        sel = [x for x in self.samples if t0 <= x[0] <= t1]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0, "source": "nvml"}
        reasons = set()
        for _, _, r, _ in sel:
            reasons.update(name for bit, name in self.REASONS.items() if r & bit)
        pw = [x[3] for x in sel if x[3] is not None]
        return {"sm_mhz": statistics.median(x[1] for x in sel), "sm_min_mhz": min(x[1] for x in sel),
                "sm_max_mhz": self.max_mhz, "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons), "samples": len(sel), "source": "nvml"}


def aggregate_over_ranks(local_ms: float, steps: int, pairs_per_step: int, world: int, dist=None,
                         device=None):
    """Max over ranks of the timed-region length; whole-job throughput =
    all ranks' pairs / that time.  Returns (max_ms, pairs_per_s)."""
    total_ms = float(local_ms)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps * pairs_per_step / (total_ms / 1000.0)


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank scores its own replica scene of the same shape."""
    return base_seed + 1000 * rank


# ----------------------------------------------------------------- oracle

def oracle_sample_run(w, m: int, threads: int):
    """The FP64 oracle on the first m primitives of a seeded permutation of
    the workload, all views: score -> select -> compact.  Returns seconds."""
    import oracle
    oracle.set_threads(threads)
    perm = np.random.default_rng(12).permutation(w.scene.n)[:m]
    sub = w.scene.subset(np.sort(perm))
    g = sub.params_f64()
    rows = np.concatenate([sub.pos, sub.attr], axis=0)
    t = time.perf_counter()
    o = oracle.score(g, w.cams, detail=False)
    mask, thr, nk = oracle.select(o["scores"], w.ratios[0])
    oracle.compact(rows, mask)
    return time.perf_counter() - t


def oracle_rate(w, budget_s: float, threads: int):
    """Pairs/s of the oracle on a bounded sample sized to ~budget_s."""
    m = min(2000, w.scene.n)
    dt = oracle_sample_run(w, m, threads)
    rate = m * len(w.cams) / max(dt, 1e-9)
    m2 = int(min(w.scene.n, max(m, rate * budget_s / len(w.cams))))
    if m2 > m:
        dt = oracle_sample_run(w, m2, threads)
        m = m2
    return m * len(w.cams) / dt, m, dt


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    w = workload(args.workload)
    threads = os.cpu_count() or 1
    steps = args.steps + args.warmup
    budget = max(0.05, min(20.0, 90.0 / max(steps, 1)))
    _, m, _ = oracle_rate(w, budget, threads)
    for _ in range(args.warmup):
        oracle_sample_run(w, m, threads)
    times = [oracle_sample_run(w, m, threads) for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps * m * len(w.cams) / tot
    sample = (f"{m} of {w.scene.n} primitives (seeded permutation) x all {len(w.cams)} views, "
              f"score+select+compact, FP64 oracle, OpenMP")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "n": w.scene.n, "views": len(w.cams),
                                            "ratio": w.ratios[0], "sample_primitives": m},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours

def end_to_end(args, torch, rb, ctx, w, attr, params, ratio, n_keep, pairs, V_all, stream):
    """Host-to-host throughput through the public API, from page-locked
    buffers: every step copies the scene and cameras in and the kept rows,
    indices and threshold out.  The headline form keeps `--e2e-inflight`
    requests in the request queue, so one request's copies overlap another's
    compute and the two link directions run together; the sequential form
    (refine_prune_host, one call after another) is reported beside it."""
    n = w.scene.n
    pos_h = torch.from_numpy(w.scene.pos).pin_memory()
    attr_h = attr.cpu().pin_memory()
    asz = rb.attr_col_bytes(attr)
    h2d = 12 * n + asz * n + 80 * V_all
    d2h = (12 + asz + 4) * n_keep + 4 + 4

    def outset():
        return {"out_pos": torch.empty((3, n_keep), dtype=torch.float32, pin_memory=True),
                "out_attr": rb.empty_attr_like(attr, n_keep, pin_memory=True),
                "idx": torch.empty(n_keep, dtype=torch.int32, pin_memory=True)}

    k_e2e = max(3, min(args.steps, 60))
    outs = outset()
    for _ in range(2):
        ctx.prune_host(pos_h, attr_h, w.cams, ratio, params=params, out=outs, stream=stream)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        ctx.prune_host(pos_h, attr_h, w.cams, ratio, params=params, out=outs, stream=stream)
    dt_seq = (time.perf_counter() - t0) / k_e2e
    sequential = {"value": pairs / dt_seq, "unit": "pairs/s", "ms_per_step": dt_seq * 1000, "steps": k_e2e,
                  "api": "refine_prune_host, one call after another"}
    if not args.no_ply:
        # the whole pruning as the paper times it (Table 2: sorting and saving
        # the primitives included): each step also writes the kept scene as a
        # 3DGS PLY file on the host
        import tempfile
        fd, path = tempfile.mkstemp(suffix=".ply")
        os.close(fd)

        def host_rows(o):
            a = o["out_attr"]
            if not isinstance(a, rb.MixedRows):
                a = a.view(torch.int16).numpy().view(np.uint16) if a.dtype == torch.bfloat16 else a.numpy()
            return o["out_pos"].numpy(), a
        k_ply = max(2, min(args.steps, 5))
        try:
            ctx.prune_host(pos_h, attr_h, w.cams, ratio, params=params, out=outs, stream=stream)
            rb.write_ply(path, *host_rows(outs))
            t0 = time.perf_counter()
            for _ in range(k_ply):
                ctx.prune_host(pos_h, attr_h, w.cams, ratio, params=params, out=outs, stream=stream)
                rb.write_ply(path, *host_rows(outs))
            dt_ply = (time.perf_counter() - t0) / k_ply
            ply_bytes = os.path.getsize(path)
        finally:
            os.remove(path)
        sequential["with_ply"] = {"value": pairs / dt_ply, "unit": "pairs/s", "ms_per_step": dt_ply * 1000,
                                  "steps": k_ply, "ply_bytes": ply_bytes,
                                  "api": "refine_prune_host + refine_write_ply of the kept scene (host temporary "
                                         "directory), one step after another"}

    D = args.e2e_inflight
    if D < 2:
        return {**sequential, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    dt_code = rb._dtype_code(attr)
    fp = rb.Queue.footprint(n, dt_code, len(w.cams), ratio)
    q = rb.Queue(ctx, budget_bytes=(D + 1) * fp, max_slots=D, params=params)
    sets = [outset() for _ in range(D + 1)]
    try:
        def run(k_total):
            inflight = []
            for k in range(k_total):
                if len(inflight) == D:
                    res, _ = q.poll(inflight.pop(0), timeout_ms=120_000)
                    if res["status"] != 0:
                        raise RuntimeError(f"queued request failed: {res['status']} {q.last_error()}")
                inflight.append(q.submit(pos_h, attr_h, w.cams, ratio, outputs=sets[k % (D + 1)], mask=False,
                                         compact=True, pin=True))
            for t in inflight:
                res, _ = q.poll(t, timeout_ms=120_000)
                if res["status"] != 0:
                    raise RuntimeError(f"queued request failed: {res['status']} {q.last_error()}")
        run(2 * D)
        t0 = time.perf_counter()
        run(k_e2e)
        dt = (time.perf_counter() - t0) / k_e2e
    finally:
        q.close()
    return {"value": pairs / dt, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1000, "steps": k_e2e,
            "api": f"refine_queue_submit / refine_queue_poll, {D} requests in flight, page-locked host buffers",
            "link_gbs": (h2d + d2h) / dt / 1e9, "sequential": sequential}


def run_ours(args, rank: int, world: int):
    import torch
    from paper_2606_09074_gb300 import binding as rb

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w = workload(args.workload, rank, args.storage)
    n, V, ratio = w.scene.n, len(w.cams), w.ratios[0]
    pos = torch.from_numpy(w.scene.pos).to(dev)
    if w.scene.dtype == "bf16s":
        attr = rb.MixedRows.from_float(w.scene.attr, device=dev)
    elif w.scene.dtype == "bf16":
        attr = torch.from_numpy(w.scene.attr.view(np.int16)).to(dev).view(torch.bfloat16)
    else:
        attr = torch.from_numpy(w.scene.attr).to(dev)
    cams = rb.cameras_to_device(w.cams, dev)
    n_keep = n - math.floor(ratio * n)
    scores = torch.empty(n, dtype=torch.float32, device=dev)
    mask = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    out_pos = torch.empty((3, n_keep), dtype=torch.float32, device=dev)
    out_attr = rb.empty_attr_like(attr, n_keep, device=dev)
    kept = torch.empty(n_keep, dtype=torch.int32, device=dev)
    ctx = rb.Context(local)
    stream = torch.cuda.current_stream(dev)
    params = rb.default_params(max_views=args.max_views) if args.max_views else None
    V_all = V
    if args.max_views and V > args.max_views:
        V = -(-V // -(-V // args.max_views))  # views scored: every ceil(V / max_views)-th

    def step():
        ctx.score(pos, attr, cams, scores=scores, params=params, stream=stream)
        ctx.select(scores, ratio, mask=mask, threshold=False, stream=stream)
        ctx.compact(pos, attr, mask, n_keep, out_pos=out_pos, out_attr=out_attr, kept_idx=True,
                    out_row_stride=n_keep, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ctx.check()
    ctx.kernel_times()

    clocks = ClockSampler(torch.cuda.get_device_properties(dev), local)
    # inside the timed region only the score kernel is bracketed by events
    # (two per step); events around all 14 kernels would add ~0.06 ms a step
    ctx.set_timing(True, score_only=True)
    launches0 = ctx.launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    clocks.sample()
    clocks.start()
    evs[0].record(stream)
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    clocks.sample()
    if dist:
        dist.barrier()
    t_wall1 = time.time()
    launches = ctx.launch_count() - launches0
    ctx.set_timing(False)
    ktimes = ctx.kernel_times()
    clocks.stop()
    ctx.check()
    # per-kernel breakdown: every kernel bracketed, a few steps after the timed region
    b_steps = max(1, min(args.steps, 50))
    ctx.set_timing(True)
    for _ in range(b_steps):
        step()
    torch.cuda.synchronize(dev)
    ctx.set_timing(False)
    kt_all = ctx.kernel_times()
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    pairs = n * V
    total_ms, value = aggregate_over_ranks(evs[0].elapsed_time(evs[-1]), args.steps, pairs, world,
                                           dist, dev)
    ms_step = total_ms / args.steps

    # roofline of the dominant kernel (score): live CUDA-event timing of the
    # timed region; the work it did from one counting pass after it
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    clk_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * clk_max * 1e6 / 1e12
    sc = ktimes.get("score", {"ms": float("nan"), "launches": 1})
    score_ms = sc["ms"] / max(sc["launches"], 1)
    score_ms_step = sc["ms"] / args.steps  # all passes of a step (one pass up to 512 views)
    _, work = ctx.score(pos, attr, cams, params=params, stats=True, stream=stream)
    flops = score_work_flops(work, n, V)
    achieved = flops / (score_ms_step / 1000.0) / 1e12
    prof = recorded_profile("score", args.workload) if args.storage == "f32" and not args.max_views else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": prof.get("dram_bytes_per_launch") if prof else None,
                "kernel": "k_score", "kernel_ms": score_ms, "flops_per_step": flops,
                "flops_basis": "FP32 work of the stages each (primitive, view) pair needed, from the kernel's own "
                               "pair-class counters of this scene: invisible tiles 0, visible tiles the Eq. 17 "
                               "weight, pairs decided one by one their open axes, footprint bound and exact "
                               "footprint test (FMA = 2, compare/max/reciprocal = 1)",
                "pair_classes": {k: work[k] for k in ("pairs", "in_pairs", "out_pairs", "mixed_pairs",
                                                      "bound_pairs", "footprint_pairs")},
                "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                              f"{clk_max:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
                "kernels_ms_per_step": {k: v["ms"] / b_steps for k, v in kt_all.items()},
                "kernels_ms_per_step_basis": f"every kernel bracketed by CUDA events, {b_steps} steps after the "
                                             f"timed region"}
    # the measured FP32 FMA rate of this device (refine_fma_rate), beside
    # the nominal peak above
    fma_rate, fma_ms = ctx.fma_rate(stream=stream)
    roofline["peak_measured"] = fma_rate / 1e12
    roofline["frac_of_measured"] = achieved / (fma_rate / 1e12)
    roofline["peak_measured_basis"] = (f"refine_fma_rate: 8 CTAs x 256 threads per SM, 8 independent FP32 FMA "
                                       f"chains per thread, one launch of {fma_ms:.2f} ms timed with CUDA events "
                                       f"after the timed region")
    # every kernel against the measured HBM copy peak, by its algorithmic bytes
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    kb = stream_bytes(n, n_keep, w.scene.dtype)
    per_kernel = {}
    for k, v in kt_all.items():
        ms_k = v["ms"] / b_steps
        entry = {"ms": ms_k}
        if k in kb and ms_k > 0:
            gbs = kb[k] / (ms_k * 1e-3) / 1e9
            entry.update({"bytes": kb[k], "gbs": gbs, "frac_hbm": gbs / hbm})
        per_kernel[k] = entry
    roofline["kernels"] = per_kernel
    roofline["kernels_basis"] = (f"algorithmic bytes per step (each input byte read once, each output byte "
                                 f"written once) / the kernel's event-bracketed time, against the measured "
                                 f"{hbm:.0f} GB/s copy peak of MEASURED_PEAKS.json")
    if prof:
        roofline["ncu"] = {k: prof[k] for k in ("fp32_flops_executed", "fp32_executed_frac", "fma_pipe_pct",
                                                "issue_active_pct", "thread_inst_per_pair", "source")
                           if k in prof}
    clock_summary = clocks.summary(t_wall0, t_wall1)

    line = None
    if rank == 0:
        # end to end through the public API from pinned host memory
        e2e = None
        if not args.no_e2e:
            e2e = end_to_end(args, torch, rb, ctx, w, attr, params, ratio, n_keep, pairs, V_all, stream)
        cpu = None
        if not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            rate, m, dt = oracle_rate(w, 12.0, threads)
            import oracle
            cpu = {"value": rate, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": f"{m} of {n} primitives (seeded permutation) x all {V} views, "
                             f"score+select+compact, {dt:.1f} s"}
        acc = accuracy_report(ctx, w, pos, attr, cams, ratio, stream) if args.accuracy else None
        lat = sorted(per_step)
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if w.scene.dtype == "f32" else f"f32 ({w.scene.dtype} storage)", "data": "synthetic",
                "config": {"workload": w.name, "n": n, "views": V, "ratio": ratio, "storage": w.scene.dtype,
                           "l2": f"inputs larger than L2 ({stream_bytes(n, 0, w.scene.dtype)['compact_scatter'] / 1e6:.0f} MB scene), no flush",
                           "parallelism": "replicas" if world > 1 else "single"},
                "scenes_per_s": world * 1000.0 / ms_step,
                "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clock_summary, "gpu": props.name}
        if acc is not None:
            line["accuracy"] = acc
        if params is not None:
            # keep masks of the subsampled and of the all-view scoring
            s_all = ctx.score(pos, attr, cams, stream=stream)
            m_all, _, _ = ctx.select(s_all, ratio, stream=stream)
            a = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:n]
            b = np.unpackbits(m_all.cpu().numpy().view(np.uint8), bitorder="little")[:n]
            line["view_subsampling"] = {"max_views": args.max_views, "views_scored": V, "views_total": V_all,
                                        "mask_agreement_vs_all_views": float((a == b).mean())}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()
    return line


def accuracy_report(ctx, w, pos, attr, cams, ratio, stream):
    """Scores against the FP64 oracle: max / p99 relative error on a seeded
    100k-primitive sample (statistics from the whole scene), against the same
    stored numbers and, for BF16 storage, against the float32 scene they were
    rounded from; and keep-mask agreement with the oracle's full-scene
    selection on the float32 scene."""
    import oracle
    from paper_2606_09074_gb300 import synth
    sc = ctx.score(pos, attr, cams, stream=stream)
    mask, _, _ = ctx.select(sc, ratio, stream=stream)
    s = sc.cpu().numpy().astype(np.float64)
    got = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[: w.scene.n].astype(bool)
    oracle.set_threads(os.cpu_count() or 1)
    idx = np.sort(np.random.default_rng(7).choice(w.scene.n, min(100_000, w.scene.n), replace=False))
    rep = {"sample": int(idx.size)}

    def rel(ref):
        clean = (ref["nborder"] == 0) & (ref["scores"] > 0)
        r = np.abs(s[idx][clean] - ref["scores"][clean]) / ref["scores"][clean]
        return {"max": float(r.max()), "p99": float(np.quantile(r, 0.99)), "mean": float(r.mean()),
                "checked": int(clean.sum())}

    rep["vs_oracle_same_inputs"] = rel(oracle.score_subset(w.scene.params_f64(), idx, w.cams))
    src = w.scene
    if w.scene.dtype in ("bf16", "bf16s"):
        src = synth.config2(seed=2, dtype="f32").scene
        rep["vs_oracle_fp32_source"] = rel(oracle.score_subset(src.params_f64(), idx, w.cams))
    ref = oracle.score(src.params_f64(), w.cams, detail=False)
    m_ref, _, _ = oracle.select(ref["scores"], ratio)
    want = np.unpackbits(m_ref.view(np.uint8), bitorder="little")[: w.scene.n].astype(bool)
    rep["mask_agreement_vs_oracle"] = float((got == want).mean())
    rep["mask_agreement_reference"] = "FP64 oracle on the float32 scene, full N"
    return rep


def run_batch_mode(args):
    """64 scenes (seeds 100..163: N log-uniform in [50k, 2M], V in 50..300,
    three resolutions, ratio 0.66): the batched BF16 form against per-scene
    calls of the plain path (FP32, and BF16 for reference)."""
    import torch
    from paper_2606_09074_gb300 import binding as rb
    from paper_2606_09074_gb300 import synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    seeds = list(range(100, 100 + args.scenes))
    scenes = []
    for sd in seeds:
        w = synth.batch_scene(sd, dtype="f32")
        pos = torch.from_numpy(w.scene.pos).to(dev)
        a32 = torch.from_numpy(w.scene.attr).to(dev)
        a16 = torch.from_numpy(synth.f32_to_bf16_bits(w.scene.attr).view(np.int16)).to(dev).view(torch.bfloat16)
        x = {"pos": pos, "a32": a32, "a16": a16, "cams": rb.cameras_to_device(w.cams, dev),
             "n": w.scene.n, "V": len(w.cams), "ratio": 0.66}
        if args.form_storage == "bf16s":
            x["amx"] = rb.MixedRows.from_float(w.scene.attr, device=dev)
        scenes.append(x)
    fkey = "amx" if args.form_storage == "bf16s" else "a16"  # attribute rows of the batched form
    pairs = sum(x["n"] * x["V"] for x in scenes)
    ctx = rb.Context(0)
    stream = torch.cuda.current_stream(dev)
    # tile and CTA shape of the score kernels from the autotuner (results do
    # not depend on it); every path below runs with the tuned shape
    best, table = ctx.autotune([{"pos": x["pos"], "attr": x[fkey], "cams": x["cams"], "ratio": x["ratio"]}
                                for x in scenes], reps=3)

    def plain(key):
        outs = []
        for x in scenes:
            nk = x["n"] - math.floor(x["ratio"] * x["n"])
            outs.append({"scores": torch.empty(x["n"], device=dev),
                         "mask": torch.empty((x["n"] + 31) // 32, dtype=torch.int32, device=dev),
                         "op": torch.empty((3, nk), device=dev),
                         "oa": rb.empty_attr_like(x[key], nk, device=dev), "nk": nk})

        def step():
            for x, o in zip(scenes, outs):
                ctx.score(x["pos"], x[key], x["cams"], scores=o["scores"], stream=stream)
                ctx.select(o["scores"], x["ratio"], mask=o["mask"], threshold=False, stream=stream)
                ctx.compact(x["pos"], x[key], o["mask"], o["nk"], out_pos=o["op"], out_attr=o["oa"],
                            kept_idx=False, out_row_stride=o["nk"], stream=stream)
        return step

    def timed(step, k):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(k):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k, (time.perf_counter() - t0) * 1000 / k

    res = {}
    plains = (("a32", "plain_f32"), ("a16", "plain_bf16")) + ((("amx", "plain_bf16s"),) if fkey == "amx" else ())
    for key, name in plains:
        dev_ms, wall_ms = timed(plain(key), args.batch_steps)
        res[name] = {"ms_per_batch": dev_ms, "wall_ms_per_batch": wall_ms,
                     "scenes_per_s": len(scenes) * 1000 / wall_ms, "pairs_per_s": pairs * 1000 / wall_ms}
    batch = rb.Batch(ctx, [{"pos": x["pos"], "attr": x[fkey], "cams": x["cams"], "ratio": x["ratio"]}
                           for x in scenes])
    dev_ms, wall_ms = timed(lambda: batch.run(stream), args.batch_steps)
    bname = f"batched_{args.form_storage}"
    res[bname] = {"ms_per_batch": dev_ms, "wall_ms_per_batch": wall_ms,
                           "scenes_per_s": len(scenes) * 1000 / wall_ms, "pairs_per_s": pairs * 1000 / wall_ms,
                           "kernels_per_run": batch.launches()}
    # the batched scores equal the per-scene BF16 path bit for bit
    plain(key=fkey)  # allocate nothing new; check a few scenes directly
    same = True
    for k in (0, len(scenes) // 2, len(scenes) - 1):
        x = scenes[k]
        s = ctx.score(x["pos"], x[fkey], x["cams"])
        same &= bool(torch.equal(s, batch.outputs[k]["scores"]))
    ctx.check()
    acc = batch_accuracy(batch, seeds, scenes) if args.accuracy else None
    line = {"mode": "batch", "metric": "scenes/s", "value": res[bname]["scenes_per_s"],
            "unit": "scenes/s", "n_gpus": 1, "steps": args.batch_steps, "warmup": args.warmup,
            "scenes": len(scenes), "pairs_per_batch": pairs, "primitives": sum(x["n"] for x in scenes),
            "storage": args.form_storage,
            "speedup_vs_plain_f32": res["plain_f32"]["wall_ms_per_batch"] / res[bname]["wall_ms_per_batch"],
            "speedup_vs_plain_bf16": res["plain_bf16"]["wall_ms_per_batch"] / res[bname]["wall_ms_per_batch"],
            "batched_scores_equal_plain": same, "results": res, "data": "synthetic",
            "autotune": {"best": best, "candidates": table},
            "config": {"workload": "64 scenes, seeds 100-163, N log-uniform 50k-2M, V 50-300, ratio 0.66"}}
    if acc is not None:
        line["accuracy"] = acc
    print(json.dumps(line), flush=True)
    batch.close()
    ctx.close()


def batch_accuracy(batch, seeds, scenes):
    """The batched BF16 scores and keep masks of every scene against the FP64
    oracle on the float32 scene each was rounded from (every primitive, all
    views): keep-mask agreement per scene and relative score error over the
    primitives whose oracle score is positive and has no borderline pair."""
    import oracle
    from paper_2606_09074_gb300 import synth
    oracle.set_threads(os.cpu_count() or 1)
    agree, rel_mean, rel_p99 = [], [], []
    t0 = time.perf_counter()
    for k, sd in enumerate(seeds):
        w = synth.batch_scene(sd, dtype="f32")
        ref = oracle.score(w.scene.params_f64(), w.cams)
        m_ref, _, _ = oracle.select(ref["scores"], scenes[k]["ratio"])
        n = w.scene.n
        want = np.unpackbits(m_ref.view(np.uint8), bitorder="little")[:n].astype(bool)
        out = batch.outputs[k]
        got = np.unpackbits(out["mask"].cpu().numpy().view(np.uint8), bitorder="little")[:n].astype(bool)
        agree.append(float((got == want).mean()))
        s = out["scores"].cpu().numpy().astype(np.float64)
        clean = (ref["nborder"] == 0) & (ref["scores"] > 0)
        r = np.abs(s[clean] - ref["scores"][clean]) / ref["scores"][clean]
        rel_mean.append(float(r.mean()))
        rel_p99.append(float(np.quantile(r, 0.99)))
    return {"reference": "FP64 oracle on the float32 scenes, every primitive, all views",
            "mask_agreement": {"min": min(agree), "mean": statistics.mean(agree),
                               "below_99.9": sum(a < 0.999 for a in agree), "per_scene": agree},
            "rel_error": {"mean_of_means": statistics.mean(rel_mean), "max_p99": max(rel_p99)},
            "oracle_s": time.perf_counter() - t0}


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


class _OutputSets:
    """Page-locked output buffers for the serving run: `count` flat sets,
    each large enough for the largest pool scene at ratio 0.5 (the queue
    writes each output contiguously, so a larger buffer serves any job)."""

    def __init__(self, torch, n_max, count, col_bytes=112):
        nk = n_max - n_max // 2
        self.free = []
        self.cv = threading.Condition()
        for _ in range(count):
            self.free.append({"mask": torch.empty((n_max + 31) // 32, dtype=torch.int32, pin_memory=True),
                              "out_pos": torch.empty(3 * nk, dtype=torch.float32, pin_memory=True),
                              "out_attr": torch.empty(col_bytes * nk, dtype=torch.uint8, pin_memory=True),
                              "idx": torch.empty(nk, dtype=torch.int32, pin_memory=True)})

    def take(self):
        with self.cv:
            while not self.free:
                self.cv.wait()
            return self.free.pop()

    def give(self, s):
        with self.cv:
            self.free.append(s)
            self.cv.notify_all()


def _serve_pass(torch, rb, pool, jobs, arrivals, q, outsets, on_done=None):
    """Submits `jobs` [(pool index, ratio)] to queue `q` at `arrivals`
    (seconds from the start; None = as fast as output buffers allow) and
    collects them.  Returns per-job latencies (ms, arrival to the last output
    byte in host memory), round sizes and the wall time (s).  on_done(k, p,
    r, result, outputs) sees every job before its buffers are reused."""
    sub = []  # (ticket, pool index, ratio, outputs, arrival perf time, submit perf time)
    lock = threading.Lock()
    ready = threading.Semaphore(0)
    t_start = time.perf_counter()

    def feeder():
        for k, (p, r) in enumerate(jobs):
            if arrivals is not None:
                delay = t_start + arrivals[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            t_arr = t_start + arrivals[k] if arrivals is not None else time.perf_counter()
            outs = outsets.take()
            sc = pool[p]
            t_sub = time.perf_counter()
            t = q.submit(sc["pos"], sc["attr"], sc["cams"], r, outputs=outs, mask=True, compact=True)
            with lock:
                sub.append((t, p, r, outs, t_arr, t_sub))
            ready.release()

    th = threading.Thread(target=feeder, daemon=True)
    th.start()
    lat, rounds = [], []
    by_ticket, seen = {}, 0
    for _ in range(len(jobs)):
        ready.acquire()  # one more job submitted
        ticket, res, _ = q.poll_any(timeout_ms=-1)  # results in completion order
        with lock:
            while seen < len(sub):
                by_ticket[sub[seen][0]] = (seen, sub[seen])
                seen += 1
            k, (t, p, r, outs, t_arr, t_sub) = by_ticket.pop(ticket)
        if res["status"] != 0:
            raise RuntimeError(f"serving job {k} failed: status {res['status']} {q.last_error()}")
        # queue clock: submit -> done; host clock: arrival -> submit
        lat.append(res["done_ms"] - res["submit_ms"] + (t_sub - t_arr) * 1000.0)
        rounds.append(res["round_size"])
        if on_done is not None:
            on_done(k, p, r, res, outs)
        outsets.give(outs)
    wall = time.perf_counter() - t_start
    th.join()
    return lat, rounds, wall


def _pool_scene(seed):
    """One serving-pool scene (FP32) in a worker process: positions, the
    attribute rows, and the cameras."""
    from paper_2606_09074_gb300 import synth
    w = synth.job_scene(seed, dtype="f32")
    return w.scene.pos, w.scene.attr, w.cams


def _round_hist(rounds):
    h = {}
    for r in rounds:
        h[str(r)] = h.get(str(r), 0) + 1
    return dict(sorted(h.items(), key=lambda kv: int(kv[0])))


def run_serve_mode(args):
    """Serving workload: `--jobs` pruning jobs (seeds 1000.., each with the
    ratio its seed draws from {0.5, 0.66, 0.9}) arriving as a Poisson stream
    at `--rate`/s (seed 999), served by the request queue with BF16 storage
    from page-locked host memory, against the plain FP32 per-scene path
    (refine_prune_host) as one FIFO server fed the same arrivals; then the
    same jobs back to back (saturation), at the full HBM budget and at a
    reduced one that makes admission bind.  Job k scores pool scene k mod
    `--pool` (distinct seeded scenes drawn as in the batch workload, N
    log-uniform in [50k, 3.5M]), generated ahead of the run."""
    import multiprocessing as mp
    from paper_2606_09074_gb300 import synth
    P = args.pool
    t_gen = time.perf_counter()
    # generated in spawned workers before this process makes any CUDA call
    with mp.get_context("spawn").Pool(max(1, min(P, (os.cpu_count() or 2) - 1))) as wp:
        raw = wp.map(_pool_scene, [1000 + k for k in range(P)], chunksize=1)
    t_gen = time.perf_counter() - t_gen
    import torch
    from paper_2606_09074_gb300 import binding as rb
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pool = []
    for pos, attr, cams in raw:
        if args.form_storage == "bf16s":
            af = rb.MixedRows.from_float(attr, pin_memory=True)  # log-scales float32, the rest bfloat16
        else:
            af = torch.from_numpy(synth.f32_to_bf16_bits(attr).view(np.int16)).view(torch.bfloat16).pin_memory()
        pool.append({"pos": torch.from_numpy(pos).pin_memory(), "a32": torch.from_numpy(attr).pin_memory(),
                     "attr": af, "cams": cams, "n": pos.shape[1], "V": len(cams)})
    del raw
    ratio_of = lambda k: synth.job_spec(1000 + k)[3]  # noqa: E731
    jobs = [(k % P, ratio_of(k)) for k in range(args.jobs)]
    arrivals = synth.job_arrivals(args.jobs, rate=args.rate, seed=999)
    sat_jobs = [(k % P, ratio_of(k)) for k in range(args.sat_jobs)]
    ctx = rb.Context(0)
    n_max = max(sc["n"] for sc in pool)

    def plain_server(job_list, arr, out):
        """The plain FP32 path as one FIFO server thread fed the same
        arrivals (None = back to back): latencies (ms) and wall (s)."""
        lat = []
        t_start = time.perf_counter()
        for k, (p, r) in enumerate(job_list):
            if arr is not None:
                delay = t_start + arr[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            t_arr = t_start + arr[k] if arr is not None else time.perf_counter()
            sc = pool[p]
            nk = sc["n"] - int(math.floor(r * sc["n"]))
            o = {"out_pos": out["out_pos"][: 3 * nk].view(3, nk), "out_attr": out["out_attr"][: 56 * nk].view(56, nk),
                 "idx": out["idx"][:nk]}
            ctx.prune_host(sc["pos"], sc["a32"], sc["cams"], r, out=o)
            lat.append((time.perf_counter() - t_arr) * 1000.0)
        return lat, time.perf_counter() - t_start

    nk_max = n_max - n_max // 2
    plain_out = {"out_pos": torch.empty(3 * nk_max, dtype=torch.float32, pin_memory=True),
                 "out_attr": torch.empty(56 * nk_max, dtype=torch.float32, pin_memory=True),
                 "idx": torch.empty(nk_max, dtype=torch.int32, pin_memory=True)}
    plain_server(sat_jobs[: min(8, len(sat_jobs))], None, plain_out)  # warm-up
    plain_lat, plain_wall_p = plain_server(jobs, arrivals, plain_out)
    _, plain_wall = plain_server(sat_jobs, None, plain_out)
    plain_sat = len(sat_jobs) / plain_wall
    del plain_out

    outsets = _OutputSets(torch, n_max, args.slots + 4, 118 if args.form_storage == "bf16s" else 112)
    budget = int(args.budget_gb * (1 << 30))
    small_budget = int(args.small_budget_gb * (1 << 30))

    # keep masks of the plain FP32 GPU path and of the FP64 oracle (on a
    # seeded subset of the pool scenes, float32 inputs), for agreement
    keep_gpu, keep_orc = {}, {}
    orc_scenes = set(np.random.default_rng(5).choice(P, min(args.oracle_scenes, P), replace=False).tolist())
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    for p, r in sorted(set(jobs)):
        sc = pool[p]
        res = ctx.prune_host(sc["pos"], sc["a32"], sc["cams"], r)
        keep = np.zeros(sc["n"], dtype=bool)
        keep[res["idx"].numpy()] = True
        keep_gpu[(p, r)] = keep
    t_orc = time.perf_counter()
    orc_scores = {}
    for p in sorted(orc_scenes):
        sc = pool[p]
        g = np.concatenate([sc["pos"].numpy(), sc["a32"].numpy()], axis=0).astype(np.float64)
        orc_scores[p] = oracle.score(g, sc["cams"], detail=False)["scores"]
    for p, r in sorted(set(jobs)):
        if p in orc_scores:
            m, _, _ = oracle.select(orc_scores[p], r)
            keep_orc[(p, r)] = np.unpackbits(m.view(np.uint8), bitorder="little")[: pool[p]["n"]].astype(bool)
    t_orc = time.perf_counter() - t_orc

    agree_gpu, agree_orc = [], []

    def record(k, p, r, res, outs):
        nk = res["n_keep"]
        keep = np.zeros(pool[p]["n"], dtype=bool)
        keep[outs["idx"][:nk].numpy()] = True
        agree_gpu.append(float(np.mean(keep == keep_gpu[(p, r)])))
        if (p, r) in keep_orc:
            agree_orc.append(float(np.mean(keep == keep_orc[(p, r)])))

    def run(job_list, arr, bud, on_done=None, slots=args.slots):
        q = rb.Queue(ctx, budget_bytes=bud, max_slots=slots)
        try:
            # warm-up on the same queue: its memory pool grows to the working
            # set of a saturated run before the measured pass
            _serve_pass(torch, rb, pool, sat_jobs[: min(4 * slots, len(sat_jobs))], None, q, outsets)
            st0 = q.stats()
            lat, rounds, wall = _serve_pass(torch, rb, pool, job_list, arr, q, outsets, on_done)
            st = q.stats()
        finally:
            q.close()
        st = {**st, "rounds": st["rounds"] - st0["rounds"], "dispatch_ms": st["dispatch_ms"] - st0["dispatch_ms"]}
        return lat, rounds, wall, st

    lat, rounds, wall, st = run(jobs, arrivals, budget, record)
    lat_s, rounds_s, wall_s, st_s = run(sat_jobs, None, budget)
    # more slots than the reduced budget can fill: admission is bounded by bytes
    lat_b, rounds_b, wall_b, st_b = run(sat_jobs, None, small_budget, slots=args.small_budget_slots)
    served_sat = len(sat_jobs) / wall_s
    pairs = sum(pool[p]["n"] * pool[p]["V"] for p, _ in sat_jobs)
    ns = [sc["n"] for sc in pool]

    def side(lat_, rounds_, wall_, st_, n_jobs):
        return {"jobs": n_jobs, "wall_s": wall_, "scenes_per_s": n_jobs / wall_,
                "p50_ms": _percentile(lat_, 0.5), "p99_ms": _percentile(lat_, 0.99),
                "mean_round": statistics.mean(rounds_), "max_round": max(rounds_),
                "round_sizes": _round_hist(rounds_), "peak_bytes": st_["peak_bytes"], "rounds": st_["rounds"],
                "slots": st_["slots"], "dispatch_ms_per_job": st_["dispatch_ms"] / max(n_jobs, 1)}

    line = {"mode": "serve", "metric": "scenes/s", "value": served_sat, "unit": "scenes/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": f"f32 ({args.form_storage} storage)", "data": "synthetic",
            "poisson": {**side(lat, rounds, wall, st, len(jobs)), "rate_per_s": args.rate,
                        "plain_f32_p50_ms": _percentile(plain_lat, 0.5),
                        "plain_f32_p99_ms": _percentile(plain_lat, 0.99), "plain_f32_wall_s": plain_wall_p},
            "saturation": {**side(lat_s, rounds_s, wall_s, st_s, len(sat_jobs)),
                           "served_pairs_per_s": pairs / wall_s, "plain_f32_scenes_per_s": plain_sat,
                           "speedup_vs_plain_f32": served_sat / plain_sat},
            "saturation_small_budget": {**side(lat_b, rounds_b, wall_b, st_b, len(sat_jobs)),
                                        "budget_bytes": small_budget,
                                        "speedup_vs_plain_f32": len(sat_jobs) / wall_b / plain_sat},
            "mask_agreement_vs_plain_f32_gpu": {"min": min(agree_gpu), "mean": statistics.mean(agree_gpu),
                                                "jobs": len(agree_gpu),
                                                "below_99.9": sum(a < 0.999 for a in agree_gpu)},
            "mask_agreement_vs_fp64_oracle": {"min": min(agree_orc) if agree_orc else None,
                                              "mean": statistics.mean(agree_orc) if agree_orc else None,
                                              "jobs": len(agree_orc), "scenes": sorted(orc_scenes),
                                              "below_99.9": sum(a < 0.999 for a in agree_orc),
                                              "oracle_s": t_orc},
            "queue": {"budget_bytes": budget, "slots": args.slots},
            "pool": {"scenes": P, "seeds": f"1000-{999 + P}", "n_min": min(ns), "n_max": max(ns),
                     "n_mean": statistics.mean(ns), "generate_s": t_gen},
            "config": {"workload": f"serving: {args.jobs} jobs, Poisson arrivals at {args.rate}/s (seed 999), then "
                                   f"{args.sat_jobs} back to back; job k scores pool scene k mod {P} (seeds "
                                   f"1000-{999 + P}, N log-uniform 50k-3.5M, V 50-300) with the ratio its seed "
                                   f"draws; {args.form_storage.upper()} storage; HBM budget {args.budget_gb} GB (and "
                                   f"{args.small_budget_gb} GB)",
                       "plain_path": "refine_prune_host, FP32, one FIFO server thread fed the same arrivals "
                                     "from page-locked host memory"}}
    print(json.dumps(line), flush=True)
    ctx.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c0"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ply", action="store_true", help="end to end: leave out the timed PLY writing")
    ap.add_argument("--e2e-inflight", type=int, default=3,
                    help="requests in flight in the end-to-end measurement (1: sequential calls only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form-storage", default="bf16", choices=["bf16", "bf16s"],
                    help="batch / serve: attribute rows of the batched and served forms (bfloat16, or bfloat16 "
                         "with float32 log-scales)")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "bf16s"],
                    help="attribute rows: float32, bfloat16, or bfloat16 with float32 log-scales")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve"],
                    help="single: the default workload; batch: 64 scenes, batched vs per-scene; "
                         "serve: the request queue under Poisson and back-to-back arrivals")
    ap.add_argument("--scenes", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--max-views", type=int, default=0,
                    help="score every ceil(V/max_views)-th view (Table B.1 subsampling); 0 = all")
    ap.add_argument("--jobs", type=int, default=2000, help="serve: Poisson jobs")
    ap.add_argument("--sat-jobs", type=int, default=2000, help="serve: back-to-back jobs")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: arrivals per second")
    ap.add_argument("--pool", type=int, default=128, help="serve: distinct scenes")
    ap.add_argument("--slots", type=int, default=32, help="serve: requests in flight")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: HBM budget")
    ap.add_argument("--small-budget-gb", type=float, default=4.0, help="serve: reduced HBM budget")
    ap.add_argument("--small-budget-slots", type=int, default=32,
                    help="serve: slots of the reduced-budget run (more than its budget can fill)")
    ap.add_argument("--oracle-scenes", type=int, default=16,
                    help="serve: pool scenes whose keep masks are also checked against the FP64 oracle")
    ap.add_argument("--accuracy", action="store_true",
                    help="also report error and mask agreement against the FP64 oracle")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(1)))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.mode == "batch":
        run_batch_mode(args)
    elif args.mode == "serve":
        run_serve_mode(args)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
