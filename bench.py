"""Benchmark of the Aggregate Risk Analysis hot path on GB300.

One step = one pass of the whole path over the paper-scale workload: the per-layer fold of
per-ELT and occurrence terms, the YET stream (trial sums, aggregate terms, YLT write) and
PML(100), PML(250), TVaR(0.99) of the YLT, with the metrics read back to the host.

Workload (paper scale): 1 layer of 15 ELTs x 20,000 events over a 2,000,000-event catalogue
(FP32 lognormal(11, 2) losses), YET of 1,000,000 trials x 1,000 events (4 GB of event IDs,
larger than L2, so no cache flush is needed between steps).  Synthetic, seeded.

Metric: event-ELT lookups per second, counted as logical (occurrence, ELT) pairs,
sum_t n_t x |ELTs of the layer| per step.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs its own replica on its own GPU (trials are independent; no
data-path collective), and value is the aggregate over ranks (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_TRIALS = 1_000_000
EVENTS_PER_TRIAL = 1000
N_ELTS = 15
CATALOGUE = 2_000_000
RPS = [100.0, 250.0]
LEVELS = [0.99]
WORKLOAD = "paper_scale: 1 layer x 15 ELTs (20k events each, 2M catalogue, FP32 losses), 1e6 trials x 1000 events"
METRIC = "event-ELT lookups/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--flags", type=int, default=0, help="ARA_RUN_* flags (measurement variants)")
    ap.add_argument("--trials", type=int, default=N_TRIALS)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU-baseline sample time")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-portfolio measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-oep", action="store_true", help="skip the occurrence-basis measurement")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--no-layouts", action="store_true", help="skip the layout-variant timings")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# Distributed plumbing (one process per GPU under torchrun)
# ------------------------------------------------------------------------------------------
def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# Clocks during the timed region
# ------------------------------------------------------------------------------------------
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a while to start: the region begins once it has sampled
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.005)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(REASONS, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# Inputs
# ------------------------------------------------------------------------------------------
def make_inputs(seed: int, n_trials: int, pinned: bool):
    import torch
    import synth
    pf = synth.paper_scale_portfolio(0)
    ids = torch.empty(n_trials * EVENTS_PER_TRIAL, dtype=torch.int32, pin_memory=pinned)
    yet = synth.paper_scale_yet(seed, n_trials=n_trials, ids_out=ids.numpy())
    off = torch.from_numpy(yet.offsets)
    if pinned:
        off = off.pin_memory()
    return pf, yet, ids, off


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def stream_kernel_name(flags):
    """The YET-stream kernel a run with these ARA_RUN_* flags launches."""
    import paper_1606_04473_gb300 as ara
    if flags & ara.ARA_RUN_PER_ELT:
        return "k_ylt_per_elt"
    if flags & (ara.ARA_RUN_LDG | ara.ARA_RUN_HOST_DIRECT):
        return "k_ylt_folded"
    return "k_ylt_bulk"


def ncu_profile_figures():
    """Per-occurrence figures of the YET-stream kernel from the committed ncu capture figures
    (profiles/k_ylt_bulk_paper_scale.txt, lines 'key: value'): dram_bytes_per_event,
    l2_hit_rate_pct, gather_sectors_per_event.  Empty when the file is absent or was taken of
    another kernel source (its 'kernel_source_sha' line differs)."""
    path = os.path.join(ROOT, "profiles", "k_ylt_bulk_paper_scale.txt")
    out = {}
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                line = line.strip()
                if line.startswith("#"):
                    continue
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip().strip("`")] = v.strip().strip("`")
        if kv.get("kernel_source_sha") != kernel_source_sha():
            return out
        for k in ("dram_bytes_per_event", "l2_hit_rate_pct", "gather_sectors_per_event"):
            if k in kv:
                out[k] = float(kv[k].split()[0])
    except Exception:
        pass
    return out


def kernel_source_sha():
    """Hash of the stream kernel's sources with line comments, trailing blanks and empty lines
    removed: a change of the code voids the recorded traffic, a change of a comment does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("ara_ylt.cu", "ara_device.cuh"):
        with open(os.path.join(ROOT, "paper_1606_04473_gb300", "csrc", name)) as f:
            for line in f:
                code = re.sub(r"//.*$", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


# ------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ------------------------------------------------------------------------------------------
def oracle_sample_rate(pf, yet_fn, target_s: float, max_trials: int = N_TRIALS, single_core=True):
    """Time the oracle on the first K trials (K sized for ~target_s on all host cores, at most the
    whole workload), and on one core over a sample 1/16 of that size."""
    import oracle
    calib = 2000
    y = yet_fn(calib)
    oracle.ylt(pf, y)  # warm (builds the direct-access tables once per call; part of the work)
    t0 = time.perf_counter()
    oracle.ylt(pf, y)
    dt = time.perf_counter() - t0
    k = int(max(calib, min(max_trials, calib * target_s / max(dt, 1e-3))))
    y = yet_fn(k)
    t0 = time.perf_counter()
    oracle.ylt(pf, y)
    dt = time.perf_counter() - t0
    lookups = k * EVENTS_PER_TRIAL * N_ELTS
    out = {"value": lookups / dt, "unit": "lookups/s", "cores": oracle.threads(), "kind": "oracle",
           "sample": f"first {k} trials of the paper-scale YET ({k * EVENTS_PER_TRIAL} occurrences x "
                     f"{N_ELTS} ELTs), FP64 C oracle, {dt:.1f} s", "trials": k}
    if single_core:
        k1 = max(calib, k // 16)
        y1 = yet_fn(k1)
        cores = oracle.threads()
        oracle.set_threads(1)
        try:
            t0 = time.perf_counter()
            oracle.ylt(pf, y1)
            dt1 = time.perf_counter() - t0
        finally:
            oracle.set_threads(cores)
        out["single_core"] = {"value": k1 * EVENTS_PER_TRIAL * N_ELTS / dt1, "cores": 1,
                              "sample": f"first {k1} trials, {dt1:.1f} s"}
    return out


def run_reference(args, rank, ws):
    """Reference arm: the FP64 CPU oracle, timed on the host cores, each step a bounded sample."""
    if rank != 0:
        return
    import oracle
    import synth
    pf = synth.paper_scale_portfolio(0)
    base = oracle_sample_rate(pf, lambda k: synth.paper_scale_yet(0, n_trials=k), 2.0,
                              single_core=False)
    k = base["trials"]
    yet = synth.paper_scale_yet(0, n_trials=k)
    for _ in range(args.warmup):
        oracle.ylt(pf, yet)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y = oracle.ylt(pf, yet)
        oracle.risk_metrics(y, RPS, LEVELS)
    dt = (time.perf_counter() - t0) / args.steps
    value = k * EVENTS_PER_TRIAL * N_ELTS / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "lookups/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_trials": k},
            "cpu_baseline": {"value": value, "unit": "lookups/s", "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": f"first {k} trials of the paper-scale YET per step"},
            "e2e": {"value": value, "unit": "lookups/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# Our arm
# ------------------------------------------------------------------------------------------
def run_ours(args, rank, ws, local):
    import torch
    import paper_1606_04473_gb300 as ara
    import synth

    n_trials = args.trials
    pf, yet, ids_h, off_h = make_inputs(seed=rank, n_trials=n_trials, pinned=True)
    g = ara.Portfolio.from_tables(pf)
    off = off_h.cuda()
    ids = ids_h.cuda()
    ylt = torch.empty((1, n_trials), dtype=torch.float64, device="cuda")
    n_events = n_trials * EVENTS_PER_TRIAL
    lookups_per_step = n_events * N_ELTS
    stream = torch.cuda.current_stream()

    # One step: the YLT of the layer and its PML / TVaR, queued stream-ordered; each step's
    # results and device status are copied to pinned host slots without a host wait, so the
    # host queues step k+1 while step k runs (one synchronisation at the end).  The selection
    # runs on a second stream behind an event.  Its blocks, like the stream kernel's, fill an SM's
    # registers and it is cooperative, so it starts once every SM is free: the next step's fold
    # (the first thing its ara_run_ylt queues, right behind the stream kernel) runs first and
    # hides the event's latency, and the selection then runs before that step's stream kernel.
    # The YLT is double-buffered so that the next step's stream kernel does not overwrite the
    # row the selection is reading.
    n_slots = max(args.steps, args.warmup, 3)
    ylts = [ylt, torch.empty_like(ylt)]
    pml_d = [torch.empty((1, len(RPS)), dtype=torch.float64, device="cuda") for _ in range(2)]
    tvar_d = [torch.empty((1, len(LEVELS)), dtype=torch.float64, device="cuda") for _ in range(2)]
    status_d = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in range(2)]
    res_h = torch.zeros((n_slots, len(RPS) + len(LEVELS)), dtype=torch.float64, pin_memory=True)
    status_h = torch.full((n_slots,), -1, dtype=torch.int32, pin_memory=True)
    sel_stream = torch.cuda.Stream()
    ev_run = [torch.cuda.Event() for _ in range(2)]
    ev_sel = [torch.cuda.Event() for _ in range(2)]
    sel_queued = [False, False]

    def step(k):
        b = k % 2
        if sel_queued[b]:                 # the selection two steps back has read ylts[b]
            stream.wait_event(ev_sel[b])
        g.run_ylt(off, ids, out=ylts[b], flags=args.flags)
        ev_run[b].record(stream)
        sel_stream.wait_event(ev_run[b])
        ara.risk_metrics_async(ylts[b], RPS, LEVELS, pml_d[b], tvar_d[b], status_d[b], stream=sel_stream)
        with torch.cuda.stream(sel_stream):
            res_h[k, :len(RPS)].copy_(pml_d[b][0], non_blocking=True)
            res_h[k, len(RPS):].copy_(tvar_d[b][0], non_blocking=True)
            status_h[k:k + 1].copy_(status_d[b], non_blocking=True)
        ev_sel[b].record(sel_stream)
        sel_queued[b] = True

    def join():
        stream.wait_stream(sel_stream)

    for k in range(max(3, args.warmup)):
        step(k)
    join()
    g.check()
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs; no per-launch events, which would cost the
    # step about 1.4 %: kernel durations come from a second, identical run below) ----
    n0 = ara.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    # clocks sampled over the timed steps and their event-timed repeat (not over the end-to-end
    # runs below: nvidia-smi polling every 20 ms slowed the host-memory reads by about 5 %)
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    join()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = (ara.launch_count() - n0)
    ms = e0.elapsed_time(e1) / args.steps
    # the same K steps again with CUDA events around every launch (on the launch stream):
    # per-kernel durations for the breakdown and the roofline
    ara.timing_reset()
    ara.timing_enable(True)
    for k in range(args.steps):
        step(k)
    join()
    torch.cuda.synchronize()
    ara.timing_enable(False)
    clk.__exit__(None, None, None)
    ylt_ms, ylt_n = ara.timing_read(ara.ARA_K_YLT)
    fold_ms, fold_n = ara.timing_read(ara.ARA_K_FOLD)
    sel_ms, sel_n = ara.timing_read(ara.ARA_K_SELECT)
    g.check()
    # every step's results: no device-side timeout, and equal to the synchronous call's
    pml, tvar = ara.risk_metrics(ylt, RPS, LEVELS)
    ref_row = np.concatenate([pml[0], tvar[0]])
    if int(status_h[:args.steps].abs().sum()) != 0 or not np.array_equal(
            res_h[:args.steps].numpy(), np.tile(ref_row, (args.steps, 1))):
        raise RuntimeError("pipelined step results differ from the synchronous risk metrics")
    ms_max = max_over_ranks(ms, ws)
    value = lookups_per_step * ws / (ms_max / 1e3)

    # ---- end to end through the host-memory entry point (H2D + D2H inside the timed region) ----
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 10))
    ylt_h = torch.empty((1, n_trials), dtype=torch.float64, pin_memory=True)
    ids_np, off_np, ylt_np = ids_h.numpy(), off_h.numpy(), ylt_h.numpy()
    def e2e_time(flags):
        for _ in range(2):
            g.run_ylt_host(off_np, ids_np, out=ylt_np, return_periods=RPS, tvar_levels=LEVELS, flags=flags)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            g.run_ylt_host(off_np, ids_np, out=ylt_np, return_periods=RPS, tvar_levels=LEVELS, flags=flags)
        torch.cuda.synchronize()
        t = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)
        barrier(ws)
        return t

    def e2e_breakdown(flags, reps=3):
        """Where one end-to-end call's time goes: per-class times from CUDA events on the
        streams they run on (fold, stream kernel, selection, the library's own copies) and the
        host-timed offset check; the rest (launch, synchronisation and small result copies) is
        the difference to the call's wall time."""
        torch.cuda.synchronize()
        ara.timing_reset()
        ara.timing_enable(True)
        t0 = time.perf_counter()
        for _ in range(reps):
            g.run_ylt_host(off_np, ids_np, out=ylt_np, return_periods=RPS, tvar_levels=LEVELS, flags=flags)
        wall = (time.perf_counter() - t0) / reps * 1e3
        ara.timing_enable(False)
        out = {"wall_ms": round(wall, 3)}
        for name, k in (("fold_ms", ara.ARA_K_FOLD), ("stream_ms", ara.ARA_K_YLT),
                        ("select_ms", ara.ARA_K_SELECT), ("copies_ms", ara.ARA_K_TRANSFER),
                        ("host_offset_check_ms", ara.ARA_K_HOST_CHECK)):
            ms, n = ara.timing_read(k)
            out[name] = round(ms / reps, 3)
        serial = out["fold_ms"] + out["stream_ms"] + out["select_ms"]
        if flags & ara.ARA_RUN_HOST_DIRECT:
            serial += out["copies_ms"]          # only the YLT copy, after the kernels
        out["rest_ms"] = round(wall - serial, 3)
        return out

    e2e_staged = e2e_time(args.flags)
    staged_parts = e2e_breakdown(args.flags)
    try:
        e2e_direct = e2e_time(args.flags | ara.ARA_RUN_HOST_DIRECT)
        direct_parts = e2e_breakdown(args.flags | ara.ARA_RUN_HOST_DIRECT)
    except ara.AraError:
        e2e_direct = float("inf")
        direct_parts = None
    e2e_s = min(e2e_staged, e2e_direct)
    e2e_api = ("ara_run_ylt_host, ARA_RUN_HOST_DIRECT (kernel reads the pinned host YET over the CPU-GPU link)"
               if e2e_direct <= e2e_staged else "ara_run_ylt_host (chunked H2D copies overlapped with kernels)")
    h2d = ids_h.numel() * 4 + off_h.numel() * 8
    d2h = n_trials * 8 + 8 * (len(RPS) + len(LEVELS))

    # ---- roofline of the dominant kernel (the YET stream) ----
    peak, peak_kind = measured_peaks()
    alg_bytes = 4 * n_events + 8 * (n_trials + 1) + 8 * n_trials + 8 * CATALOGUE
    per_launch_ms = ylt_ms / max(ylt_n, 1)
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    prof = ncu_profile_figures()
    tpe = prof.get("dram_bytes_per_event")
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": (tpe * n_events if tpe else None),
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one capture of "
                               "this kernel source at 1e8 occurrences "
                               "(profiles/k_ylt_bulk_paper_scale.txt), scaled per occurrence to "
                               "this launch" if tpe else "no capture of the current kernel source"),
            "l2_hit_rate_pct": prof.get("l2_hit_rate_pct"),
            "gather_sectors_per_occurrence": prof.get("gather_sectors_per_event"),
            "l2_source": "same ncu capture" if prof.get("l2_hit_rate_pct") is not None else None,
            "peak_source": peak_kind, "kernel": stream_kernel_name(args.flags),
            "alg_bytes_per_launch": alg_bytes, "ms_per_launch": round(per_launch_ms, 4),
            "frac_8byte_events": round((alg_bytes + 4 * n_events) / (per_launch_ms / 1e3) / 1e9 / peak, 4),
            "frac_of_nominal_8tbs": round(achieved / 8000.0, 4),
            "frac_basis": "frac: 4 B of event ID per occurrence (timestamps are never read) + "
                          "offsets + YLT + the q table once, over the measured copy bandwidth; "
                          "frac_8byte_events adds 4 B of timestamp per occurrence; "
                          "frac_of_nominal_8tbs divides by 8 TB/s instead"}

    oep_line = None if args.no_oep else measure_oep(g, off, ids, ylt, lookups_per_step)
    layout_line = None if args.no_layouts else measure_layouts(pf, g, off, ids, ylt, n_events)
    g.close()
    del ids, off, ylt
    torch.cuda.empty_cache()
    adjoint_line = None if args.no_adjoint else measure_adjoint(rank)
    batched_line = None if args.no_batched else measure_batched(rank)
    serving_line = None if args.no_serving else measure_serving(rank, args.serving_requests)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample_rate(
            pf, lambda k: synth.YET(yet.offsets[:k + 1], yet.event_ids[:int(yet.offsets[k])]),
            args.cpu_seconds, max_trials=n_trials)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "lookups/s", "n_gpus": ws,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_max,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded SplitMix64 YET, lognormal ELT losses)",
                "config": {"workload": WORKLOAD, "n_trials": n_trials, "events_per_trial": EVENTS_PER_TRIAL,
                           "n_elts": N_ELTS, "catalogue": CATALOGUE, "flags": args.flags,
                           "layout": "folded per-event table + smem hit bitmap",
                           "accumulation": "exact 128-bit fixed-point trial sums, FP64 terms",
                           "l2": f"inputs larger than L2 ({4 * n_events / 1e9:.2g} GB of event IDs "
                                 "per step), no flush",
                           "parallelism": f"replicas x{ws}",
                           "step": "YLT + PML/TVaR queued stream-ordered (ara_run_ylt, then "
                                   "ara_risk_metrics_async on a second stream after an event, YLT "
                                   "double-buffered; the next fold runs right behind the stream "
                                   "kernel, then the cooperative selection before the next stream "
                                   "kernel), each step's results copied to pinned host memory; "
                                   "one host synchronisation after the last step"},
                "lookups_per_step": lookups_per_step,
                "kernel_ms": {"fold_and_coarsen_per_step": round(fold_ms / max(args.steps, 1), 4),
                              "ylt_stream": round(per_launch_ms, 4),
                              "select": round(sel_ms / max(sel_n, 1), 4),
                              "measured": "CUDA events around every launch on its stream, over a "
                                          "second run of the same steps right after the timed one; "
                                          "the fold and the previous step's selection run at the "
                                          "same time on two streams, so their intervals include "
                                          "time they share"},
                "roofline": roof,
                "cpu_baseline": cpu,
                "e2e": {"value": lookups_per_step * ws / e2e_s, "unit": "lookups/s",
                        "ms_per_step": e2e_s * 1e3, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "api": e2e_api,
                        "ms_per_step_staged": e2e_staged * 1e3,
                        "ms_per_step_direct": (e2e_direct * 1e3 if e2e_direct != float("inf") else None),
                        "link_floor_ms": round(h2d / 211e9 * 1e3, 3),
                        "link_floor_basis": "h2d bytes / 211 GB/s, the host-to-device rate measured "
                                            "on this box for copies and for SM loads of host memory",
                        "breakdown_direct": direct_parts, "breakdown_staged": staged_parts},
                "layout_variants": layout_line,
                "occurrences_per_s": n_events * ws / (ms_max / 1e3),
                "metric_note": "logical (occurrence, ELT) pairs, 15 per occurrence; the folded "
                               "path makes at most one table gather per occurrence (the "
                               "occurrences that pass the shared-memory hit filter)",
                "oep": oep_line,
                "adjoint": adjoint_line,
                "batched": batched_line,
                "serving": serving_line,
                "gpu_launches": launches,
                "clocks": dict(clk.summary(), covers="the timed steps and their event-timed "
                               "repeat (nvidia-smi every 20 ms)"),
                "results": {"pml100": float(pml[0, 0]), "pml250": float(pml[0, 1]),
                            "tvar99": float(tvar[0, 0])}}
        print(json.dumps(line), flush=True)


def measure_oep(g, off, ids, ylt, lookups: int, reps: int = 20):
    """Occurrence basis (ARA_RUN_OEP: y_t = the largest net occurrence loss of trial t) on the
    resident paper-scale YET: the same stream with an exact fixed-point max per trial."""
    import torch
    import paper_1606_04473_gb300 as ara
    for _ in range(3):
        g.run_ylt(off, ids, out=ylt, flags=ara.ARA_RUN_OEP)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.run_ylt(off, ids, out=ylt, flags=ara.ARA_RUN_OEP)
    e1.record()
    torch.cuda.synchronize()
    g.check()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": "paper scale, occurrence basis (largest net occurrence loss per trial)",
            "ms_per_run": round(ms, 4), "lookups_per_s": lookups / (ms / 1e3)}


def measure_layouts(pf, g, off, ids, ylt, n_events: int, reps: int = 5):
    """The YET-stream kernel at paper scale under the layouts the ELT lookup can take: the folded
    per-event table behind the shared-memory hit filter (the default), the same table without the
    filter (a gather for every occurrence), and the literal direct-access tables of every ELT
    (dense FP32 [15][catalogue], 15 lookups per occurrence).  Kernel time only (CUDA events
    around each stream launch), results compared with the default's."""
    import torch
    import paper_1606_04473_gb300 as ara

    def kernel_ms(port, flags):
        y = torch.empty_like(ylt)
        port.run_ylt(off, ids, out=y, flags=flags)
        torch.cuda.synchronize()
        ara.timing_reset()
        ara.timing_enable(True)
        for _ in range(reps):
            port.run_ylt(off, ids, out=y, flags=flags)
        torch.cuda.synchronize()
        ara.timing_enable(False)
        port.check()
        ms, n = ara.timing_read(ara.ARA_K_YLT)
        return ms / max(n, 1), y

    base_ms, y0 = kernel_ms(g, 0)
    nf_ms, y1 = kernel_ms(g, ara.ARA_RUN_NO_FILTER)
    dense = ara.Portfolio.from_tables(pf, dense_tables=True)
    pe_ms, y2 = kernel_ms(dense, ara.ARA_RUN_PER_ELT)
    dense.close()
    same = bool(torch.equal(y0, y1) and torch.equal(y0, y2))
    return {"folded_filtered_ms": round(base_ms, 4), "folded_no_filter_ms": round(nf_ms, 4),
            "per_elt_dense_fp32_ms": round(pe_ms, 4),
            "per_elt_lookups_per_s": n_events * N_ELTS / (pe_ms / 1e3),
            "results_identical": same,
            "note": "kernel time of the YET stream only; the folded layouts add a fold of "
                    "the 2M-event catalogue per run (see kernel_ms)"}


def measure_adjoint(rank: int, reps: int = 5):
    """Adjoint/forward time ratio on the adjoint workload: 16 layers x 15 ELTs (2M catalogue),
    2e5 trials x 1000 events.  Forward = YLT of all layers (recording regimes) + mean and
    TVaR99; adjoint = gradients of both w.r.t. every term and ELT loss."""
    import torch
    import paper_1606_04473_gb300 as ara
    import synth
    pf = synth.adjoint_portfolio(0)
    yet = synth.adjoint_yet(rank, n_trials=200_000)
    g = ara.Portfolio.from_tables(pf)
    off = torch.from_numpy(yet.offsets).cuda()
    ids = torch.from_numpy(yet.event_ids).cuda()
    reg = torch.empty((pf.n_layers, yet.n_trials), dtype=torch.uint8, device="cuda")
    y = torch.empty((pf.n_layers, yet.n_trials), dtype=torch.float64, device="cuda")

    def fwd():
        g.run_ylt(off, ids, out=y, regimes=reg)
        return ara.risk_metrics(y, [], [0.99], want_mean=True)

    def adj():
        return g.adjoint(off, ids, y, reg, 0.99)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    f_ms = timed(fwd)
    a_ms = timed(adj)
    g.check()
    # the same adjoint over an event-major index of the YET (built once per YET)
    g.yet_index(off, ids).close()                 # first build: one-time set-up costs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    yx = g.yet_index(off, ids)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3

    def adjx():
        return g.adjoint(None, None, y, reg, 0.99, index=yx)

    ax_ms = timed(adjx)
    ra, rb = adj(), adjx()
    same = all(torch.equal(ra[k], rb[k]) for k in ("elt", "layer", "loss"))
    yx.close()
    out = {"workload": "16 layers x 15 ELTs (2M catalogue, 20k events each), 2e5 trials x 1000 events",
           "forward_ms": round(f_ms, 3), "adjoint_ms": round(a_ms, 3), "ratio": round(a_ms / f_ms, 3),
           "indexed": {"adjoint_ms": round(ax_ms, 3), "ratio": round(ax_ms / f_ms, 3),
                       "index_build_ms": round(build_ms, 3),
                       "equal_to_trial_major": bool(same),
                       "what": "ara_adjoint_indexed over an event-major index of the same YET "
                               "(ara_yet_index_create, once per YET, not in adjoint_ms)"},
           "objectives": "mean year loss and TVaR99 per layer; gradients w.r.t. every retention, "
                         "limit and ELT loss",
           "check": check_adjoint(pf, yet, g, off, ids, y, reg)}
    g.close()
    return out


def check_adjoint(pf, yet, g, off, ids, y, reg, sel=(0, 1), slice_trials: int = 4000):
    """The timed adjoint against the FP64 oracle's chain rule (rtol 1e-4): the TVaR99 gradients
    of two layers over the whole YET, read from the timed computation's own output (the oracle
    follows only the top trials back), and both objectives of the same layers on the first
    slice_trials trials of the same device YET (the mean objective needs every trial)."""
    import oracle
    import synth
    sel = list(sel)
    sub = pf.with_terms(pf.terms_dict())
    sub.layer_elts = [pf.layer_elts[i] for i in sel]
    for name in ["occ_ret", "occ_lim", "agg_ret", "agg_lim"]:
        setattr(sub, name, np.asarray(getattr(pf, name))[sel])
    k_slots = sum(len(pf.layer_elts[i]) for i in sel)
    m_recs = sum(pf.elt_ids[j].size for i in sel for j in pf.layer_elts[i])
    worst = 0.0

    def rel(got, want):
        got, want = np.asarray(got), np.asarray(want)
        scale = max(1.0, float(np.abs(want).max())) if want.size else 1.0
        return float(np.max(np.abs(got - want) / (1e-4 * np.abs(want) + 1e-12 * scale))) if want.size else 0.0

    t0 = time.perf_counter()
    full = g.adjoint(off, ids, y, reg, 0.99)
    ref = oracle.adjoint(sub, yet, "tvar", 0.99)
    worst = max(worst, rel(full["elt"][1][:k_slots].cpu().numpy(), ref["elt"]),
                rel(full["layer"][1][:len(sel)].cpu().numpy(), ref["layer"]),
                rel(full["loss"][1][:m_recs].cpu().numpy(), ref["loss"]))
    import torch
    n = slice_trials
    ys = synth.YET(yet.offsets[:n + 1], yet.event_ids[:int(yet.offsets[n])])
    reg_s = torch.empty((len(sel), n), dtype=torch.uint8, device="cuda")
    y_s = g.run_ylt(off[:n + 1], ids, layers=sel, regimes=reg_s)
    part = g.adjoint(off[:n + 1], ids, y_s, reg_s, 0.99, layers=sel)
    g.check()
    for obj, name in ((0, "mean"), (1, "tvar")):
        r = oracle.adjoint(sub, ys, name, 0.99)
        worst = max(worst, rel(part["elt"][obj].cpu().numpy(), r["elt"]),
                    rel(part["layer"][obj].cpu().numpy(), r["layer"]),
                    rel(part["loss"][obj].cpu().numpy(), r["loss"]))
    return {"ok": bool(worst <= 1.0), "worst_error_over_tolerance": round(worst, 6),
            "what": f"TVaR99 gradients of layers {sel} over all trials; mean and TVaR99 "
                    f"gradients of the same layers on the first {n} trials; rtol 1e-4 against "
                    "the FP64 chain-rule oracle", "seconds": round(time.perf_counter() - t0, 1)}


def measure_batched(rank: int, reps: int = 5):
    """Batched portfolio: 64 layers of U{3..30} ELTs from a pool of 200 (2M catalogue), YET of
    2e5 trials with Poisson counts of per-trial mean U[200, 2000]; one autotuned plan (one CUDA
    graph: folds, event-major table, one persistent stream kernel) against 64 sequential
    single-layer ara_run_ylt launches of the same layers."""
    import torch
    import paper_1606_04473_gb300 as ara
    import synth
    pf = synth.batched_portfolio(0)
    yet = synth.batched_yet(rank, n_trials=200_000)
    g = ara.Portfolio.from_tables(pf)
    off = torch.from_numpy(yet.offsets).cuda()
    ids = torch.from_numpy(yet.event_ids).cuda()
    y_seq = torch.empty((pf.n_layers, yet.n_trials), dtype=torch.float64, device="cuda")
    lookups = int(yet.n_events) * sum(len(l) for l in pf.layer_elts)

    def seq():
        for l in range(pf.n_layers):
            g.run_ylt(off, ids, layers=[l], out=y_seq[l:l + 1])

    t_plan0 = time.perf_counter()
    plan = ara.BatchedPlan(g, off, ids, autotune=True)
    t_plan = time.perf_counter() - t_plan0

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    seq_ms = timed(seq)
    plan_ms = timed(plan.launch)
    g.check()
    identical = bool(torch.equal(plan.out, y_seq))
    info = plan.info()
    # Roofline of the stream kernel (its autotuned time, CUDA events around the launch): the bytes
    # it gathers per pass are every occurrence's ID and row descriptor and every table entry of
    # its row, plus the trial offsets and the YLT writes.
    rows, n_entries = plan.table()
    lens = (rows >> 32) & 0xFF
    freq = torch.bincount(ids.long(), minlength=pf.catalogue)
    walked = int((lens * freq).sum().item())
    n_occ = int(yet.n_events)
    alg = 4 * n_occ + 8 * n_occ + 8 * walked + 8 * (yet.n_trials + 1) + 8 * pf.n_layers * yet.n_trials
    peak, peak_kind = measured_peaks()
    stream_ms = info["tuned_ms"]
    roof = {"bound": "l1 / l2 gathers and shared-memory atomics (not hbm)",
            "alg_bytes_per_launch": alg, "entries_walked": walked, "table_entries": n_entries,
            "table_mb": round(8 * n_entries / 1e6, 1), "stream_ms": round(stream_ms, 4),
            "achieved_gbs": round(alg / (stream_ms / 1e3) / 1e9, 1), "peak_gbs": peak,
            "frac": round(alg / (stream_ms / 1e3) / 1e9 / peak, 4), "peak_source": peak_kind,
            "bytes": "4 B ID + 8 B row descriptor per occurrence, 8 B per table entry walked, "
                     "offsets, 8 B YLT per (layer, trial); gathered bytes, not DRAM traffic"}
    plan.close()
    # The same 64 layers as two plans of 32, each table about half the size, run back to back.
    plans = [ara.BatchedPlan(g, off, ids, layers=list(range(h * 32, h * 32 + 32)), autotune=True)
             for h in range(2)]
    split_ms = timed(lambda: [p.launch() for p in plans])
    split_tables = [round(8 * p.table()[1] / 1e6, 1) for p in plans]
    for p in plans:
        p.close()
    out = {"workload": "64 layers x U{3..30} ELTs from a pool of 200 (2M catalogue), 2e5 trials x "
                       "Poisson(U[200,2000]) events",
           "events": n_occ, "lookups_per_pass": lookups,
           "sequential_ms": round(seq_ms, 3), "batched_ms": round(plan_ms, 3),
           "speedup": round(seq_ms / plan_ms, 3),
           "batched_lookups_per_s": lookups / (plan_ms / 1e3),
           "identical_to_sequential": identical, "schedule": info,
           "plan_build_s": round(t_plan, 3), "roofline": roof,
           "split_two_plans_of_32_layers_ms": round(split_ms, 3),
           "split_table_mb": split_tables}
    g.close()
    return out


def measure_serving(rank: int, n_requests: int = 200, workers: int = 1, saturating_rate: float = 1000.0):
    """Serving: a seeded Poisson stream of risk queries from 32 tenants over a resident pool of
    500 ELTs and a resident YET of 1e6 trials x Poisson(1000) events (1-32 layers of 5-20 ELTs
    each, slices of 1e4-1e6 trials, 20 % with the adjoint), served by the native server:
    continuous admission by device memory, queued requests with overlapping slices merged into
    one YET pass (up to 4); by default one worker (a second worker, whose host work and small
    kernels overlap the first's passes, is reported beside it).
    Capacity is measured at a saturating offered load (the trace's arrivals at saturating_rate
    per second, well above what any mode serves, so every makespan is set by the server and not
    by the last arrival), and compared with the same queries run one at a time (one worker, no
    merging; the batched path for requests of 4 or more layers, as in the served mode) and with
    sequential plain runs (one at a time, every layer by the single-layer path).  The server's
    adjoint requests read an event-major index of the resident YET, built when each server is set
    up, in every arm but the sequential plain runs and one served arm without it.  Latencies are
    then taken at 2x and 0.5x of the served mode's measured capacity.  Results must be identical
    in every mode."""
    import threading
    import torch
    import paper_1606_04473_gb300 as ara
    import synth
    pool_t = synth.serving_pool(0)
    yet = synth.serving_yet(rank)
    pool = ara.Portfolio.from_tables(pool_t)
    off = torch.from_numpy(yet.offsets).cuda()
    ev = torch.from_numpy(yet.event_ids).cuda()
    del yet.event_ids
    base_rate = 200.0
    trace = synth.serving_trace(pool_t, off.numel() - 1, n_requests, base_rate, seed=rank)
    offs = yet.offsets
    lookups = [sum(len(l) for l in q["layer_elts"]) * int(offs[q["trials"][1]] - offs[q["trials"][0]])
               for q in trace]

    def query_args(q, plain):
        batched = len(q["layer_elts"]) >= 4 and not plain
        return dict(layer_elts=q["layer_elts"], occ_ret=q["occ_ret"], occ_lim=q["occ_lim"],
                    agg_ret=q["agg_ret"], agg_lim=q["agg_lim"], trials=q["trials"],
                    return_periods=[100.0, 250.0], tvar_levels=[0.99], want_mean=True,
                    want_adjoint=q["want_adjoint"], adjoint_level=0.99,
                    flags=ara.ARA_RUN_BATCHED if batched else 0, tenant=q["tenant"])

    index_ms = []

    def serve(max_concurrent, merge, plain=False, stretch=1.0, index=True):
        srv = ara.Server(pool, off, ev, max_concurrent=max_concurrent, max_merge=merge)
        if index:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            srv.set_adjoint_index(True)
            index_ms.append((time.perf_counter() - t0) * 1e3)
        srv.wait(srv.submit(**dict(query_args(trace[0], plain), trials=(0, 1000))))
        c0 = srv.counters()
        tickets = [None] * len(trace)
        t_start = time.perf_counter()

        def feeder():
            for k, q in enumerate(trace):
                d = q["arrival"] * stretch - (time.perf_counter() - t_start)
                if d > 0:
                    time.sleep(d)
                tickets[k] = srv.submit(**query_args(q, plain))

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        res = [srv.wait(t) for t in tickets]
        makespan = time.perf_counter() - t_start
        stats, cnt = srv.stats(), srv.counters()
        srv.close()
        lat = np.array([r["latency_s"] for r in res]) * 1e3
        arm = {"workers": max_concurrent, "max_merge": merge,
               "p50_ms": round(float(np.percentile(lat, 50)), 2),
               "p99_ms": round(float(np.percentile(lat, 99)), 2), "makespan_s": round(makespan, 3),
               "lookups_per_s": float(sum(lookups)) / makespan,
               "requests_per_s": len(trace) / makespan, "peak_running": stats["peak_running"],
               "passes": cnt["passes"] - c0["passes"],
               "merged_requests": cnt["merged_requests"] - c0["merged_requests"],
               "head_passed": cnt["head_passed"] - c0["head_passed"],
               "indexed_adjoints": cnt["indexed_adjoints"] - c0["indexed_adjoints"]}
        return res, arm

    sat = base_rate / saturating_rate
    res_s, served = serve(workers, 4, stretch=sat)
    res_2, served_2 = serve(2, 4, stretch=sat)
    res_1, one = serve(1, 1, stretch=sat)
    res_p, plain = serve(1, 1, plain=True, stretch=sat, index=False)
    res_n, served_noidx = serve(workers, 4, stretch=sat, index=False)
    capacity = served["requests_per_s"]
    loads = {}
    others = [res_s, res_2, res_p, res_n]
    for name, factor in (("2x_capacity", 2.0), ("0.5x_capacity", 0.5)):
        rate = factor * capacity
        r_s, a_s = serve(workers, 4, stretch=base_rate / rate)
        r_1, a_1 = serve(1, 1, stretch=base_rate / rate)
        others += [r_s, r_1]
        loads[name] = {"offered_requests_per_s": round(rate, 1), "served": a_s, "one_at_a_time": a_1}
    keys = ("pml", "tvar", "mean", "grad_layer")
    same = all(all((a[k] is None and b[k] is None) or np.array_equal(a[k], b[k]) for k in keys)
               for other in others for a, b in zip(other, res_1))
    out = {"workload": f"{n_requests} requests, Poisson arrivals, 32 tenants; 1-32 layers x 5-20 ELTs "
                       "of a 500-ELT pool; slices of 1e4-1e6 trials of a 1e6 x Poisson(1000) YET; "
                       "20% adjoint",
           "offered_load_saturating": f"{saturating_rate:g} requests/s (above every mode's capacity: "
                                      "makespans are set by the server)",
           "served": served, "served_2_workers": served_2, "one_at_a_time": one,
           "sequential_plain": plain, "served_without_yet_index": served_noidx,
           "yet_index": {"build_ms": round(float(np.median(index_ms)), 2) if index_ms else None,
                         "what": "event-major index of the resident YET, built when the server "
                                 "is set up (ara_server_set_adjoint_index); adjoint requests "
                                 "whose slice covers at least half of the index blocks it "
                                 "touches read it. Every arm but sequential_plain and "
                                 "served_without_yet_index uses it"},
           "capacity_requests_per_s": {"served": round(capacity, 1),
                                       "one_at_a_time": round(one["requests_per_s"], 1),
                                       "sequential_plain": round(plain["requests_per_s"], 1)},
           "latency_at_load": loads,
           "throughput_gain": round(one["makespan_s"] / served["makespan_s"], 3),
           "throughput_gain_vs_sequential_plain": round(plain["makespan_s"] / served["makespan_s"], 3),
           "results_identical": bool(same), "total_lookups": float(sum(lookups))}
    pool.close()
    return out


def main():
    args = parse()
    rank, ws, local = dist_setup()
    try:
        if args.impl == "reference":
            run_reference(args, rank, ws)
        else:
            run_ours(args, rank, ws, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
