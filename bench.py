"""Benchmark of the rDDMC walk: packet transitions/s (and escaped packets/s) on
the tau0 = 1e7 slab (256 cells x 512 bins over x in [-60, 60], T = 1e4 K,
1e7 packets, FP32/integer walk, FP64 leakage precompute, uint64 escape
histogram).

A step is one pass of the whole walk over the resident packet population: one
persistent-kernel launch that resumes every one of the 1e7 packets (or starts
it at the source), advances it by `--slice` transitions or until it escapes,
tallies escapes and saves its state.  A full run to escape needs ~3e8
transitions per packet (3e15 in total), so the job is timed slice by slice.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
For N > 1 launch with torchrun; each rank walks its own packets under its own
Philox key (seed offset by rank: weak scaling, no data-path collective).  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same workload on the host cores.
"""
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

from paper_1709_10187_gb300 import workloads as W  # noqa: E402

METRIC = "packet transitions/s (rDDMC walk, tau0=1e7 slab)"
UNIT = "transitions/s"
# Gather bytes per transition of the slab walk: the 8-byte fast head of the
# state's row (a frequency move, ~all transitions at this resolution); the
# generic step's 16-byte row is read on the rare other outcomes.
GATHER_BYTES = 8
PEAK_SM_MHZ = 2070.0  # maximum SM clock of a GB300
N_SM = 152
SMSP_PER_SM = 4       # warp schedulers per SM, one instruction issued per cycle each


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _profile_walk():
    """Counters of one ncu capture of the bench's walk launch (committed under
    profiles/): DRAM bytes and issued instructions per launch, with the kernel
    source hash and launch configuration they were taken on."""
    p = os.path.join(ROOT, "profiles", "walk_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_sample(seconds_target=12.0, slice_=4096):
    """Time the FP64 oracle on a bounded sample of the workload on the host cores."""
    from oracle import coracle as C
    w = W.C2
    g = C.Grid(w)
    tb = g.table()
    cores = os.cpu_count() or 1
    npk = max(cores * 64, 2048)
    t0 = time.perf_counter()
    C.walk_slice(g, tb, w.seed, 0, npk, slice_, nthreads=cores)
    dt = time.perf_counter() - t0
    npk2 = int(npk * max(1.0, seconds_target / max(dt, 1e-3)))
    t0 = time.perf_counter()
    r = C.walk_slice(g, tb, w.seed, npk, npk2, slice_, nthreads=cores)
    dt = time.perf_counter() - t0
    return dict(value=r["steps"] / dt, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{npk2} packets of the tau0=1e7 slab x {slice_} transitions each from the source "
                       f"({r['steps']} transitions, {dt:.1f} s, FP64 C oracle, {cores} threads)"), dt


def _cpu_completed():
    """The FP64 oracle on completed packet subsets (every packet walked to
    escape), on all host cores: C1 and the paper's two a tau0 = 1e9 slabs in
    full, C2 and C3 on subsets.  Transitions/s and escaped packets/s, in total
    and per core.  The batched instances are left out: their packet lengths
    span five decades, so no bounded subset represents them."""
    from oracle import coracle as C
    cores = os.cpu_count() or 1
    out = {"cores": cores, "kind": "oracle"}
    for w, npk in ((W.C1, W.C1.packets), (W.P2, W.P2.packets), (W.P1, W.P1.packets), (W.C3, 1000), (W.C2, 100)):
        g = C.Grid(w)
        tb = g.table()
        t0 = time.perf_counter()
        r = C.walk(g, tb, w.seed, 0, npk, nthreads=cores)
        dt = time.perf_counter() - t0
        out[w.name] = {"packets": npk, "s": dt, "escaped": int(r["escaped"]), "transitions": int(r["steps"]),
                       "transitions_per_s": r["steps"] / dt, "transitions_per_s_per_core": r["steps"] / dt / cores,
                       "escaped_per_s": r["escaped"] / dt}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import coracle as C
    w = W.C2
    g = C.Grid(w)
    tb = g.table()
    cores = os.cpu_count() or 1
    npk = cores * 2048
    slice_ = args.slice
    for i in range(args.warmup):
        C.walk_slice(g, tb, w.seed, i * npk, npk, slice_, nthreads=cores)
    tot, t_all = 0, 0.0
    for i in range(args.steps):
        t0 = time.perf_counter()
        r = C.walk_slice(g, tb, w.seed, (args.warmup + i) * npk, npk, slice_, nthreads=cores)
        t_all += time.perf_counter() - t0
        tot += r["steps"]
    v = tot / t_all
    sample = f"{npk} packets x {slice_} transitions per step from the source (FP64 C oracle, {cores} threads)"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "packets_per_step": npk, "slice_transitions": slice_},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rank_seed(seed: int, rank: int, packets_per_rank: int) -> int:
    """Philox key of a rank's packets: every rank walks its own packets under
    its own key (weak scaling; no data-path exchange)."""
    return seed + rank * packets_per_rank


def combine_ranks(dist, device, tsec, trans, escaped, e2e_dt, e2e_trans):
    """Whole-job figures from per-rank ones: the slowest rank's times, the sum of
    the work (transitions, escapes) over all ranks."""
    if not dist:
        return tsec, float(trans), float(escaped), e2e_dt, float(e2e_trans)
    import torch
    t = torch.tensor([tsec, float(trans), float(escaped), e2e_dt, float(e2e_trans)], device=device,
                     dtype=torch.float64)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1]), float(t[2]), float(tmax[3]), float(t[4])


def run_native(args, rank, world, local_rank):
    import torch
    from paper_1709_10187_gb300 import build as B
    from paper_1709_10187_gb300 import rddmc as R

    B.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = W.C2
    npk = w.packets
    seed = w.seed
    key = rank_seed(seed, rank, npk)
    slice_ = args.slice
    stream = torch.cuda.Stream(dev)
    sched = dict(ctas_per_sm=args.ctas_per_sm, threads_per_cta=args.threads, chunk=args.chunk,
                 table_in_smem=args.table_in_smem)

    with torch.cuda.stream(stream):
        prob = R.Problem(w, device=dev)
        prob.ensure_state(npk)
        prob.reset()
        s = stream.cuda_stream

        def launch(resume):
            o = R.RunOpts(key, npk, 0, slice_, resume, sched["ctas_per_sm"], sched["threads_per_cta"],
                          sched["chunk"], sched["table_in_smem"], 0)
            R.launch_packets(prob.grid, prob.table.data_ptr(), o, prob.state.data_ptr(), prob.state.numel(),
                             prob.tally.data_ptr(), prob.tally.numel() * 8, s)

        for i in range(args.warmup):
            launch(1 if i else 0)
        before = prob.read()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clocks = ClockSampler(local_rank)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks.start()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            launch(1 if (args.warmup or i) else 0)
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        if dist:
            dist.barrier()
        elapsed_ms = t_start.elapsed_time(t_end)
        launch_ms = [a.elapsed_time(b) for a, b in ev]
        after = prob.read()
        trans = after["steps"] - before["steps"]
        escaped = after["escaped"] - before["escaped"]

        # e2e through the public API: per step the table inputs go host -> device
        # (rddmc_precompute_leakage), the slice runs, and the tallies come back
        # to the host (rddmc_read_tallies, synchronising).
        e2e_steps = max(1, min(args.steps, 5))
        sz = R.grid_sizes(prob.grid, 1)
        h2d = int(sz.table_bytes - prob.J * sz.row_bytes * sz.n_class)
        t0 = time.perf_counter()
        e2e_trans = 0
        for i in range(e2e_steps):
            R.precompute_leakage(prob.grid, prob.params, prob.table.data_ptr(), prob.table.numel(), s)
            b0 = after["steps"] if i == 0 else tl["steps"]
            launch(1)
            tl = prob.read()
            e2e_trans += tl["steps"] - b0
        e2e_dt = time.perf_counter() - t0
        d2h = (22 + prob.J + 2) * 8

    tsec = elapsed_ms / 1e3
    tsec_max, trans_tot, esc_tot, e2e_dt_max, e2e_tot = combine_ranks(
        dist, dev, tsec, trans, escaped, e2e_dt, e2e_trans)
    if rank != 0:
        return
    value = trans_tot / tsec_max
    peaks, peak_kind = _peaks()
    mean_launch_s = float(np.mean(launch_ms)) / 1e3
    trans_per_launch = trans / args.steps
    # issue-slot roofline: issued instructions per transition from the committed
    # ncu capture of this launch (smsp__inst_executed.sum over the launch's
    # transitions), valid while the kernel source and configuration match it
    prof = _profile_walk()
    current = bool(prof and prof.get("kernel_hash") == _kernel_hash() and prof.get("packets") == npk
                   and prof.get("slice_transitions") == slice_)
    traffic = prof["dram_bytes_per_launch"] if current else None
    inst = prof.get("warp_inst_per_transition") if current else None
    issue_peak = N_SM * SMSP_PER_SM * PEAK_SM_MHZ * 1e6 * 32 / 1e12  # lane-instructions, T/s
    achieved = inst * 32 * trans_per_launch / mean_launch_s / 1e12 if inst else None
    roof = {"bound": "alu", "achieved": achieved, "peak": issue_peak, "unit": "T lane-instr/s",
            "frac": achieved / issue_peak if achieved else None, "traffic": traffic,
            "note": (f"issued instructions: {inst * 32:.2f} lane-instructions per transition (ncu "
                     f"smsp__inst_executed, profiles/walk_kernel_traffic.json); peak = {N_SM} SMs x "
                     f"{SMSP_PER_SM} schedulers x 1 warp-instruction/cycle x {PEAK_SM_MHZ:.0f} MHz")
            if inst else "no ncu capture of the current walk kernel: issue fraction not stated"}
    if world == 1 and not args.no_gather:
        with torch.cuda.stream(stream):
            gp = _gather_peaks(R, torch)
        l1 = gp["l1_8B_32KiB"]
        gather_gbs = GATHER_BYTES * trans_per_launch / mean_launch_s / 1e9
        roof["gather"] = {"achieved": gather_gbs, "peak": l1["GB_per_s"], "unit": "GB/s",
                          "frac": gather_gbs / l1["GB_per_s"],
                          "note": f"{GATHER_BYTES}-byte fast heads per transition against the measured random "
                                  "dependent-gather rate of 8-byte rows from a 32 KiB table through L1 (the "
                                  "C2 table's footprint; rddmc_gather_probe, best of two occupancies)",
                          "probe": gp}
        roof["gather_frac"] = roof["gather"]["frac"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "packets": npk, "slice_transitions": slice_, "cells": w.n[0],
                   "bins": w.J, "tau0": w.tau0, "T": w.T, "mode": "ddmc", "layout": "dedup",
                   "l2": "inputs larger than L2: 1e7-packet state (250 MB) streamed every step; the 24 KiB "
                         "leakage table stays L1/L2-resident by design",
                   "schedule": sched},
        "escaped_packets_per_s": None,
        "escaped_in_timed_region_per_s": esc_tot / tsec_max,
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": args.steps,
        "e2e": {"value": e2e_tot / e2e_dt_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "peaks_source": peak_kind,
    }
    if world == 1 and not args.no_complete:
        # escaped packets/s at tau0 = 1e7: a 1e5-packet subset of the workload
        # walked to escape (each packet ~3e8 transitions, the slowest ~3e9)
        with torch.cuda.stream(stream):
            comp = _complete_sliced(R, torch, w, 100_000)
        line["escaped_packets_per_s"] = comp["escaped_per_s"]
        line["completed_subset"] = comp
    if world == 1 and not args.no_extras:
        with torch.cuda.stream(stream):
            line["extras"] = _extras(R, torch)
    if world == 1 and not args.no_cpu_baseline:
        cb, _ = _cpu_sample()
        if args.cpu_baseline_completed:
            cb["completed"] = _cpu_completed()
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- extras
# Measured after the timed region, on one GPU: the other workloads of the
# method and the learned proposal against the plain walk.  Each is timed with
# CUDA events or a device synchronisation on both sides.

def _gather_peaks(R, torch, threads=256):
    """Random dependent-gather rates (rddmc_gather_probe) at the table
    footprints the walks use: 32 KiB through L1 (the C2 slab table) and in
    shared memory, 2 MiB (served by L2), 1 GiB (served by HBM); 8- and 16-byte
    rows.  Each rate is the better of 4 CTAs/SM (the walk's occupancy) and as
    many as fit, timed with CUDA events on the current stream after one
    untimed launch."""
    cases = [("l1_8B_32KiB", 32 << 10, 8, False, 16384), ("l1_16B_32KiB", 32 << 10, 16, False, 16384),
             ("smem_8B_32KiB", 32 << 10, 8, True, 16384), ("l2_8B_2MiB", 2 << 20, 8, False, 4096),
             ("l2_16B_2MiB", 2 << 20, 16, False, 4096), ("hbm_8B_1GiB", 1 << 30, 8, False, 1024),
             ("hbm_16B_1GiB", 1 << 30, 16, False, 1024)]
    st = torch.cuda.current_stream().cuda_stream
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = {}
    buf = None
    for name, nbytes, rb, smem, chain in cases:
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        best = None
        for i, ctas in enumerate((4, 0)):
            R.gather_probe(buf.data_ptr(), nbytes, rb, smem, chain, ctas, threads, 7, i == 0, sink.data_ptr(), st)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            n = R.gather_probe(buf.data_ptr(), nbytes, rb, smem, chain, ctas, threads, 8, False, sink.data_ptr(), st)
            a1.record()
            torch.cuda.synchronize()
            rate = n / (a0.elapsed_time(a1) / 1e3)
            if best is None or rate > best["gathers_per_s"]:
                best = {"gathers_per_s": rate, "GB_per_s": rate * rb / 1e9, "ctas_per_sm": ctas or "max"}
        out[name] = best
    del buf
    return out


def _complete_sliced(R, torch, w, npk, slice_=1 << 24):
    """npk packets of the workload walked to escape in step slices of slice_
    transitions (every launch short), timed with CUDA events from the first
    launch to the last packet's escape: escaped packets/s and transitions/s
    of the completed run, and the transitions per packet."""
    prob = R.Problem(w)
    prob.ensure_state(npk)
    prob.run(min(npk, 2000), w.seed + 1, steps_per_launch=slice_)  # warm-up
    prob.reset()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record()
    n = 0
    while True:
        prob.launch(npk, w.seed, steps_per_launch=slice_, resume=1 if n else 0)
        n += 1
        t = prob.read()
        if t["escaped"] + t["aborted"] == npk:
            break
    a1.record()
    torch.cuda.synchronize()
    dt = a0.elapsed_time(a1) / 1e3
    prob.close()
    return {"workload": w.name, "packets": npk, "s": dt, "launches": n, "slice_transitions": slice_,
            "escaped": t["escaped"], "aborted": t["aborted"], "escaped_per_s": t["escaped"] / dt,
            "transitions_per_s": t["steps"] / dt, "transitions_per_packet": t["steps"] / npk}


def _sliced_rate(R, torch, prob, npk, seed, slice_, launches=5, warm=2):
    """Transitions/s (and MC events/s) of time-sliced launches over npk packets."""
    s = prob.stream()
    prob.ensure_state(npk)
    prob.reset()
    for i in range(warm):
        prob.launch(npk, seed, steps_per_launch=slice_, resume=1 if i else 0)
    b = prob.read()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record(torch.cuda.current_stream())
    for i in range(launches):
        prob.launch(npk, seed, steps_per_launch=slice_, resume=1)
    a1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    dt = a0.elapsed_time(a1) / 1e3
    e = prob.read()
    return {"transitions_per_s": (e["steps"] - b["steps"]) / dt,
            "mc_events_per_s": (e["mc_events"] - b["mc_events"]) / dt,
            "escaped_per_s": (e["escaped"] - b["escaped"]) / dt, "packets": npk, "slice": slice_,
            "launches": launches}


def _grouped_rate(R, torch, npk=1_000_000, slice_=4096):
    """The C2 hybrid walk with frequency-grouped MC in thin states (Sec. 5.3):
    the eq. R_discrete thresholds (512 x 511, FP64, timed) and the rates of the
    sliced walk, beside the same walk with the continuous MC."""
    prob = R.Problem(W.C2, mode=R.MODE_HYBRID)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record(torch.cuda.current_stream())
    red = prob.redistribution(3)
    a1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    t_pre = a0.elapsed_time(a1) / 1e3
    s = prob.stream()
    prob.ensure_state(npk)
    prob.reset()
    for i in range(2):
        prob.launch(npk, W.C2.seed, steps_per_launch=slice_, resume=1 if i else 0, redist=red)
    b = prob.read()
    torch.cuda.synchronize()
    a0.record(torch.cuda.current_stream())
    for i in range(5):
        prob.launch(npk, W.C2.seed, steps_per_launch=slice_, resume=1, redist=red)
    a1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    dt = a0.elapsed_time(a1) / 1e3
    e = prob.read()
    del s
    return {"redistribution_precompute_s": t_pre, "transitions_per_s": (e["steps"] - b["steps"]) / dt,
            "mc_events_per_s": (e["mc_events"] - b["mc_events"]) / dt, "packets": npk, "slice": slice_,
            "launches": 5}


def _complete(R, torch, w, npk):
    """A run to completion: escaped packets/s over the wall time from launch to
    the last packet's escape (CUDA events around one launch)."""
    prob = R.Problem(w)
    prob.run(min(npk, 2000), w.seed + 1)  # warm-up
    prob.reset()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record(torch.cuda.current_stream())
    prob.launch(npk, w.seed)
    a1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    dt = a0.elapsed_time(a1) / 1e3
    t = prob.read()
    return {"workload": w.name, "packets": npk, "s": dt, "escaped": t["escaped"], "aborted": t["aborted"],
            "escaped_per_s": t["escaped"] / dt, "transitions_per_s": t["steps"] / dt,
            "transitions_per_packet": t["steps"] / npk}


def _batched(R, torch, packet_scale=0.01, max_steps=0, trial_packets=600_000):
    """The batched workload: 512 slab/sphere instances in one persistent launch,
    schedule picked by the autotuner, replayed from a captured CUDA graph.
    max_steps = 0: no watchdog, every packet is walked to escape.  The
    autotuner's trial takes a GPU-filling share of every instance's packets
    (about trial_packets in all), each for at most 65536 transitions: the
    schedules' throughput on the run's own instances."""
    ws = W.batched_instances(512, packet_scale=packet_scale)
    npk = [w.packets for w in ws]
    t0 = time.perf_counter()
    probs = [R.Problem(w) for w in ws]
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    b = R.Batch(probs, npk, trial_fraction=min(1.0, trial_packets / float(sum(npk))))
    base = R.RunOpts(0xBA7C4, 0, max_steps, 0, 0, 0, 0, 0, 0, 0)
    t0 = time.perf_counter()
    best, trial_rate = b.autotune(base)
    t_tune = time.perf_counter() - t0
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ge = b.graph(best)
        try:
            b.tally.zero_()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record(side)
            b.graph_launch(ge)
            a1.record(side)
            torch.cuda.synchronize()
            dt = a0.elapsed_time(a1) / 1e3
            tot = {"steps": 0, "escaped": 0, "aborted": 0, "emitted": 0}
            for i in range(len(ws)):
                t = b.read(i)
                for k in tot:
                    tot[k] += t[k]
        finally:
            R.Batch.graph_destroy(ge)
    torch.cuda.current_stream().wait_stream(side)
    return {"instances": len(ws), "packets": int(sum(npk)), "packet_scale": packet_scale, "max_steps": max_steps,
            "transitions_per_s": tot["steps"] / dt, "escaped_per_s": tot["escaped"] / dt,
            "escaped": tot["escaped"], "aborted": tot["aborted"], "transitions": tot["steps"], "ms": dt * 1e3,
            "schedule": {"threads_per_cta": best.threads_per_cta, "ctas_per_sm": best.ctas_per_sm,
                         "chunk": best.chunk},
            "autotune_trial_transitions_per_s": trial_rate, "autotune_s": t_tune, "setup_s": t_setup}


def _l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a / a.sum() - b / b.sum()).sum())


def _arms(torch, learned_run, plain_run, npk, runs, n_ref, seed0):
    """`runs` independent runs of npk packets per arm (learned_run(n, seed) and
    plain_run(n, seed) return the walk's tallies), timed with a device
    synchronisation on both sides, and an independent plain reference of n_ref
    packets from its own seeds."""
    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    learned_run(2000, seed0 - 1)  # warm-up
    plain_run(2000, seed0 - 1)
    runs_l, runs_p, stats = [], [], {"learned_transitions": 0, "learned_proposals": 0, "learned_launches": 0,
                                     "plain_transitions": 0, "aborted": 0}
    for i in range(runs):
        s, r = timed(lambda: learned_run(npk, seed0 + i))
        runs_l.append((s, r["hist"]))
        stats["learned_transitions"] += r["steps"]
        stats["learned_proposals"] += r["proposals"]
        stats["learned_launches"] += r["launches"]
        stats["aborted"] += r["aborted"]
        s, r = timed(lambda: plain_run(npk, seed0 + 0x100 + i))
        runs_p.append((s, r["hist"]))
        stats["plain_transitions"] += r["steps"]
        stats["aborted"] += r["aborted"]
    ref, t_ref, chunk = None, 0.0, 1_000_000
    for k in range(0, n_ref, chunk):
        s, r = timed(lambda: plain_run(min(chunk, n_ref - k), seed0 + 0x200 + k // chunk))
        ref = r["hist"].astype(np.float64) if ref is None else ref + r["hist"]
        t_ref += s
    out = {"reference_s": t_ref, "learned_transitions_per_packet": stats["learned_transitions"] / (runs * npk),
           "learned_proposals_per_packet": stats["learned_proposals"] / (runs * npk),
           "learned_launches_per_run": stats["learned_launches"] / runs,
           "plain_transitions_per_packet": stats["plain_transitions"] / (runs * npk), "aborted": stats["aborted"],
           "equal_l1": _equal_l1(runs_l, runs_p, ref, n_ref, npk)}
    return out


def _learned_bricks(R, torch, n=64, brick=16, margin=1, J=64, x_max=64.0, tau0=1.0e7, npk=400_000, runs=4,
                    n_ref=6_400_000, ndata=1_500_000, iters=4000, time_slice_us=1000):
    """The exact uniform-brick proposal on the clumpy medium drawn per brick
    (the "clumpy bricks" variant: density and velocity constant inside each
    16^3-cell brick, so a brick's inner cube is a uniform medium whose first
    passages the network learns from uniform cubes), against the plain walk
    at equal escape-spectrum L1 (_arms, _equal_l1)."""
    from paper_1709_10187_gb300 import learned as Lr
    out = {"workload": f"clumpy_bricks_{n}c_{J}b_brick{brick}_tau{tau0:.0e}", "tau0": tau0}
    med = W.clumpy_medium(n=n, J=J, x_max=x_max, tau0=tau0, brick=brick, packets=npk)
    prob = R.Problem.clumpy(med)
    rho = med.brick_rho
    levels = np.logspace(np.log10(rho.min()) - 0.05, np.log10(rho.max()) + 0.05, 24)
    t0 = time.perf_counter()
    prop = Lr.ExitProposal(med.workload, brick - 2 * margin, levels, tau_lo=5.0, tau_hi=1.0e12)
    data = prop.generate(ndata, seed=11, cap=50_000_000)
    torch.cuda.synchronize()
    out["data_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    prop.train(data, iters=iters, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t0
    del data
    out.update(train_samples=ndata, train_iters=iters, region=brick - 2 * margin, levels=len(prop.levels),
               time_slice_us=time_slice_us)
    kw = dict(margin=margin, tau_lo=5.0, tau_hi=1.0e12, time_slice_us=time_slice_us)
    out.update(_arms(torch, lambda n_, s_: prop.run(prob, rho, n_, s_, **kw), lambda n_, s_: prob.run(n_, s_),
                     npk, runs, n_ref, 0xB0000))
    prob.close()
    return out


def _equal_l1(runs_l, runs_p, ref_hist, n_ref, npk, targets=(0.02, 0.01), n_boot=200, seed=0x5EED0B00):
    """Learned against plain at equal escape-spectrum L1, from independent seed
    runs of npk packets per arm (each run: (seconds, histogram)) and an
    independent plain reference of n_ref packets.

    Model of an arm's expected L1 against the reference at N packets:
    L1(N)^2 = B^2 + K^2 (1/N + 1/n_ref), with K = sqrt(2/pi) sum_b sqrt(p_b (1 -
    p_b)) the multinomial noise constant of the spectrum p (taken from the
    reference): E|X| = sqrt(2/pi) sd for each bin's normal fluctuation, and the
    arm's and the reference's noise add.  B, the arm's bias floor, is the part
    of the pooled runs' L1 the noise does not explain (0 for an unbiased arm,
    up to noise).  The packets an arm needs for a target L1 follow from its
    model, the wall time from its measured seconds per packet.  The measured
    cumulative curves L1(first m runs) are reported beside the model.  Errors:
    bootstrap over the runs (resampled with replacement)."""
    ref = np.asarray(ref_hist, dtype=np.float64)
    ref = ref / ref.sum()
    K = float(np.sqrt(2.0 / np.pi) * np.sqrt(ref * (1.0 - ref)).sum())
    rng = np.random.default_rng(seed)

    def curve(runs, order):
        acc = np.zeros_like(ref)
        l1s, ts, t = [], [], 0.0
        for i in order:
            sec, h = runs[i]
            acc = acc + np.asarray(h, dtype=np.float64)
            t += sec
            l1s.append(float(np.abs(acc / acc.sum() - ref).sum()))
            ts.append(t)
        return np.array(l1s), np.array(ts)

    def arm(runs, order):
        l1s, ts = curve(runs, order)
        n = len(l1s) * npk
        noise2 = K * K * (1.0 / n + 1.0 / n_ref)
        b2 = max(l1s[-1] ** 2 - noise2, 0.0)
        return b2, ts[-1] / n, l1s, ts

    def need(b2, tgt):
        d = tgt * tgt - b2 - K * K / n_ref
        return K * K / d if d > 0 else float("inf")

    def summary(order_l, order_p):
        bl, spp_l, l1l, tl = arm(runs_l, order_l)
        bp, spp_p, l1p, tp = arm(runs_p, order_p)
        out = {"bias_floor_learned": np.sqrt(bl), "bias_floor_plain": np.sqrt(bp),
               "s_per_packet_learned": spp_l, "s_per_packet_plain": spp_p}
        for tgt in targets:
            nl, npl = need(bl, tgt), need(0.0, tgt)  # the plain walk is unbiased
            out[f"s_to_{tgt:g}_learned"] = nl * spp_l
            out[f"s_to_{tgt:g}_plain"] = npl * spp_p
            out[f"speedup_at_{tgt:g}"] = (npl * spp_p) / (nl * spp_l) if np.isfinite(nl) else 0.0
        return out, (l1l, tl, l1p, tp)

    n = len(runs_l)
    base, (l1l, tl, l1p, tp) = summary(range(n), range(len(runs_p)))
    boots = [summary(rng.integers(0, n, n), rng.integers(0, len(runs_p), len(runs_p)))[0] for _ in range(n_boot)]
    res = {"runs_per_arm": n, "packets_per_run": npk, "reference_packets": n_ref, "noise_constant_K": K,
           "curve_learned": {"packets": [int((i + 1) * npk) for i in range(n)], "s": tl.tolist(), "l1": l1l.tolist()},
           "curve_plain": {"packets": [int((i + 1) * npk) for i in range(len(tp))], "s": tp.tolist(),
                           "l1": l1p.tolist()},
           "curve_model_unbiased": [float(K * np.sqrt(1.0 / ((i + 1) * npk) + 1.0 / n_ref)) for i in range(n)]}
    for k, v in base.items():
        vals = np.array([b[k] for b in boots], dtype=np.float64)
        fin = vals[np.isfinite(vals)]
        res[k] = {"value": float(v), "err": float(fin.std()) if fin.size > 1 else None,
                  "bootstrap_finite": int(fin.size)}
    return res


def _learned_c5(R, torch, tau0=1.0e7, npk=100_000, runs=8, n_ref=10_000_000, ndata=4_000_000, iters=4000,
                brick=16, margin=1, n=128, J=256, x_max=256.0, time_slice_us=1000):
    """The learned proposal on the clumpy workload at cell resolution (128^3
    cells x 256 bins over [-256, 256], lognormal density sigma_ln = 1 with
    spectral slope -11/3, turbulent velocity 10 km/s per component, tau0 at
    the mean density): region proposals over bricks of `brick` cells (inner
    cubes of brick - 2 margin) trained on first passages the plain walk takes
    through the medium's own regions, then `runs` independent runs of npk
    packets per arm against a plain reference of n_ref packets (_arms,
    _equal_l1)."""
    from paper_1709_10187_gb300 import learned as Lr
    out = {"workload": f"clumpy_cells_{n}c_{J}b_tau{tau0:.0e}", "tau0": tau0}

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    med = W.clumpy_medium(n=n, J=J, x_max=x_max, tau0=tau0, brick=1, packets=npk)
    out["precompute_s"], prob = timed(lambda: R.Problem.clumpy(med))
    out["table_bytes"] = int(prob.table.numel())
    out["setup_s"], prop = timed(lambda: Lr.RegionProposal(prob, med.n_rel, med.v_kms, brick, margin, tau_lo=5.0,
                                                           tau_hi=1.0e12))
    out["data_s"], data = timed(lambda: prop.generate(ndata, seed=11))
    held = prop.generate(65536, seed=12, p0=1 << 40)
    out["train_s"], _ = timed(lambda: prop.train(data, iters=iters, batch=8192, lr=2e-3))
    out["heldout_loss"] = prop.mean_loss(held)
    out.update(train_samples=ndata, train_iters=iters, region=brick - 2 * margin, n_out=prop.n_out,
               time_slice_us=time_slice_us)
    del data, held
    out.update(_arms(torch, lambda n_, s_: prop.run(n_packets=n_, seed=s_, time_slice_us=time_slice_us),
                     lambda n_, s_: prob.run(n_, s_), npk, runs, n_ref, 0xC5000))
    prob.close()
    return out


def _c5_plain(R, torch, n=64, J=256, x_max=256.0, tau0=1.0e7, npk=400_000, slice_=65536, warm=4):
    """Transitions/s of the plain walk on the cell-resolution lognormal medium
    (n^3 cells x J bins, every cell its own density and velocity): npk packets
    in launches of slice_ transitions each, timed after `warm` launches have
    carried the packets away from the source (_sliced_rate)."""
    med = W.clumpy_medium(n=n, J=J, x_max=x_max, tau0=tau0, brick=1, packets=npk)
    prob = R.Problem.clumpy(med)
    out = {"workload": f"clumpy_cells_{n}c_{J}b_tau{tau0:.0e}", "table_bytes": int(prob.table.numel()),
           "untimed_transitions_per_packet": warm * slice_}
    out.update(_sliced_rate(R, torch, prob, npk, 0xC5064, slice_, warm=warm))
    prob.close()
    return out


def _time_dependent(R, torch, w, npk, t_edges, kind, marks, chunk=0, ctas_per_sm=0, with_leaks=False,
                    compare_regroup=False):
    """A flash of npk packets advanced through constant time steps, one launch
    of the time-dependent walk per step (Sec. 2.3; eq. E_estimator), timed with
    CUDA events around all launches (a warm-up pass over the first steps runs
    before).  Physics summary at the `marks` times: for the grey test the L1
    distance of the bin estimate from the Fick Gaussian (D = 1/(3k)); for the
    resonant slab the slope d ln E_z / d|z/R| of the frequency-integrated path
    estimate, beside the paper's fit -2.24 (t/t_diff)^-0.72 (Sec. 3)."""
    prob = R.Problem(w)
    s = prob.stream()
    nt = len(t_edges) - 1
    S = w.ncell * prob.J
    state = torch.empty(R.time_state_bytes(npk), dtype=torch.uint8, device=prob.device)
    bins = torch.zeros((nt, S), dtype=torch.int64, device=prob.device)
    path = torch.zeros((nt, S), dtype=torch.int64, device=prob.device)
    counts = torch.zeros((nt, 5), dtype=torch.int64, device=prob.device)
    nf = 2 * w.ndim
    leak = torch.zeros((nt, w.ncell * nf * 2), dtype=torch.float64, device=prob.device)
    use_leak = [False]
    regroup = [0]  # 0: the library default; -1: warps never regroup

    def steps(k_end):
        for k in range(k_end):
            st = R.TimeStep(w.seed, npk, 0, float(t_edges[k]), float(t_edges[k + 1]), 1 if k == 0 else 0, chunk, 0,
                            ctas_per_sm, regroup[0])
            R.time_step_launch(prob.grid, prob.table.data_ptr(), st, state.data_ptr(), state.numel(),
                               prob.tally.data_ptr(), prob.tally.numel() * 8, bins[k].data_ptr(), path[k].data_ptr(),
                               counts[k].data_ptr(), s, leak[k].data_ptr() if use_leak[0] else 0)

    steps(min(nt, 4))  # warm-up
    for b in (bins, path, counts):
        b.zero_()
    prob.reset()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record(torch.cuda.current_stream())
    steps(nt)
    a1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    dt = a0.elapsed_time(a1) / 1e3
    c = counts.cpu().numpy()
    tr, dw = int(c[:, 2].sum()), int(c[:, 1].sum())
    out = {"workload": w.name, "packets": npk, "time_steps": nt, "dt": float(t_edges[1] - t_edges[0]), "s": dt,
           "ms_per_time_step": 1e3 * dt / nt, "packet_steps_per_s": npk * nt / dt, "transitions_per_s": tr / dt,
           "dwells_per_s": dw / dt, "transitions_per_packet": tr / npk, "escaped": int(c[:, 0].sum()),
           "alive_at_end": int(c[-1, 3]), "launches": nt}
    if with_leaks:
        # the same run with the leak tally of eq. a_estimator: its cost, and the
        # net acceleration direction sum_f (out - in) n_f of the cells (slab:
        # faces -z, +z) at the last mark
        for b in (bins, path, counts):
            b.zero_()
        prob.reset()
        use_leak[0] = True
        torch.cuda.synchronize()
        a0.record(torch.cuda.current_stream())
        steps(nt)
        a1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        dtl = a0.elapsed_time(a1) / 1e3
        lk = leak.cpu().numpy().reshape(nt, w.ncell, nf, 2)[-1]
        acc = (lk[:, 1, 0] - lk[:, 1, 1]) - (lk[:, 0, 0] - lk[:, 0, 1])
        zc = w.cell_centres()[:, 0]
        outward = float(np.mean(np.sign(acc[np.abs(zc) > 0.1 * w.R]) == np.sign(zc[np.abs(zc) > 0.1 * w.R])))
        out["with_leak_estimator"] = {"s": dtl, "overhead": dtl / dt - 1.0,
                                      "share_of_cells_accelerated_outward": outward}
    if compare_regroup:
        # the same run with warps that never regroup (rddmc_time_step.regroup =
        # -1): the estimates are identical, only the time differs
        b_ref, p_ref = bins.clone(), path.clone()
        for b in (bins, path, counts):
            b.zero_()
        prob.reset()
        use_leak[0] = False
        regroup[0] = -1
        torch.cuda.synchronize()
        a0.record(torch.cuda.current_stream())
        steps(nt)
        a1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        dtr = a0.elapsed_time(a1) / 1e3
        same = bool(torch.equal(bins, b_ref) and torch.equal(path, p_ref))
        out["without_regrouping"] = {"s": dtr, "regrouping_speedup": dtr / dt, "estimates_identical": same}
        regroup[0] = 0
    ks = [int(round(m / (t_edges[1] - t_edges[0]))) - 1 for m in marks]
    b = bins.cpu().numpy()
    pth = path.cpu().numpy().astype(np.float64)
    z = w.cell_centres()[:, 0] / w.R
    if kind == "grey":
        tau_c = R.cell_tau(prob.grid, prob.table.data_ptr(), w.n[0] // 2, prob.J, prob.stream())
        k = float(tau_c[0]) / (2.0 * w.R / w.n[0])
        from scipy.special import erf
        e = np.linspace(-w.R, w.R, w.n[0] + 1)
        out["grey_l1_vs_fick"] = {}
        for m, kk in zip(marks, ks):
            g = 0.5 * np.diff(erf(e / np.sqrt(4.0 * t_edges[kk + 1] / (3.0 * k))))
            out["grey_l1_vs_fick"][f"{m:.4g}"] = _l1(b[kk].astype(np.float64), g)
    else:
        t_diff = w.atau0_nominal ** (1.0 / 3.0) * w.R
        sel = (np.abs(z) >= 0.05) & (np.abs(z) <= 0.8)
        out["slope_dlnEz_dz"] = {}
        for m, kk in zip(marks, ks):
            ez = pth[kk].reshape(w.ncell, prob.J).sum(axis=1)
            ok = sel & (ez > 0)
            slope = float(np.polyfit(np.abs(z[ok]), np.log(ez[ok]), 1)[0])
            out["slope_dlnEz_dz"][f"{m / t_diff:.2f}"] = {"measured": slope,
                                                          "paper_fit": -2.24 * (m / t_diff) ** -0.72}
    return out


def _time_grey(R, torch, npk=10_000_000):
    """Sec. 3 grey test: 101 cells, steps of 1e-3 t_diff, t_diff = k R^2 / 2c, to 0.16 t_diff."""
    w = W.GREY101
    p = R.Problem(w)
    k = float(R.cell_tau(p.grid, p.table.data_ptr(), w.n[0] // 2, p.J, p.stream())[0]) / (2.0 * w.R / w.n[0])
    p.close()
    t_diff = 0.5 * k * w.R ** 2
    te = W.time_edges(1e-3 * t_diff, 0.16 * t_diff)
    return _time_dependent(R, torch, w, npk, te, "grey", [f * t_diff for f in (0.01, 0.02, 0.04, 0.08, 0.16)])


def _time_p2(R, torch, npk=10_000_000, t_frac=0.32):
    """Sec. 3 time-dependent resonant slab: a tau0 = 1e9, T = 10 K, 101 cells, 51
    bins of ~0.1 (a tau0)^(1/3), steps of 1e-3 (a tau0)^(1/3) R/c."""
    w = W.P2
    t_diff = w.atau0_nominal ** (1.0 / 3.0) * w.R
    te = W.time_edges(1e-3 * t_diff, t_frac * t_diff)
    marks = [f * t_diff for f in (0.01, 0.02, 0.04, 0.08, 0.16, 0.32) if f <= t_frac + 1e-9]
    return _time_dependent(R, torch, w, npk, te, "slab", marks, with_leaks=True, compare_regroup=True)


def _extras(R, torch, only=None):
    out = {}
    jobs = [("c3_sphere_static", lambda: _sliced_rate(R, torch, R.Problem(W.C3), 1_000_000, W.C3.seed, 4096)),
            ("c3_sphere_v20", lambda: _sliced_rate(R, torch, R.Problem(W.C3_V20), 1_000_000, W.C3.seed, 4096)),
            ("c3_sphere_v200", lambda: _sliced_rate(R, torch, R.Problem(W.C3_V200), 1_000_000, W.C3.seed, 4096)),
            ("c2_hybrid", lambda: _sliced_rate(R, torch, R.Problem(W.C2, mode=R.MODE_HYBRID), 1_000_000,
                                               W.C2.seed, 4096)),
            ("c2_hybrid_grouped", lambda: _grouped_rate(R, torch)),
            ("c1_complete", lambda: _complete(R, torch, W.C1, W.C1.packets)),
            ("c2_widecore_complete", lambda: _complete(R, torch, W.C2_WIDECORE, W.C2_WIDECORE.packets)),
            ("batched_512", lambda: _batched(R, torch)),
            ("time_grey_paper", lambda: _time_grey(R, torch)),
            ("time_slab_atau1e9_paper", lambda: _time_p2(R, torch)),
            # eight seeded runs of 4e5 packets per arm against a 1e7-packet plain reference
            ("learned_bricks", lambda: _learned_bricks(R, torch, npk=400_000, runs=8, n_ref=10_000_000,
                                                       time_slice_us=4000)),
            ("learned_c5", lambda: _learned_c5(R, torch, tau0=1.0e7, npk=400_000, runs=8, n_ref=10_000_000,
                                               brick=8, margin=1, time_slice_us=8000))]
    if only:
        small = {"learned_small": lambda: _learned_bricks(R, torch, n=32, brick=8, tau0=1.0e6, npk=100_000,
                                                          n_ref=1_600_000, ndata=300_000, iters=300),
                 "learned_c5_tau1e8": lambda: _learned_c5(R, torch, tau0=1.0e8, npk=50_000, runs=4, n_ref=800_000,
                                                          ndata=2_000_000, brick=8, margin=1, time_slice_us=8000),
                 "learned_c5_tau1e9": lambda: _learned_c5(R, torch, tau0=1.0e9, npk=5_000, runs=4, n_ref=80_000,
                                                          ndata=500_000, brick=8, margin=1, time_slice_us=8000),
                 # the batched workload at its full size (1.1e8 packets, ~7.8e14 transitions: ~14 min); the
                 # watchdog (2e10 transitions, ~10x the slowest packet expected) only bounds the launch
                 "batched_512_full": lambda: _batched(R, torch, packet_scale=1.0, max_steps=20_000_000_000),
                 # a 1e5-packet subset of the tau0 = 1e7 slab walked to escape (~5 min)
                 "c2_complete_1e5": lambda: _complete_sliced(R, torch, W.C2, 100_000),
                 # the plain walk on a 64^3-cell lognormal medium (256 bins, tau0 = 1e7, a 3 GB table): the
                 # cell-resolution workload at a size a counter capture can hold
                 "c5_cells_64_plain": lambda: _c5_plain(R, torch, n=64),
                 # a short time-dependent run for profiling: 1e6 packets, 16 steps
                 "time_slab_small": lambda: _time_p2(R, torch, npk=1_000_000, t_frac=0.016)}
        jobs = [(k, f) for k, f in jobs + list(small.items()) if k == only]
        if not jobs:
            raise SystemExit(f"unknown extra {only!r}")
    for name, fn in jobs:
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as exc:  # reported, not hidden: the main line still prints
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def _kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("walk.cu", "walk_common.cuh", "escape.cuh", "rddmc_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1709_10187_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--slice", type=int, default=4096, help="transitions per packet per step")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--table-in-smem", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-completed", action="store_true",
                    help="also time the oracle on completed packet subsets (C1, P1, P2 in full; C2, C3 subsets; "
                         "several minutes of host time)")
    ap.add_argument("--no-gather", action="store_true", help="skip the gather-rate probe (no gather fraction)")
    ap.add_argument("--no-complete", action="store_true",
                    help="skip the completed 1e5-packet subset (no escaped packets/s)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads and the learned-vs-plain comparison")
    ap.add_argument("--extra", default="", help="run only this extra (c3_sphere_static, c3_sphere_v20, "
                    "c3_sphere_v200, c2_hybrid, c2_hybrid_grouped, c1_complete, c2_widecore_complete, batched_512, "
                    "time_grey_paper, time_slab_atau1e9_paper, learned_bricks, learned_c5; opt-in only: "
                    "learned_small, learned_c5_tau1e8, learned_c5_tau1e9, batched_512_full, c2_complete_1e5, "
                    "time_slab_small, c5_cells_64_plain) and print it")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.extra:
        # one extra workload alone (for profiling); no timed region, no bench line
        import torch
        from paper_1709_10187_gb300 import build as B
        from paper_1709_10187_gb300 import rddmc as R
        B.build()
        print(json.dumps({"extra": args.extra, **_extras(R, torch, only=args.extra)}), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_native(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
