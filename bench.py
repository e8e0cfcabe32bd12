#!/usr/bin/env python
"""Benchmark of the LArTPC signal-simulation hot path (rasterize + scatter-add + convolve).

Workload: one MicroBooNE-sized collection plane, 3456 wires x 9600 ticks (0.5 us), 100k depos
on 20 straight tracks, drift 0-2.3 ms, fluctuation on, 21 x 200 synthetic response.  A step
is one run_batch over --batch such events (distinct seeds / event ids, depos resident in HBM),
each going through the whole path: grid clear, fused drift/window + rasterize + fluctuate +
scatter, forward row FFT, wire stage, inverse row FFT.  value = depos/s over the whole job.
Per-kernel times (roofline) and single-event latency come from a second pass of run_event
calls with CUDA events on the launching stream.  The JSON
line also carries the batched form (64 uneven three-plane events per run_batch) and the served
form (APA-like stream, continuous batching, p50/p99 latency).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun), events sharded across ranks (weak scaling, no
data-path collective).  The reference arm times the FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "depos/s and events/s (rasterize+scatter+convolve); p50/p99 event latency"
WORKLOAD = "uboone_plane"
FALLBACK_HBM_GBS = 6800.0
ORACLE_SAMPLE_DEPOS = 25_000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16, help="events per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / served measurements")
    ap.add_argument("--schedule", type=int, default=-1,
                    help="kernel schedule: -1 default, 0 register-staged rows, 1 persistent bulk-copy rows, "
                         "4 paired rows, 8 paired rows with composite radices; +2 CTA-level rasterizer")
    return ap.parse_args()


# --------------------------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                if self.bus_id and self.bus_id[-12:] not in p[1].lower():
                    continue
                rows.append(p)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), float(j.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, 2070.0, "fallback"


# The rasterize kernel is bound by instruction issue (Philox integer multiplies, SFU, shared
# memory), not by HBM: its roofline is the issue rate, 4 warp-instructions per clock per SM
# (one per scheduler) x 152 SMs x the maximum SM clock.
N_SMS = 152
ISSUE_PER_SM_CLK = 4


def stage_bytes(plane, n_depos, spec_bins, resp_ticks=200):
    """Algorithmic bytes per event of each stage (f32 = 4 B, c64 = 8 B).  The spectrum is
    counted at the bins that carry signal: those below the response spectrum's support (the
    library's spectrum_bins_used), at most the unpadded half length of n_ticks + 199."""
    nw, nt = plane.n_wires, plane.n_ticks
    grid = 4 * nw * nt
    spec = 8 * nw * min(spec_bins, (nt + resp_ticks - 1) // 2 + 1)
    return {
        "prep_binning": 20 * n_depos,
        "raster_scatter": 20 * n_depos + grid,
        "row_r2c": grid + spec,
        "wire_stage": 2 * spec,
        "row_c2r": spec + grid,
        "convolve": 2 * grid + 2 * spec,
    }


def kernel_counters():
    """ncu counters per launch of the main kernels (profiles/kernel_counters.json), valid only
    while the CUDA sources are unchanged (csrc digest)."""
    p = os.path.join(ROOT, "profiles", "kernel_counters.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


def csrc_digest():
    import hashlib
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_2304_01841_gb300", "csrc")
    for name in sorted(os.listdir(cdir)):
        with open(os.path.join(cdir, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def shard_plan(rank: int, world: int, events_per_rank: int, base_seed: int):
    """Weak scaling: rank r simulates its own events_per_rank events (seeds and event ids
    disjoint across ranks); no data crosses ranks."""
    return [(base_seed + 1000 * rank + e, rank * events_per_rank + e) for e in range(events_per_rank)]


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The job's time is the slowest rank's (all-reduce MAX; identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(wl, n_sample=ORACLE_SAMPLE_DEPOS, seed_offset=0, threads=None):
    """Time the FP64 oracle on a bounded sample of one event: the first n_sample depos
    rasterized + scattered (C, 1 thread) and the full-grid FFT convolution (scipy, all cores).
    Returns (estimated seconds for the whole event, threads): the raster part scales with the
    depo count, the convolution is once per event."""
    import oracle
    d = wl.depos(seed=wl.seed + seed_offset).subset(slice(0, n_sample))
    plane = wl.planes[0]
    resp = wl.responses()[0]
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    pt = oracle.rasterize(d, plane, wl.diffusion)
    grid = oracle.scatter(pt, plane)
    t1 = time.perf_counter()
    oracle.convolve_fft(grid, resp, workers=threads)
    t2 = time.perf_counter()
    return (t1 - t0) * wl.n_depos / d.n + (t2 - t1), threads


# --------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# --------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    wl = synth.workload(WORKLOAD)
    for w in range(args.warmup):
        oracle_sample(wl, seed_offset=w)
    times = []
    threads = 1
    for k in range(args.steps):
        t, threads = oracle_sample(wl, seed_offset=100 + k)
        times.append(t)
    total = sum(times)                          # estimated whole-event seconds, one event per step
    value = wl.n_depos * args.steps / total
    sample = (f"per step one event: {ORACLE_SAMPLE_DEPOS} of its 100k depos rasterized + scattered (C, 1 thread; "
              f"time scaled to the 100k) + the full 3456x9600 FFT convolution (scipy FP64, {threads} threads)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "depos/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "planes": "1 x 3456 wires x 9600 ticks", "depos_per_event": 100_000,
                   "fluctuation": True, "sample_depos_per_step": ORACLE_SAMPLE_DEPOS},
        "cpu_baseline": {"value": value, "unit": "depos/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "depos/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
# batched and served forms (three-plane batch of uneven events; APA-like serving stream)
# --------------------------------------------------------------------------------------------
def _slice_pool(pool, counts, rng, first_event_id):
    """Events of the given depo counts cut from a pool of large generated events (each a
    contiguous slice, i.e. whole track segments), with distinct event ids."""
    import synth
    out = []
    for i, n in enumerate(counts):
        base = pool[int(rng.integers(len(pool)))]
        n = int(min(n, base.n))
        s0 = int(rng.integers(0, base.n - n + 1))
        d = base.subset(slice(s0, s0 + n))
        out.append(synth.Depos(d.t0, d.x, d.y, d.z, d.q, event_id=first_event_id + i))
    return out


def measure_batch(n_events=64, reps=5):
    """Batched: n_events three-plane events (2400/2400/3456 x 9600), depo counts lognormal
    10k..500k, one run_batch (batched raster launch + graph-replayed convolutions) against the
    same events one run_event at a time.  Returns events/s of both."""
    import numpy as np
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload("three_plane")
    counts = synth.batch_depo_counts(n_events)
    pool = [wl.depos(n_depos=500_000, seed=wl.seed + k) for k in range(3)]
    evs = _slice_pool(pool, counts, np.random.default_rng(7), 5000)
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    dev = [pkg.DeviceDepos.from_host(e) for e in evs]
    outs = [[torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, device="cuda") for p in wl.planes]
            for _ in evs]
    st = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1000.0

    t_batch = timed(lambda: sim.run_batch(dev, outs))
    t_single = timed(lambda: [sim.run_event(d, o) for d, o in zip(dev, outs)])
    sim.sync()
    n = reps * n_events
    sim.close()
    return {"workload": "64 three-plane events (2400/2400/3456 x 9600), depos lognormal 10k-500k",
            "depos_per_batch": int(sum(e.n for e in evs)), "events_per_s_batched": n / t_batch,
            "events_per_s_one_at_a_time": n / t_single,
            "depos_per_s_batched": reps * sum(e.n for e in evs) / t_batch}


def measure_impact(n_events=4, reps=2):
    """Impact mode (per-impact-position responses, 10 phases) on the uboone_plane workload:
    run_event per event (unfused patches, 10 phase grids, 10 transforms + stencils, one inverse
    transform), CUDA events around reps x n_events events, against the folded mode."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload(WORKLOAD)
    pl = wl.planes[0]
    evs = [pkg.DeviceDepos.from_host(wl.depos(seed=wl.seed + 100 + e, event_id=500 + e)) for e in range(n_events)]
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    out = torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def timed():
        for d in evs[:2]:
            sim.run_event(d, [out])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            for d in evs:
                sim.run_event(d, [out])
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1000.0 / (reps * n_events)

    t_folded = timed()
    sim.set_impact_responses(0, synth.make_response_impact(pl.response_kind, n_impact=pl.n_impact_per_pitch))
    t_impact = timed()
    sim.set_timing(True)
    for d in evs:
        sim.run_event(d, [out])
    sim.sync()
    stages = sim.stage_times()
    sim.set_timing(False)
    sim.close()
    n = evs[0].n
    return {"workload": f"{WORKLOAD}, 10 per-impact-position responses (21 x 200 each)",
            "events_per_s": 1.0 / t_impact, "depos_per_s": n / t_impact, "ms_per_event": 1e3 * t_impact,
            "folded_ms_per_event": 1e3 * t_folded,
            "stages_us": {"patches_rasterize_scatter": round(stages["raster_scatter"] + stages["prep_binning"], 1),
                          "phase_transforms": round(stages["row_r2c"], 1),
                          "phase_stencils": round(stages["wire_stage"], 1),
                          "inverse_transform": round(stages["row_c2r"], 1)}}


def measure_deterministic(n_events=16, reps=5):
    """Cost of the deterministic mode (fixed-point integer accumulation, bitwise reproducible):
    one run_batch of n_events uboone_plane events on a deterministic handle against the default
    handle, CUDA events around reps batches each (graph replay after the first call)."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload(WORKLOAD)
    pl = wl.planes[0]
    evs = [pkg.DeviceDepos.from_host(wl.depos(seed=wl.seed + 200 + e, event_id=700 + e)) for e in range(n_events)]
    outs = [[torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.float32, device="cuda")] for _ in evs]
    st = torch.cuda.current_stream()
    res = {}
    for det in (False, True):
        sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion, deterministic=det)
        for _ in range(3):
            sim.run_batch(evs, outs)
        sim.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            sim.run_batch(evs, outs)
        b.record(st)
        torch.cuda.synchronize()
        sim.sync()
        res[det] = a.elapsed_time(b) / 1000.0 / (reps * n_events)
        sim.close()
    n = evs[0].n
    return {"workload": f"{WORKLOAD}, {n_events}-event run_batch", "events_per_s": 1.0 / res[True],
            "depos_per_s": n / res[True], "default_events_per_s": 1.0 / res[False],
            "slowdown": res[True] / res[False]}


def measure_cufft(reps=10):
    """Comparison only (not on the path): the same row transforms through the vendor FFT
    (torch.fft, i.e. cuFFT) on the uboone_plane grid, full half spectrum of length P, against
    this library's forward / inverse row kernels timed inside run_event."""
    import torch
    import synth
    import paper_2304_01841_gb300 as pkg
    wl = synth.workload(WORKLOAD)
    pl = wl.planes[0]
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    P = sim.plane_info(0)["fft_length"]
    g = torch.randn((pl.n_wires, pl.n_ticks), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1000.0 / reps

    spec = torch.fft.rfft(g, n=P, dim=1)
    fwd = timed(lambda: torch.fft.rfft(g, n=P, dim=1))
    inv = timed(lambda: torch.fft.irfft(spec, n=P, dim=1))
    dev = pkg.DeviceDepos.from_host(wl.depos())
    sim.set_timing(True)
    for _ in range(reps):
        sim.run_event(dev)
    sim.sync()
    ours = sim.stage_times()
    sim.set_timing(False)
    sim.close()
    return {"workload": f"{pl.n_wires} rows x {pl.n_ticks} ticks, real transform length {P}",
            "cufft_forward_us": round(fwd, 1), "cufft_inverse_us": round(inv, 1),
            "ours_forward_us": round(ours["row_r2c"], 1), "ours_inverse_us": round(ours["row_c2r"], 1),
            "note": "cuFFT computes every bin (4901 per row) and its inverse writes the padded length; "
                    "ours stops at the response's support and writes the kept ticks"}


def measure_scan_free(reps=5):
    """Unfused rasterize on the uboone_plane event: the prefix-sum version (size query, host
    synchronisation, packed patches) against the scan-free one (a fixed slot per depo sized for
    the largest window at the maximum drift), as the paper's OpenMP port does."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload(WORKLOAD)
    pl = wl.planes[0]
    d = wl.depos()
    dd = pkg.DeviceDepos.from_host(d)
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    slot = sim.patch_slot_bins(0, float(d.x.max()))
    desc, patches = sim.rasterize(0, dd)
    total = patches.numel()
    desc_f, patches_f = sim.rasterize_fixed(0, dd, slot)
    st = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e3 / reps

    import ctypes
    total_c = ctypes.c_int64()
    ds = dd.c_struct()
    lib, h = sim._lib, sim._h

    def scanned():   # size query + patches, as a caller of the scanned API does it
        lib.wct_sim_rasterize(h, 0, ctypes.byref(ds), None, 0, desc.data_ptr(), ctypes.byref(total_c), None)
        lib.wct_sim_rasterize(h, 0, ctypes.byref(ds), patches.data_ptr(), total, desc.data_ptr(),
                              ctypes.byref(total_c), None)

    def fixed():
        lib.wct_sim_rasterize_fixed(h, 0, ctypes.byref(ds), patches_f.data_ptr(), slot, desc_f.data_ptr(), None)

    t_scan, t_fixed = timed(scanned), timed(fixed)
    sim.sync()
    sim.close()
    return {"workload": f"{WORKLOAD}, unfused rasterize with fluctuation", "slot_bins": slot,
            "scanned_us": round(t_scan, 1), "scan_free_us": round(t_fixed, 1),
            "scanned_patch_bytes": 4 * total, "scan_free_patch_bytes": 4 * d.n * slot}


def measure_digitize(reps=20):
    """Noise + digitisation of one uboone_plane waveform (3456 x 9600): algorithmic bytes 4 B
    read + 2 B written per bin; CUDA events over reps launches."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload(WORKLOAD)
    pl = wl.planes[0]
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    # two waveforms and two outputs used alternately: 400 MB, more than the L2
    wfs = [torch.randn((pl.n_wires, pl.n_ticks), device="cuda") * 100.0 for _ in range(2)]
    outs = [torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.int16, device="cuda") for _ in range(2)]
    st = torch.cuda.current_stream()
    for k in range(3):
        sim.digitize(0, wfs[k % 2], 1.0, 900.0, 2.5, out=outs[k % 2], event_id=1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for k in range(reps):
        sim.digitize(0, wfs[k % 2], 1.0, 900.0, 2.5, out=outs[k % 2], event_id=k)
    b.record(st)
    torch.cuda.synchronize()
    sim.sync()
    us = a.elapsed_time(b) * 1e3 / reps
    sim.close()
    peak, _, kind = measured_peaks()
    gbs = 6.0 * pl.n_wires * pl.n_ticks / (us * 1e-6) / 1e9
    return {"workload": f"{WORKLOAD} waveform, 12-bit codes with white noise", "us": round(us, 2),
            "alg_bytes": 6 * pl.n_wires * pl.n_ticks, "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
            "peak_source": f"{kind} (burst copy)"}


def measure_serving(n_events=120, loads=(0.5, 0.8, 0.95)):
    """Served: APA-like planes (800/800/960 x 6000), heavy-tailed depo counts (90% 5k-50k,
    10% 1M-3M), open-loop Poisson arrivals at fractions of the measured capacity."""
    import numpy as np
    import synth
    from paper_2304_01841_gb300.serve import EventServer, pin_depos, run_open_loop
    wl = synth.workload("dune_apa")
    pool = [wl.depos(n_depos=3_000_000, seed=wl.seed + k) for k in range(2)]
    counts = synth.serving_depo_counts(n_events)
    evs = [pin_depos(e) for e in _slice_pool(pool, counts, np.random.default_rng(9), 9000)]
    srv = EventServer(wl.planes, wl.responses(), wl.diffusion, n_slots=4, max_batch=8,
                      hbm_budget_bytes=24 << 30)
    # capacity: everything submitted at once
    for e in evs[:16]:
        srv.submit(e)
    srv.drain()
    t0 = time.perf_counter()
    for e in evs:
        srv.submit(e)
    srv.drain()
    cap = len(evs) / (time.perf_counter() - t0)
    points = []
    for i, f in enumerate(loads):
        r = run_open_loop(srv, evs, rate_hz=f * cap, seed=i)
        r["load"] = f
        points.append(r)
    srv.close()
    return {"workload": "APA-like 800/800/960 x 6000, 90% 5k-50k / 10% 1M-3M depos, Poisson arrivals",
            "capacity_events_per_s": cap, "open_loop": points}


# --------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2304_01841_gb300 as pkg
    import synth

    pkg.load(build_if_missing=True)
    wl = synth.workload(WORKLOAD)
    plane = wl.planes[0]
    n_depos = wl.n_depos
    E = args.batch
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion, schedule_id=args.schedule)
    # E distinct events per rank, resident in HBM (weak scaling: each rank its own events)
    host_events = [wl.depos(seed=seed, event_id=eid) for seed, eid in shard_plan(rank, world, E, wl.seed)]
    dev_events = [pkg.DeviceDepos.from_host(d) for d in host_events]
    outs = [[torch.empty((plane.n_wires, plane.n_ticks), dtype=torch.float32, device="cuda")] for _ in range(E)]
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        sim.run_batch(dev_events, outs)
    sim.sync()
    torch.cuda.synchronize()

    # ---- timed region: K steps, each one run_batch of the E resident events -------------
    # (run_batch overlaps the rasterize of event e + 1 with the convolution of event e and
    # replays a recorded CUDA graph from its second call on; every step recomputes everything)
    K = args.steps
    bus = None
    try:
        bus = getattr(torch.cuda.get_device_properties(local), "pci_bus_id", None)
    except Exception:
        pass
    clocks = ClockSampler(bus)
    launches0 = sim.counters()["kernel_launches"]
    clocks.start()
    time.sleep(0.2)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(K):
        sim.run_batch(dev_events, outs)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    sim.sync()
    elapsed_ms = start.elapsed_time(stop)
    launches = sim.counters()["kernel_launches"] - launches0
    elapsed_ms = max_over_ranks(elapsed_ms, world, "cuda")
    total_events = world * K * E
    value = total_events * n_depos / (elapsed_ms / 1000.0)

    # ---- per-kernel times and single-event latency: E x min(K, 4) run_event calls, each
    # kernel bracketed by CUDA events recorded on the launching stream ---------------------
    n_lat = E * min(K, 4)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_lat + 1)]
    sim.set_timing(True)
    ev[0].record(stream)
    for i in range(n_lat):
        sim.run_event(dev_events[i % E], outs[i % E])
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    stages = sim.stage_times()
    sim.set_timing(False)
    lat = sorted(ev[j].elapsed_time(ev[j + 1]) for j in range(n_lat))
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]

    # ---- roofline of the dominant kernel -----------------------------------------------
    peak_gbs, sm_mhz_max, peak_kind = measured_peaks()
    issue_peak = N_SMS * ISSUE_PER_SM_CLK * sm_mhz_max * 1e6          # warp-instructions / s
    sb = stage_bytes(plane, n_depos, sim.plane_info(0)["spectrum_bins_used"])
    kern = {k: stages[k] for k in ("raster_scatter", "row_r2c", "wire_stage", "row_c2r")}
    dom = max(kern, key=kern.get)
    cnt = kernel_counters()
    valid = cnt.get("csrc_digest") == csrc_digest()
    kname = {"raster_scatter": "k_raster_warps", "row_r2c": "k_row_r2c_pair", "wire_stage": "k_wire_stage_tma",
             "row_c2r": "k_row_c2r_pair"}
    stage_report = {}
    for k, us in list(kern.items()) + [("grid_clear", stages["prep_binning"])]:
        if k == "raster_scatter":
            insts = cnt.get("kernels", {}).get(kname[k], {}).get("warp_instructions_per_launch") if valid else None
            ach = insts / (us * 1e-6) if (insts and us > 0) else None
            stage_report[k] = {"us": round(us, 2), "bound": "alu", "warp_inst_per_s": ach,
                               "frac_of_issue_peak": round(ach / issue_peak, 4) if ach else None}
            continue
        alg = sb[k] if k != "grid_clear" else 4 * plane.n_wires * plane.n_ticks
        gbs = alg / (us * 1e-6) / 1e9 if us > 0 else None
        stage_report[k] = {"us": round(us, 2), "bound": "hbm", "alg_bytes": alg, "GB/s": round(gbs, 1) if gbs else None,
                           "frac": round(gbs / peak_gbs, 4) if gbs else None}
    conv_us = kern["row_r2c"] + kern["wire_stage"] + kern["row_c2r"]
    conv_gbs = sb["convolve"] / (conv_us * 1e-6) / 1e9
    # the same convolution counted without the support pruning (every bin of the unpadded half
    # spectrum), and as the classical three-pass 2D-FFT schedule would move it (row transform;
    # column transform x 2D response spectrum x inverse column transform; inverse row transform)
    grid_b = 4 * plane.n_wires * plane.n_ticks
    spec_full = 8 * plane.n_wires * ((plane.n_ticks + 199) // 2 + 1)
    unpruned, classical = 2 * grid_b + 2 * spec_full, 2 * grid_b + 5 * spec_full
    stage_report["convolve_total"] = {"us": round(conv_us, 2), "alg_bytes": sb["convolve"],
                                      "GB/s": round(conv_gbs, 1), "frac": round(conv_gbs / peak_gbs, 4),
                                      "unpruned_alg_bytes": unpruned,
                                      "unpruned_frac": round(unpruned / (conv_us * 1e-6) / 1e9 / peak_gbs, 4),
                                      "classical_3pass_bytes": classical,
                                      "classical_equiv_GB/s": round(classical / (conv_us * 1e-6) / 1e9, 1)}
    sc_us = kern["raster_scatter"] + stages["prep_binning"]
    sc_gbs = sb["raster_scatter"] / (sc_us * 1e-6) / 1e9
    stage_report["scatter_total"] = {"us": round(sc_us, 2), "alg_bytes": sb["raster_scatter"],
                                     "GB/s": round(sc_gbs, 1), "frac": round(sc_gbs / peak_gbs, 4),
                                     "what": "grid clear + rasterize/scatter, against depo read + grid write"}
    traffic = cnt["kernels"].get(kname[dom], {}).get("dram_bytes_per_launch") if valid else None
    if dom == "raster_scatter":
        insts = cnt["kernels"].get(kname[dom], {}).get("warp_instructions_per_launch") if valid else None
        ach = insts / (kern[dom] * 1e-6) if insts else None
        roofline = {"bound": "alu", "kernel": kname[dom], "achieved": ach, "peak": issue_peak,
                    "unit": "warp-inst/s", "frac": round(ach / issue_peak, 4) if ach else None, "traffic": traffic,
                    "peak_source": f"issue rate: {N_SMS} SMs x {ISSUE_PER_SM_CLK} warp-inst/clk x {sm_mhz_max:.0f} MHz "
                                   f"(max SM clock, {peak_kind}); instructions per launch from the committed ncu profile"}
    else:
        achieved = sb[dom] / (kern[dom] * 1e-6) / 1e9
        roofline = {"bound": "hbm", "kernel": kname[dom], "achieved": round(achieved, 1), "peak": peak_gbs,
                    "unit": "GB/s", "frac": round(achieved / peak_gbs, 4), "traffic": traffic,
                    "peak_source": f"{peak_kind} (burst copy)"}

    # ---- end to end through the public API with host buffers ---------------------------
    # wct_sim_run_host: pinned host depos in, pinned host waveforms out; the library pipelines
    # the upload of event e + 1 and the download of event e - 1 under the kernels of event e
    e2e = None
    if not args.no_e2e:
        pinned_in = []
        for d in host_events:
            o = type("PinnedDepos", (), {})()
            for k in ("t0", "x", "y", "z", "q"):
                setattr(o, k, torch.from_numpy(np.ascontiguousarray(getattr(d, k))).pin_memory())
            o.event_id = d.event_id
            pinned_in.append(o)
        n_host = 2
        host_out = [torch.empty((plane.n_wires, plane.n_ticks), dtype=torch.float32).pin_memory()
                    for _ in range(n_host)]
        outs_host = [[host_out[e % n_host]] for e in range(E)]
        h2d = 5 * 4 * n_depos * E
        d2h = 4 * plane.n_wires * plane.n_ticks * E

        def e2e_step():
            sim.run_host(pinned_in, outs=outs_host)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for k in range(K):
            e2e_step()
        s1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = s0.elapsed_time(s1)
        e2e_ms = max_over_ranks(e2e_ms, world, "cuda")
        e2e = {"value": world * K * E * n_depos / (e2e_ms / 1000.0), "unit": "depos/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "events_per_s": world * K * E / (e2e_ms / 1000.0),
               "d2h_GBps": round(d2h * K / (e2e_ms * 1e-3) / 1e9, 1),
               "what": "wct_sim_run_host: pinned host depos -> device -> pinned host waveform, every event; "
                       "uploads / downloads overlap the kernels (the download of 133 MB per event bounds it)"}

    # ---- CPU baseline (oracle, bounded sample) -------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t, threads = oracle_sample(wl)
        t1, _ = oracle_sample(wl, threads=1)
        cpu = {"value": wl.n_depos / t, "unit": "depos/s", "cores": threads, "kind": "oracle",
               "value_one_thread": wl.n_depos / t1,
               "sample": f"one event: {ORACLE_SAMPLE_DEPOS} of its {wl.n_depos} depos rasterized + scattered "
                         f"(C FP64, 1 thread; time scaled to the whole event) + the full-grid FFT convolution "
                         f"(scipy FP64, {threads} threads), one run"}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["batch"] = measure_batch()
        extras["serving"] = measure_serving()
        extras["impact_mode"] = measure_impact()
        extras["deterministic"] = measure_deterministic()
        extras["cufft_comparison"] = measure_cufft()
        extras["scan_free_rasterize"] = measure_scan_free()
        extras["digitize"] = measure_digitize()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "depos/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "planes": "1 x 3456 wires x 9600 ticks (0.5 us)",
                       "depos_per_event": n_depos, "tracks": 20, "fluctuation": True, "response": "21 x 200",
                       "events_per_step": E, "events_resident_in_hbm": E,
                       "l2": "each event touches its own 133 MB grid plus 2 x 59 MB spectra (> 126 MB L2) and a step cycles through 16 events; no flush needed"},
            "events_per_s": total_events / (elapsed_ms / 1000.0),
            "latency_ms": {"p50": p50, "p99": p99,
                           "what": "device time of one event through run_event, events back to back"},
            "roofline": roofline,
            "stages": stage_report,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s": wall,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
