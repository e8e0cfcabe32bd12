#!/usr/bin/env python
"""Benchmark of the LArTPC signal-simulation hot path (rasterize + scatter-add + convolve).

Workload (the largest single-GPU configuration): a batch of 64 three-plane events, planes of
2400 / 2400 / 3456 wires x 9600 ticks (0.5 us, +60 / -60 / 0 degrees), depo counts lognormal
with 10k / 500k at the 1st / 99th percentiles, each event cut from a generated 500k-depo event
of 200 straight tracks plus 20% isolated low-charge depos; fluctuation on; 21 x 200 synthetic
responses (bipolar induction, unipolar collection).  A step is one run_batch over the 64
events with their depos resident in HBM: one persistent rasterize + scatter launch over every
(event, plane) pair, then the convolutions (forward row FFT, wire stage, inverse row FFT) of
all 192 grids, replayed from a CUDA graph.  value = depos/s over the whole job; also events/s,
the same events one run_event at a time, per-event latency p50 / p99 and the single 1M-depo
three-plane event.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun), each rank its own 64 events (weak scaling, no
data-path collective).  The reference arm times the FP64 CPU oracle on whole events of the
same batch, on every host core.
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
WORKLOAD = "three_plane_batch"
PLANE_WORKLOAD = "three_plane"
FALLBACK_HBM_GBS = 6800.0
CPU_SAMPLE_S = 10.0          # all-core oracle: whole events until this much time has passed


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64, help="events per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the extra measurements")
    ap.add_argument("--schedule", type=int, default=-1,
                    help="kernel schedule (wct_opts_t.schedule_id): -1 default; bits 0-3 row transforms, "
                         "bit 1 CTA-level rasterizer, bits 4-7 events per raster launch, bit 8 one conv stream")
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
    """Algorithmic bytes per event-plane of each stage (f32 = 4 B, c64 = 8 B).  The spectrum
    is counted at the bins that carry signal: those below the response spectrum's support (the
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


def unpruned_convolve_bytes(plane, resp_ticks=200):
    """The convolution's bytes at every bin of the unpadded half spectrum: grid read, one write
    and one read of the time-frequency spectrum, waveform write; and the classical three-pass
    2D-FFT schedule's (row transform, column transform x 2D response x inverse column
    transform, inverse row transform)."""
    grid = 4 * plane.n_wires * plane.n_ticks
    spec = 8 * plane.n_wires * ((plane.n_ticks + resp_ticks - 1) // 2 + 1)
    return 2 * grid + 2 * spec, 2 * grid + 5 * spec


def kernel_counters():
    """ncu counters per launch of the main kernels (profiles/kernel_counters.json), valid only
    while the device-code sources are unchanged (csrc_digest)."""
    p = os.path.join(ROOT, "profiles", "kernel_counters.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


def csrc_digest():
    """Digest of the sources that hold device code (the kernels k_*.cu and the headers they
    include); the host-only orchestration (wct_sim.cu, wct_response.cu) does not enter it."""
    import hashlib
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_2304_01841_gb300", "csrc")
    for name in sorted(os.listdir(cdir)):
        if not (name.startswith("k_") and name.endswith(".cu")) and not name.endswith(".cuh"):
            continue
        with open(os.path.join(cdir, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def shard_plan(rank: int, world: int, events_per_rank: int, base_seed: int):
    """Weak scaling: rank r simulates its own events_per_rank events (seeds and event ids
    disjoint across ranks); no data crosses ranks."""
    return [(base_seed + 1000 * rank + e, rank * events_per_rank + e) for e in range(events_per_rank)]


def rank_events(rank: int, n_events: int):
    """The batch of one rank: its own pool seed and event-id range (weak scaling)."""
    import synth
    wl = synth.workload(PLANE_WORKLOAD)
    return synth.batch_events(n_events, pool_seed=wl.seed + 1000 * rank, first_event_id=5000 + rank * n_events)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The job's time is the slowest rank's (all-reduce MAX; identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cuda_timed(fn, reps: int, warm: int = 1):
    """Seconds per call of fn, CUDA events on the current stream around reps calls."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1000.0 / reps


# --------------------------------------------------------------------------------------------
# the oracle on the host cores
# --------------------------------------------------------------------------------------------
def oracle_events(events, planes, diff, responses, threads=0, budget_s=None):
    """Whole events through the FP64 oracle (every step of the path, every plane): all host
    cores (threads=0) or the given thread count.  Stops after budget_s seconds (at least one
    event).  Returns (seconds, depos, events, threads used)."""
    import oracle
    used = oracle.omp_threads(threads)
    t_total, n_depos, n_ev = 0.0, 0, 0
    for ev in events:
        t0 = time.perf_counter()
        oracle.simulate_event_all_cores(ev, planes, diff, responses, n_threads=threads)
        t_total += time.perf_counter() - t0
        n_depos += ev.n
        n_ev += 1
        if budget_s is not None and t_total >= budget_s:
            break
    return t_total, n_depos, n_ev, used


def run_reference(args):
    """Reference arm: the FP64 oracle (rasterize + scatter in C on every host core, scipy's FP64
    FFT convolution with one worker per core), timed on whole events of the benchmarked batch:
    step k is event k of the batch (cycling), every plane, nothing sampled or scaled."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    wl = synth.workload(PLANE_WORKLOAD)
    evs = rank_events(0, args.batch)
    resp = wl.responses()
    for w in range(args.warmup):
        oracle_events([evs[w % len(evs)]], wl.planes, wl.diffusion, resp)
    total, depos, threads = 0.0, 0, 1
    for k in range(args.steps):
        t, n, _, threads = oracle_events([evs[k % len(evs)]], wl.planes, wl.diffusion, resp)
        total += t
        depos += n
    value = depos / total
    sample = (f"per step one whole event of the {args.batch}-event batch (events 0..{args.steps - 1} in order, "
              f"{depos} depos in total), all 3 planes: C FP64 rasterize + scatter on {threads} threads (depos "
              f"spread over threads; each thread owns a band of wires in the scatter) and the scipy FP64 FFT "
              f"convolution with {threads} workers")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "depos/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "planes": "3 x (2400/2400/3456 wires x 9600 ticks)",
                   "events_per_batch": args.batch, "depos_per_event": "lognormal 10k-500k",
                   "fluctuation": True, "events_per_step": 1},
        "events_per_s": args.steps / total,
        "cpu_baseline": {"value": value, "unit": "depos/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "depos/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
# extra measurements (rank 0, one GPU)
# --------------------------------------------------------------------------------------------
def measure_single_event(reps=5):
    """The full three-plane event (1M depos: 800k on 200 tracks + 200k isolated) through
    run_event, device time per event (CUDA events), against the same event through run_batch."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload(PLANE_WORKLOAD)
    d = pkg.DeviceDepos.from_host(wl.depos(event_id=77))
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    outs = [torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, device="cuda") for p in wl.planes]
    st = torch.cuda.current_stream()
    sim.run_event(d, outs)
    torch.cuda.synchronize()
    lat = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.run_event(d, outs)
        b.record(st)
        torch.cuda.synchronize()
        lat.append(a.elapsed_time(b))
    t_batch = cuda_timed(lambda: sim.run_batch([d], [outs]), reps, warm=2)
    sim.sync()
    sim.close()
    med = statistics.median(lat)
    return {"workload": "one three-plane event, 2400/2400/3456 x 9600, 1M depos (200 tracks + 20% isolated)",
            "run_event_ms_p50": med, "run_event_ms_max": max(lat), "events_per_s": 1e3 / med,
            "depos_per_s": d.n * 1e3 / med, "run_batch_ms": 1e3 * t_batch}


def measure_uboone(n_events=16, reps=10):
    """The single MicroBooNE-sized plane (3456 x 9600, 100k depos on 20 tracks): a 16-event
    run_batch (events/s, depos/s) and the per-kernel times of run_event with their HBM fractions
    (the convolution's three kernels against the unpadded half-spectrum bytes)."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload("uboone_plane")
    pl = wl.planes[0]
    evs = [pkg.DeviceDepos.from_host(wl.depos(seed=wl.seed + e, event_id=e)) for e in range(n_events)]
    outs = [[torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.float32, device="cuda")] for _ in evs]
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    t = cuda_timed(lambda: sim.run_batch(evs, outs), reps, warm=3)
    sim.set_timing(True)
    for e, o in zip(evs, outs):
        sim.run_event(e, o)
    sim.sync()
    st = sim.stage_times()
    # the batch's convolutions (two streams), timed on their streams
    sim.set_timing(True)
    sim.run_batch(evs, outs)
    sim.sync()
    conv_batch_us = sim.stage_times()["batch_convolve"] / n_events
    sim.set_timing(False)
    peak, _, kind = measured_peaks()
    sb = stage_bytes(pl, wl.n_depos, sim.plane_info(0)["spectrum_bins_used"])
    unp, classical = unpruned_convolve_bytes(pl)
    conv_us = st["row_r2c"] + st["wire_stage"] + st["row_c2r"]
    sim.close()
    kern = {}
    for k in ("row_r2c", "wire_stage", "row_c2r"):
        gbs = sb[k] / (st[k] * 1e-6) / 1e9
        kern[k] = {"us": round(st[k], 2), "alg_bytes": sb[k], "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4)}
    return {"workload": "uboone_plane: 1 plane 3456 x 9600, 100k depos, 16-event run_batch",
            "events_per_s": n_events / t, "depos_per_s": n_events * wl.n_depos / t,
            "raster_scatter_us": round(st["raster_scatter"], 1), "kernels": kern,
            "convolve_us": round(conv_us, 1),
            "convolve_frac_unpruned": round(unp / (conv_us * 1e-6) / 1e9 / peak, 4),
            "convolve_batched_us_per_event": round(conv_batch_us, 1),
            "convolve_batched_frac_unpruned": round(unp / (conv_batch_us * 1e-6) / 1e9 / peak, 4),
            "convolve_frac_supported_bins": round(sb["convolve"] / (conv_us * 1e-6) / 1e9 / peak, 4),
            "convolve_unpruned_bytes": unp, "classical_3pass_bytes": classical,
            "peak_source": f"{kind} (burst copy)"}


def measure_impact(n_events=4, reps=2):
    """Impact mode (per-impact-position responses, 10 phases) on the uboone_plane workload:
    run_event per event, CUDA events around reps x n_events events, against the folded mode."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload("uboone_plane")
    pl = wl.planes[0]
    evs = [pkg.DeviceDepos.from_host(wl.depos(seed=wl.seed + 100 + e, event_id=500 + e)) for e in range(n_events)]
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    out = torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.float32, device="cuda")

    def timed():
        return cuda_timed(lambda: [sim.run_event(d, [out]) for d in evs], reps, warm=1) / n_events

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
    return {"workload": "uboone_plane, 10 per-impact-position responses (21 x 200 each)",
            "events_per_s": 1.0 / t_impact, "depos_per_s": n / t_impact, "ms_per_event": 1e3 * t_impact,
            "folded_ms_per_event": 1e3 * t_folded,
            "stages_us": {"patches_rasterize_scatter": round(stages["raster_scatter"] + stages["prep_binning"], 1),
                          "phase_transforms": round(stages["row_r2c"], 1),
                          "phase_stencils": round(stages["wire_stage"], 1),
                          "inverse_transform": round(stages["row_c2r"], 1)}}


def measure_deterministic(n_events=16, reps=5):
    """Cost of the deterministic mode (fixed-point integer accumulation, bitwise reproducible):
    one run_batch of n_events uboone_plane events on a deterministic handle against the default
    handle (graph replay after the first call)."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload("uboone_plane")
    pl = wl.planes[0]
    evs = [pkg.DeviceDepos.from_host(wl.depos(seed=wl.seed + 200 + e, event_id=700 + e)) for e in range(n_events)]
    outs = [[torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.float32, device="cuda")] for _ in evs]
    res = {}
    for det in (False, True):
        sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion, deterministic=det)
        res[det] = cuda_timed(lambda: sim.run_batch(evs, outs), reps, warm=3) / n_events
        sim.sync()
        sim.close()
    n = evs[0].n
    return {"workload": f"uboone_plane, {n_events}-event run_batch", "events_per_s": 1.0 / res[True],
            "depos_per_s": n / res[True], "default_events_per_s": 1.0 / res[False],
            "slowdown": res[True] / res[False]}


def measure_cufft(reps=10):
    """Comparison only (not on the path): the same row transforms through the vendor FFT
    (torch.fft, i.e. cuFFT) on the uboone_plane grid, full half spectrum of length P, against
    this library's forward / inverse row kernels timed inside run_event."""
    import torch
    import synth
    import paper_2304_01841_gb300 as pkg
    wl = synth.workload("uboone_plane")
    pl = wl.planes[0]
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    P = sim.plane_info(0)["fft_length"]
    g = torch.randn((pl.n_wires, pl.n_ticks), dtype=torch.float32, device="cuda")
    spec = torch.fft.rfft(g, n=P, dim=1)
    fwd = 1e6 * cuda_timed(lambda: torch.fft.rfft(g, n=P, dim=1), reps, warm=3)
    inv = 1e6 * cuda_timed(lambda: torch.fft.irfft(spec, n=P, dim=1), reps, warm=3)
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
    import ctypes
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload("uboone_plane")
    d = wl.depos()
    dd = pkg.DeviceDepos.from_host(d)
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    slot = sim.patch_slot_bins(0, float(d.x.max()))
    desc, patches = sim.rasterize(0, dd)
    total = patches.numel()
    desc_f, patches_f = sim.rasterize_fixed(0, dd, slot)
    total_c = ctypes.c_int64()
    ds = dd.c_struct()
    lib, h = sim._lib, sim._h

    def scanned():   # size query + patches, as a caller of the scanned API does it
        lib.wct_sim_rasterize(h, 0, ctypes.byref(ds), None, 0, desc.data_ptr(), ctypes.byref(total_c), None)
        lib.wct_sim_rasterize(h, 0, ctypes.byref(ds), patches.data_ptr(), total, desc.data_ptr(),
                              ctypes.byref(total_c), None)

    def fixed():
        lib.wct_sim_rasterize_fixed(h, 0, ctypes.byref(ds), patches_f.data_ptr(), slot, desc_f.data_ptr(), None)

    t_scan, t_fixed = 1e6 * cuda_timed(scanned, reps), 1e6 * cuda_timed(fixed, reps)
    sim.sync()
    sim.close()
    return {"workload": "uboone_plane, unfused rasterize with fluctuation", "slot_bins": slot,
            "scanned_us": round(t_scan, 1), "scan_free_us": round(t_fixed, 1),
            "scanned_patch_bytes": 4 * total, "scan_free_patch_bytes": 4 * d.n * slot}


def measure_digitize(reps=20):
    """Noise + digitisation of one uboone_plane waveform (3456 x 9600): algorithmic bytes 4 B
    read + 2 B written per bin."""
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    wl = synth.workload("uboone_plane")
    pl = wl.planes[0]
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    # two waveforms and two outputs used alternately: 400 MB, more than the L2
    wfs = [torch.randn((pl.n_wires, pl.n_ticks), device="cuda") * 100.0 for _ in range(2)]
    outs = [torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.int16, device="cuda") for _ in range(2)]
    k = [0]

    def step():
        sim.digitize(0, wfs[k[0] % 2], 1.0, 900.0, 2.5, out=outs[k[0] % 2], event_id=k[0])
        k[0] += 1

    us = 1e6 * cuda_timed(step, reps, warm=3)
    sim.sync()
    sim.close()
    peak, _, kind = measured_peaks()
    gbs = 6.0 * pl.n_wires * pl.n_ticks / (us * 1e-6) / 1e9
    return {"workload": "uboone_plane waveform, 12-bit codes with white noise", "us": round(us, 2),
            "alg_bytes": 6 * pl.n_wires * pl.n_ticks, "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
            "peak_source": f"{kind} (burst copy)"}


def measure_serving(n_events=120, loads=(0.5, 0.8, 0.95)):
    """Served: APA-like planes (800/800/960 x 6000), heavy-tailed depo counts (90% 5k-50k,
    10% 1M-3M), host depos in pinned memory.  Capacity (everything submitted at once) and
    open-loop Poisson arrivals at fractions of it, against the same events one at a time
    (upload, run_event, wait, next event) on one stream."""
    import numpy as np
    import torch
    import paper_2304_01841_gb300 as pkg
    import synth
    from paper_2304_01841_gb300.serve import EventServer, pin_depos, run_open_loop
    wl = synth.workload("dune_apa")
    pool = [wl.depos(n_depos=3_000_000, seed=wl.seed + k) for k in range(2)]
    counts = synth.serving_depo_counts(n_events)
    host = synth.slice_events(pool, counts, np.random.default_rng(9), 9000)
    evs = [pin_depos(e) for e in host]
    # one event at a time: the same work (upload, all planes, result ready) serialised
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion)
    outs = [torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, device="cuda") for p in wl.planes]

    def one(e):
        d = pkg.DeviceDepos(*(getattr(e, k).to("cuda", non_blocking=True) for k in ("t0", "x", "y", "z", "q")),
                            event_id=e.event_id)
        sim.run_event(d, outs)
        torch.cuda.current_stream().synchronize()

    for e in evs[:8]:
        one(e)
    t0 = time.perf_counter()
    for e in evs:
        one(e)
    t_one = time.perf_counter() - t0
    sim.sync()
    sim.close()
    srv = EventServer(wl.planes, wl.responses(), wl.diffusion, n_slots=4, max_batch=8,
                      hbm_budget_bytes=24 << 30)
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
            "events": len(evs), "depos": int(sum(int(c) for c in counts)),
            "capacity_events_per_s": cap, "events_per_s_one_at_a_time": len(evs) / t_one,
            "served_over_one_at_a_time": cap * t_one / len(evs), "open_loop": points,
            "what": "latency = host submit -> completion seen by the scheduler; heavy (>= 500k-depo) events run "
                    "alone on a low-priority slot, light ones in batches of <= 8 events / 400k depos"}


# --------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.steps < 1 or args.warmup < 0 or args.batch < 1:
        raise SystemExit("bench.py: --steps and --batch must be >= 1, --warmup >= 0")
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
    wl = synth.workload(PLANE_WORKLOAD)
    E = args.batch
    host_events = rank_events(rank, E)
    depos_per_batch = int(sum(e.n for e in host_events))
    sim = pkg.Simulator(wl.planes, wl.responses(), wl.diffusion, schedule_id=args.schedule)
    dev_events = [pkg.DeviceDepos.from_host(d) for d in host_events]
    outs = [[torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, device="cuda") for p in wl.planes]
            for _ in range(E)]
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        sim.run_batch(dev_events, outs)
    sim.sync()
    torch.cuda.synchronize()

    # ---- timed region: K steps, each one run_batch of the E resident events -------------
    # (one persistent raster launch over every event and plane, then the convolutions of all
    # grids; replayed from a recorded CUDA graph from the second call on; every step recomputes
    # everything)
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
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    start.record(stream)
    for k in range(K):
        sim.run_batch(dev_events, outs)
        marks[k].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    sim.sync()
    elapsed_ms = start.elapsed_time(stop)
    step_ms = sorted([start.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, K)])
    launches = sim.counters()["kernel_launches"] - launches0
    elapsed_ms = max_over_ranks(elapsed_ms, world, "cuda")
    value = world * K * depos_per_batch / (elapsed_ms / 1000.0)
    events_per_s = world * K * E / (elapsed_ms / 1000.0)

    # ---- the same events one run_event at a time (no overlap between events) ------------
    t_one = cuda_timed(lambda: [sim.run_event(d, o) for d, o in zip(dev_events, outs)], 1, warm=1)
    sim.sync()

    # ---- per-event latency: run_event as a caller runs it, CUDA events on the launching
    # stream around each event -----------------------------------------------------------
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(E + 1)]
    ev[0].record(stream)
    for i in range(E):
        sim.run_event(dev_events[i], outs[i])
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    lat = sorted(ev[j].elapsed_time(ev[j + 1]) for j in range(E))
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    # ---- the same through a stream of the highest priority: run_event then convolves each
    # plane on one of two library streams of that priority while the next plane is rasterized
    try:
        top = torch.cuda.Stream.priority_range()[1]
    except Exception:
        top = -1
    hp = torch.cuda.Stream(priority=top)
    hp.wait_stream(stream)
    evh = [torch.cuda.Event(enable_timing=True) for _ in range(E + 1)]
    for i in range(min(2, E)):
        sim.run_event(dev_events[i], outs[i], stream=hp)
    evh[0].record(hp)
    for i in range(E):
        sim.run_event(dev_events[i], outs[i], stream=hp)
        evh[i + 1].record(hp)
    hp.synchronize()
    sim.sync(stream=hp)
    stream.wait_stream(hp)
    lat_hp = sorted(evh[j].elapsed_time(evh[j + 1]) for j in range(E))
    latency_hp = {"p50": lat_hp[len(lat_hp) // 2],
                  "p99": lat_hp[min(len(lat_hp) - 1, int(math.ceil(0.99 * len(lat_hp))) - 1)],
                  "events_per_s": E * 1e3 / sum(lat_hp), "stream_priority": top,
                  "what": "as latency_ms, on a stream of the highest priority (convolutions on two streams)"}
    # ---- per-kernel times: the same events with the library's stage timing on (the planes
    # then run one after the other on the stream, so each kernel's time is its own) --------
    sim.set_timing(True)
    for i in range(E):
        sim.run_event(dev_events[i], outs[i])
    torch.cuda.synchronize()
    sim.sync()
    st_ev = sim.stage_times()
    # ---- the batch's persistent raster launch and its convolutions, timed on their streams
    sim.set_timing(True)
    sim.run_batch(dev_events, outs)
    sim.sync()
    st_b = sim.stage_times()
    sim.set_timing(False)

    # ---- work counts of the rasterizer from the library's own windows (patch descriptors):
    # one normal per impact bin (fluctuation on), one erf per bin edge of each axis ---------
    normals = erfs = 0
    for d in dev_events:
        for p in range(len(wl.planes)):
            desc, _ = sim.rasterize(p, d, with_patches=False)
            dn = desc.cpu().numpy().astype(np.int64)
            ok = dn[:, 3] > 0
            normals += int((dn[ok, 3] * dn[ok, 4]).sum())
            erfs += int((dn[ok, 3] + dn[ok, 4] + 2).sum())
    sim.sync()

    # ---- roofline of the dominant kernel -----------------------------------------------
    peak_gbs, sm_mhz_max, peak_kind = measured_peaks()
    issue_peak = N_SMS * ISSUE_PER_SM_CLK * sm_mhz_max * 1e6          # warp-instructions / s
    raster_us, conv_us_b = st_b["batch_raster"], st_b["batch_convolve"]
    cnt = kernel_counters()
    valid = cnt.get("csrc_digest") == csrc_digest() and cnt.get("workload") == WORKLOAD
    kcnt = cnt.get("kernels", {}) if valid else {}
    kc = kcnt.get("k_raster_batch_persistent", {})
    insts = kc.get("warp_instructions_per_launch")
    ach = insts / (raster_us * 1e-6) if (insts and raster_us > 0) else None
    # per-kernel totals of one batch: the raster launch, and each convolution kernel summed over
    # the 192 grids (run_event's per-event kernel times x E)
    per_batch = {"k_raster_batch_persistent": raster_us, "k_row_r2c_pair": st_ev["row_r2c"] * E,
                 "k_wire_stage_tma": st_ev["wire_stage"] * E, "k_row_c2r_pair": st_ev["row_c2r"] * E}
    dominant = max(per_batch, key=per_batch.get)
    bytes_ev = {k: 0 for k in ("row_r2c", "wire_stage", "row_c2r", "convolve")}
    unpruned = classical = 0
    for p, pl in enumerate(wl.planes):
        sb = stage_bytes(pl, 0, sim.plane_info(p)["spectrum_bins_used"])
        for k in bytes_ev:
            bytes_ev[k] += sb[k]
        u, c = unpruned_convolve_bytes(pl)
        unpruned += u
        classical += c
    grid_bytes = sum(4 * p.n_wires * p.n_ticks for p in wl.planes)
    kernels = {}
    for k, name in (("row_r2c", "k_row_r2c_pair"), ("wire_stage", "k_wire_stage_tma"), ("row_c2r", "k_row_c2r_pair")):
        us = st_ev[k]
        gbs = bytes_ev[k] / (us * 1e-6) / 1e9 if us > 0 else None
        kernels[name] = {"us_per_event": round(us, 2), "alg_bytes_per_event": bytes_ev[k],
                         "GB/s": round(gbs, 1) if gbs else None, "frac": round(gbs / peak_gbs, 4) if gbs else None}
    conv_ev_us = st_ev["row_r2c"] + st_ev["wire_stage"] + st_ev["row_c2r"]
    raster_report = {"us_per_batch": round(raster_us, 1), "launches_per_batch": 1, "bound": "alu",
                     "normals_per_batch": normals, "erf_per_batch": erfs,
                     "normals_per_s": normals / (raster_us * 1e-6) if raster_us > 0 else None,
                     "erf_per_s": erfs / (raster_us * 1e-6) if raster_us > 0 else None,
                     "warp_inst_per_launch": insts,
                     "warp_inst_per_s": ach, "frac_of_issue_peak": round(ach / issue_peak, 4) if ach else None,
                     "depo_read_plus_grid_write_GB/s": round((20 * depos_per_batch * len(wl.planes) + E * grid_bytes)
                                                            / (raster_us * 1e-6) / 1e9, 1) if raster_us > 0 else None}
    if dominant == "k_raster_batch_persistent":
        roofline = {"bound": "alu", "kernel": dominant, "achieved": ach, "peak": issue_peak, "unit": "warp-inst/s",
                    "frac": round(ach / issue_peak, 4) if ach else None,
                    "traffic": kc.get("dram_bytes_per_launch"),
                    "peak_source": f"issue rate: {N_SMS} SMs x {ISSUE_PER_SM_CLK} warp-inst/clk x {sm_mhz_max:.0f} MHz "
                                   f"(max SM clock, {peak_kind}); instructions per launch from the committed ncu "
                                   f"capture of this launch (profiles/kernel_counters.json)",
                    "normals_per_s": raster_report["normals_per_s"], "erf_per_s": raster_report["erf_per_s"]}
    else:
        k = {"k_row_r2c_pair": "row_r2c", "k_wire_stage_tma": "wire_stage", "k_row_c2r_pair": "row_c2r"}[dominant]
        achieved = bytes_ev[k] / (st_ev[k] * 1e-6) / 1e9
        roofline = {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1), "peak": peak_gbs,
                    "unit": "GB/s", "frac": round(achieved / peak_gbs, 4),
                    "traffic": kcnt.get(dominant, {}).get("dram_bytes_per_launch"),
                    "peak_source": f"{peak_kind} (burst copy)"}
    stages = {
        "batch_raster_launch": raster_report,
        "batch_convolutions_us": round(conv_us_b, 1),
        "batch_convolutions_frac_unpruned": round(E * unpruned / (conv_us_b * 1e-6) / 1e9 / peak_gbs, 4)
        if conv_us_b > 0 else None,
        "per_batch_kernel_us": {k: round(v, 1) for k, v in per_batch.items()},
        "convolve_kernels_run_event": kernels,
        "convolve_total_run_event": {
            "us_per_event": round(conv_ev_us, 1), "alg_bytes_per_event": bytes_ev["convolve"],
            "frac": round(bytes_ev["convolve"] / (conv_ev_us * 1e-6) / 1e9 / peak_gbs, 4),
            "unpruned_bytes_per_event": unpruned,
            "unpruned_frac": round(unpruned / (conv_ev_us * 1e-6) / 1e9 / peak_gbs, 4),
            "classical_3pass_bytes_per_event": classical},
        "raster_scatter_run_event_us": round(st_ev["raster_scatter"], 1),
    }

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
        host_sets = [[torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32).pin_memory() for p in wl.planes]
                     for _ in range(2)]
        outs_host = [host_sets[e % 2] for e in range(E)]
        h2d = 20 * depos_per_batch
        d2h = E * grid_bytes

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
        e2e_ms = max_over_ranks(s0.elapsed_time(s1), world, "cuda")
        e2e = {"value": world * K * depos_per_batch / (e2e_ms / 1000.0), "unit": "depos/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "events_per_s": world * K * E / (e2e_ms / 1000.0),
               "d2h_GBps": round(d2h * K / (e2e_ms * 1e-3) / 1e9, 1),
               "what": "wct_sim_run_host: pinned host depos -> device -> pinned host waveforms (3 planes), every "
                       "event of the batch; uploads / downloads overlap the kernels; bound by the 317 MB download "
                       "per event"}

    # ---- CPU baseline: the FP64 oracle on whole events of this batch ------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        resp = wl.responses()
        t_all, n_all, ev_all, threads = oracle_events(host_events, wl.planes, wl.diffusion, resp, budget_s=CPU_SAMPLE_S)
        small = min(host_events, key=lambda e: e.n)
        t_one_cpu, n_one, _, _ = oracle_events([small], wl.planes, wl.diffusion, resp, threads=1)
        cpu = {"value": n_all / t_all, "unit": "depos/s", "cores": threads, "kind": "oracle",
               "events_per_s": ev_all / t_all, "value_one_thread": n_one / t_one_cpu, "cores_one_thread": 1,
               "sample": f"whole events of this batch, all 3 planes, in batch order until {CPU_SAMPLE_S:.0f} s had "
                         f"passed: {ev_all} events, {n_all} depos, {t_all:.1f} s on {threads} threads (C FP64 "
                         f"rasterize + scatter over all threads, scipy FP64 FFT with {threads} workers); one thread: "
                         f"the batch's smallest event ({n_one} depos), {t_one_cpu:.1f} s"}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["single_event_1M"] = measure_single_event()
        extras["uboone_plane"] = measure_uboone()
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
            "config": {"workload": WORKLOAD,
                       "planes": "3: 2400 / 2400 / 3456 wires x 9600 ticks (0.5 us), +60 / -60 / 0 deg",
                       "events_per_step": E, "depos_per_step": depos_per_batch,
                       "depos_per_event": "lognormal, 10k / 500k at the 1st / 99th percentiles",
                       "depo_mix": "200 straight tracks + 20% isolated low-charge depos (per 500k-depo pool event)",
                       "fluctuation": True, "response": "21 x 200 (bipolar U/V, unipolar W)",
                       "events_resident_in_hbm": E,
                       "l2": "every event has its own 317 MB of grids and 317 MB of waveforms (> 126 MB L2) and a "
                             "step cycles through 64 events: no flush needed"},
            "events_per_s": events_per_s,
            "step_ms": {"median": step_ms[len(step_ms) // 2],
                        "p99": step_ms[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)],
                        "min": step_ms[0], "max": step_ms[-1],
                        "what": "device time of each timed step on this rank (CUDA events on the launching stream)"},
            "one_at_a_time": {"events_per_s": E / t_one, "depos_per_s": depos_per_batch / t_one,
                              "batched_over_one_at_a_time": events_per_s / world / (E / t_one)},
            "latency_ms": {"p50": p50, "p99": p99,
                           "what": "device time of one event of the batch through run_event, events back to back"},
            "latency_ms_priority_stream": latency_hp,
            "roofline": roofline,
            "stages": stages,
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
