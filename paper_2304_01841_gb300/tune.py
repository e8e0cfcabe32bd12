"""Schedule autotuning with a persistent cache.

The library has several kernel schedules per handle (wct_opts_t::schedule_id: the row
transforms' form and the rasterizer's granularity; for run_batch, the events per persistent
raster launch and the number of convolution streams).  `autotune` times one event through
`run_event` under each candidate schedule on the current device and keeps the fastest;
`autotune_batch` does the same for a batch through `run_batch`.  The choice is cached in a JSON
file keyed by the device name and the planes' geometry (and the batch size), so later processes
reuse it without timing again (`Simulator(..., schedule_id=best)`).

The timing and handle creation go through callables so the selection and the cache can be
tested without a GPU.
"""
from __future__ import annotations

import json
import os
import statistics
import tempfile
from typing import Callable, Dict, Optional, Sequence

# -1: paired row transforms with composite radices (the default); 4: paired, radices <= 8;
# 1: one persistent row CTA per SM; 0: register-staged rows; +2: CTA-level rasterizer
CANDIDATES = (-1, 4, 1, 0, 6)


# run_batch candidates (bit 3: paired composite row transforms, the default's): -1 the default
# (one raster launch for the whole batch, two convolution streams); +256 one convolution
# stream; +512 three; (v << 4): 2^(v-1) events per raster launch, pipelined with the previous
# launch's convolutions
BATCH_CANDIDATES = (-1, 8 | 256, 8 | 512, 8 | (5 << 4), 8 | (4 << 4))


def default_cache_path() -> str:
    p = os.environ.get("WCT_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "wct_gb300", "tune.json")


def tune_key(device: str, planes: Sequence, deterministic: bool = False) -> str:
    geo = ";".join(f"{p.n_wires}x{p.n_ticks}x{p.n_impact_per_pitch}" for p in planes)
    return f"{device}|{geo}|det={int(bool(deterministic))}"


class TuneCache:
    """JSON file of {key: {"schedule_id": int, "ms": {schedule: median ms}}}; written atomically."""

    def __init__(self, path: Optional[str] = None):
        self.path = path or default_cache_path()
        self.entries: Dict[str, dict] = {}
        try:
            with open(self.path) as f:
                data = json.load(f)
            if isinstance(data, dict):
                self.entries = data
        except (OSError, ValueError):
            self.entries = {}

    def get(self, key: str) -> Optional[int]:
        e = self.entries.get(key)
        return int(e["schedule_id"]) if isinstance(e, dict) and "schedule_id" in e else None

    def put(self, key: str, schedule_id: int, ms: Dict[int, float]) -> None:
        self.entries[key] = {"schedule_id": int(schedule_id), "ms": {str(k): float(v) for k, v in ms.items()}}
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _cuda_timer(sim, depos, reps: int) -> float:
    """Median device time (ms) of run_event on `depos` after one warm-up call."""
    import torch
    st = torch.cuda.current_stream()
    sim.run_event(depos)
    sim.sync()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.run_event(depos)
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
    sim.sync()
    return statistics.median(times)


def autotune(planes, responses, diffusion, depos, candidates: Sequence[int] = CANDIDATES, reps: int = 5,
             deterministic: bool = False, cache: Optional[TuneCache] = None, device: Optional[str] = None,
             make_sim: Optional[Callable] = None, timer: Optional[Callable] = None) -> int:
    """The fastest schedule_id among `candidates` for these planes on this device (from the cache
    when present, else measured on `depos`, a DeviceDepos, and stored).  Deterministic handles
    always use the warp-level rasterizer, so +2 variants are skipped for them."""
    if device is None:
        import torch
        device = torch.cuda.get_device_name()
    cache = cache if cache is not None else TuneCache()
    key = tune_key(device, planes, deterministic)
    hit = cache.get(key)
    if hit is not None:
        return hit
    if make_sim is None:
        from . import Simulator

        def make_sim(sched):
            return Simulator(planes, responses, diffusion, schedule_id=sched, deterministic=deterministic)
    timer = timer or _cuda_timer
    cands = [c for c in candidates if not (deterministic and c >= 0 and (c & 2))]
    ms: Dict[int, float] = {}
    for c in cands:
        sim = make_sim(c)
        try:
            ms[c] = float(timer(sim, depos, reps))
        finally:
            close = getattr(sim, "close", None)
            if close:
                close()
    best = min(ms, key=lambda c: (ms[c], cands.index(c)))
    cache.put(key, best, ms)
    return best


def _cuda_batch_timer(sim, events, reps: int) -> float:
    """Median device time (ms) of run_batch on `events` after two warm-up calls (the second
    records the batch's graph, later calls replay it)."""
    import torch
    st = torch.cuda.current_stream()
    outs = sim.run_batch(events)
    sim.run_batch(events, outs)
    sim.sync()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sim.run_batch(events, outs)
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
    sim.sync()
    return statistics.median(times)


def autotune_batch(planes, responses, diffusion, events, candidates: Sequence[int] = BATCH_CANDIDATES, reps: int = 3,
                   deterministic: bool = False, cache: Optional[TuneCache] = None, device: Optional[str] = None,
                   make_sim: Optional[Callable] = None, timer: Optional[Callable] = None) -> int:
    """The fastest run_batch schedule_id among `candidates` for a batch of len(events) events
    (DeviceDepos) on these planes (from the cache when present, else measured and stored)."""
    if device is None:
        import torch
        device = torch.cuda.get_device_name()
    cache = cache if cache is not None else TuneCache()
    key = "batch|" + tune_key(device, planes, deterministic) + f"|events={len(events)}"
    hit = cache.get(key)
    if hit is not None:
        return hit
    if make_sim is None:
        from . import Simulator

        def make_sim(sched):
            return Simulator(planes, responses, diffusion, schedule_id=sched, deterministic=deterministic)
    timer = timer or _cuda_batch_timer
    ms: Dict[int, float] = {}
    for c in candidates:
        sim = make_sim(c)
        try:
            ms[c] = float(timer(sim, events, reps))
        finally:
            close = getattr(sim, "close", None)
            if close:
                close()
    best = min(ms, key=lambda c: (ms[c], list(candidates).index(c)))
    cache.put(key, best, ms)
    return best
