"""Continuous-batching event server over the CUDA library.

Requests (one event's depos each, in host memory) arrive at any time.  The scheduler keeps
`n_slots` slots; each slot owns a simulator handle (its own scratch) and a CUDA stream, so
slots run concurrently on the device.  Whenever a slot is free, the scheduler admits pending
requests whose device memory (depo arrays + waveforms) fits the remaining HBM budget, copies
their depos to the device and launches them as one batch (rasterize + scatter and the
convolutions, wct_sim_run_batch) on that slot's stream.  A request that arrives while others
are on the GPU is admitted as soon as a slot and memory free up.  Latency is submit ->
completion observed on the host.

Admission is size aware, so that small events never wait behind a large one:
  - a request of at least `heavy_depos` depos is heavy: it runs in a batch of its own on a
    low-priority stream, on one of the last `heavy_slots` slots (or on an idle light slot, see
    below);
  - light requests are batched in arrival order (skipping heavy ones) up to `max_batch`
    requests and `max_batch_depos` depos per batch, on high-priority streams, so the device's
    block scheduler runs their kernels ahead of a heavy event's whenever SMs free up;
  - a heavy slot with no heavy request pending takes a light batch; a light slot with no light
    request pending takes a heavy request as long as another slot stays free for light
    traffic; heavy requests are admitted in arrival order among themselves.

The results of a request do not depend on what it was batched with: the fluctuation stream is
keyed by (seed, event id, plane, depo index, bin), so each event is the same alone and in a mix
up to the FP32 summation order of the scatter.

The scheduling logic (admission, budget, FIFO order) is independent of the device: the device
work goes through a backend object (`CudaBackend` here; tests drive the scheduler with a fake).

Failures stay with their batch: if a backend's launch or retire raises (an invalid event, an
allocation beyond the budget, a device error reported at sync), every request of that batch
completes with `error` set, its memory is released and the server carries on with the others.
A pending request can be cancelled (it is never launched); cancelling one already on the
device only drops its results.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field
from typing import Deque, List, Optional, Sequence

import numpy as np


@dataclass
class Request:
    rid: int
    depos: object                    # host-side SoA (t0, x, y, z, q arrays, event_id)
    t_submit: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    waveforms: Optional[List] = None   # host float32 arrays, one per plane (if keep_results)
    done: threading.Event = field(default_factory=threading.Event)
    cancelled: bool = False            # cancel() was called: no results are kept
    error: Optional[BaseException] = None   # the device work of its batch failed

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


def _host_tensor(torch, a):
    # pinned host tensors are copied asynchronously; numpy arrays are pinned here
    if isinstance(a, torch.Tensor):
        return a
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()


def pin_depos(d):
    """Host depos with their arrays moved to pinned memory (for asynchronous uploads)."""
    import torch
    out = type("PinnedDepos", (), {})()
    for k in ("t0", "x", "y", "z", "q"):
        setattr(out, k, _host_tensor(torch, getattr(d, k)))
    out.event_id = int(d.event_id)
    return out


class CudaBackend:
    """Device side of a slot: a simulator handle and a stream."""

    def __init__(self, planes, responses, diffusion, keep_results: bool, heavy_depos: int = 500_000):
        import torch
        from . import Simulator
        self.torch = torch
        self.planes = list(planes)
        self.sim = Simulator(planes, responses, diffusion)
        # lower numbers run first: light batches on a high-priority stream (the library's own
        # batch streams follow its priority), heavy events on a low-priority one
        self.stream_light = torch.cuda.Stream(priority=-2)
        self.stream_heavy = torch.cuda.Stream(priority=0)
        self.stream = self.stream_light
        self.heavy_depos = int(heavy_depos)
        self.keep = keep_results
        self.dev, self.outs, self.host, self.event = [], [], [], None

    def launch(self, batch: List[Request]):
        from . import DeviceDepos
        torch = self.torch
        heavy = len(batch) == 1 and int(len(batch[0].depos.t0)) >= self.heavy_depos
        self.stream = self.stream_heavy if heavy else self.stream_light
        with torch.cuda.stream(self.stream):
            self.dev = []
            for r in batch:
                d = r.depos
                dev = [_host_tensor(torch, a).to("cuda", non_blocking=True) for a in (d.t0, d.x, d.y, d.z, d.q)]
                self.dev.append(DeviceDepos(*dev, event_id=int(d.event_id)))
            self.outs = [[torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, device="cuda")
                          for p in self.planes] for _ in batch]
            if len(batch) == 1:
                # one event (e.g. a heavy one, alone on a low-priority slot): run_event, whose
                # rasterizer is a plain grid of short CTAs, so higher-priority work from other
                # slots takes over SMs as its CTAs finish (the batch's persistent raster launch
                # would hold every SM until it is done); on the high-priority stream it also
                # convolves the planes on two streams, on the low-priority one it keeps to one
                self.sim.run_event(self.dev[0], self.outs[0], stream=self.stream)
            else:
                self.sim.run_batch(self.dev, self.outs, stream=self.stream)
            if self.keep:
                self.host = [[o.to("cpu", non_blocking=True) for o in ev] for ev in self.outs]
            self.event = torch.cuda.Event()
            self.event.record(self.stream)

    def done(self) -> bool:
        return self.event is not None and self.event.query()

    def retire(self, batch: List[Request]):
        self.sim.sync(stream=self.stream)
        if self.keep:
            for r, h in zip(batch, self.host):
                r.waveforms = [x.numpy() for x in h]
        self.dev, self.outs, self.host, self.event = [], [], [], None

    def close(self):
        self.sim.close()


class _Slot:
    def __init__(self, backend, heavy: bool):
        self.backend = backend
        self.heavy = heavy               # runs heavy requests (alone, at low priority)
        self.batch: List[Request] = []
        self.bytes = 0


class EventServer:
    def __init__(self, planes, responses, diffusion, n_slots: int = 4, max_batch: int = 8,
                 hbm_budget_bytes: int = 16 << 30, keep_results: bool = False, backend_factory=None,
                 heavy_depos: int = 500_000, max_batch_depos: int = 400_000, heavy_slots: Optional[int] = None):
        self.planes = list(planes)
        if heavy_slots is None:
            heavy_slots = 1 if n_slots > 1 else 0
        heavy_slots = max(0, min(heavy_slots, n_slots))
        n_light = n_slots - heavy_slots

        def make():
            if backend_factory is not None:
                return backend_factory()
            return CudaBackend(planes, responses, diffusion, keep_results, heavy_depos=heavy_depos)

        self.slots = [_Slot(make(), i >= n_light) for i in range(n_slots)]
        self.heavy_depos = int(heavy_depos)
        self.max_batch_depos = int(max_batch_depos)
        self.max_batch = max_batch
        self.budget = int(hbm_budget_bytes)
        self.in_use = 0
        self.pending: Deque[Request] = collections.deque()
        self.lock = threading.Lock()
        self.completed: List[Request] = []
        self._next = 0
        self.plane_bytes = sum(4 * p.n_wires * p.n_ticks for p in self.planes)

    # -- request side ------------------------------------------------------------------------
    def submit(self, depos) -> Request:
        with self.lock:
            r = Request(self._next, depos, t_submit=time.perf_counter())
            self._next += 1
            self.pending.append(r)
        return r

    def cancel(self, r: Request) -> bool:
        """Cancel a request: True if it was still pending (it completes now, never launched);
        False if it is already on the device or done (its results, if any, are dropped)."""
        with self.lock:
            r.cancelled = True
            if r in self.pending:
                self.pending.remove(r)
                r.t_done = time.perf_counter()
                r.done.set()
                self.completed.append(r)
                return True
        r.waveforms = None
        return False

    def _finish(self, slot: "_Slot", error: Optional[BaseException]):
        now = time.perf_counter()
        for r in slot.batch:
            r.t_done = now
            if error is not None:
                r.error = error
            if r.cancelled or error is not None:
                r.waveforms = None
            r.done.set()
            self.completed.append(r)
        self.in_use -= slot.bytes
        slot.batch, slot.bytes = [], 0

    def request_bytes(self, r: Request) -> int:
        return 20 * int(len(r.depos.t0)) + self.plane_bytes

    def is_heavy(self, r: Request) -> bool:
        return int(len(r.depos.t0)) >= self.heavy_depos

    def _fits(self, need: int, need_total: int, batch) -> bool:
        # within the budget; a request larger than the whole budget runs alone on an idle device
        return self.in_use + need_total + need <= self.budget or not (batch or self.in_use > 0)

    def _take(self, slot: "_Slot"):
        """The batch a free slot launches next (removed from pending; caller holds the lock)."""
        heavy_slots_exist = any(s.heavy for s in self.slots)
        light_waiting = any(not self.is_heavy(r) for r in self.pending)
        # a light slot helps with heavy requests only while no light request waits and another
        # slot stays free for light traffic arriving meanwhile
        spare = sum(1 for s in self.slots if not s.batch and s is not slot) >= 1
        if slot.heavy or (heavy_slots_exist and not light_waiting and spare):
            for r in self.pending:                     # the oldest heavy request, alone
                if self.is_heavy(r):
                    need = self.request_bytes(r)
                    if not self._fits(need, 0, []):
                        return [], 0                   # wait for memory; light slots carry on
                    self.pending.remove(r)
                    return [r], need
        batch: List[Request] = []
        need_total = depos = 0
        for r in list(self.pending):                   # light requests in arrival order
            if len(batch) >= self.max_batch:
                break
            heavy = self.is_heavy(r)
            if heavy and heavy_slots_exist:
                continue                               # heavy requests wait for a heavy slot
            n = int(len(r.depos.t0))
            if heavy and batch:
                continue                               # no heavy slots: it still runs alone
            if batch and depos + n > self.max_batch_depos:
                break
            need = self.request_bytes(r)
            if not self._fits(need, need_total, batch):
                break                                  # wait for memory to free up
            self.pending.remove(r)
            batch.append(r)
            need_total += need
            depos += n
            if heavy:
                break
        return batch, need_total

    # -- scheduler ---------------------------------------------------------------------------
    def step(self) -> int:
        """One scheduler pass: retire finished slots, admit pending requests into free slots.
        Returns the number of requests still pending or in flight."""
        for slot in self.slots:
            if slot.batch and slot.backend.done():
                err = None
                try:
                    slot.backend.retire(slot.batch)
                except Exception as e:          # noqa: BLE001 - the batch carries the error
                    err = e
                self._finish(slot, err)
        for slot in self.slots:
            if slot.batch:
                continue
            with self.lock:
                batch, need_total = self._take(slot) if self.pending else ([], 0)
            if not batch:
                continue
            now = time.perf_counter()
            for r in batch:
                r.t_admit = now
            slot.batch, slot.bytes = batch, need_total
            self.in_use += need_total
            try:
                slot.backend.launch(batch)
            except Exception as e:              # noqa: BLE001 - the batch carries the error
                self._finish(slot, e)
        with self.lock:
            return len(self.pending) + sum(len(s.batch) for s in self.slots)

    def drain(self):
        while self.step() > 0:
            time.sleep(0)

    def close(self):
        self.drain()
        for s in self.slots:
            s.backend.close()


def run_open_loop(server: EventServer, events: Sequence, rate_hz: float, seed: int = 0) -> dict:
    """Submit `events` with Poisson inter-arrival times at `rate_hz` while running the
    scheduler; return latency percentiles (ms) and throughput."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, len(events))
    t_next = time.perf_counter()
    reqs = []
    i = 0
    t0 = time.perf_counter()
    while i < len(events) or server.step() > 0:
        now = time.perf_counter()
        while i < len(events) and now >= t_next:
            reqs.append(server.submit(events[i]))
            t_next += gaps[i]
            i += 1
        server.step()
    t1 = time.perf_counter()
    lat = np.array([r.latency for r in reqs]) * 1e3
    return {"events": len(reqs), "offered_hz": rate_hz, "events_per_s": len(reqs) / (t1 - t0),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
