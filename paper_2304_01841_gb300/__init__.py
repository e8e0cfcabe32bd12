"""GB300-native LArTPC signal-simulation hot path (rasterize + scatter-add + FFT convolve).

The arithmetic runs in the CUDA library built from csrc/ (C ABI in include/wct_sim.h); this
package only marshals arguments to it.  PyTorch provides device memory and streams.

    sim = Simulator(planes, responses, diffusion)
    dep = DeviceDepos.from_host(depos)            # SoA float32 on the GPU
    waveforms = sim.run_event(dep)                # one [n_wires, n_ticks] float32 per plane
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import _abi
from ._abi import WctError, load  # noqa: F401

__all__ = ["Simulator", "DeviceDepos", "WctError", "load", "philox4x32_10", "FieldResponse", "load_field_response",
           "response_from_field"]


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr()) if t is not None else 0


@dataclass
class DeviceDepos:
    """One event's depos as device float32 arrays (t0 us, x/y/z mm, q electrons)."""
    t0: "object"
    x: "object"
    y: "object"
    z: "object"
    q: "object"
    event_id: int = 0

    @property
    def n(self) -> int:
        return int(self.t0.numel())

    @classmethod
    def from_host(cls, d, device="cuda", non_blocking: bool = False) -> "DeviceDepos":
        torch = _torch()
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(device, non_blocking=non_blocking)
        return cls(f(d.t0), f(d.x), f(d.y), f(d.z), f(d.q), int(getattr(d, "event_id", 0)))

    def c_struct(self) -> _abi.wct_depos_t:
        for a in (self.t0, self.x, self.y, self.z, self.q):
            if not (a.is_cuda and a.dtype == _torch().float32 and a.is_contiguous() and a.numel() == self.n):
                raise ValueError("depo arrays must be contiguous float32 CUDA tensors of equal length")
        return _abi.wct_depos_t(_ptr(self.t0), _ptr(self.x), _ptr(self.y), _ptr(self.z), _ptr(self.q),
                                self.n, int(self.event_id))


class Simulator:
    """Owns one wct_sim handle (planes, responses, diffusion) on the current CUDA device."""

    def __init__(self, planes: Sequence, responses: Sequence[np.ndarray], diffusion,
                 hbm_budget_bytes: int = 0, schedule_id: int = -1, deterministic: bool = False):
        self._lib = load()
        self.planes = list(planes)
        n = len(self.planes)
        P = (_abi.wct_plane_t * n)()
        for i, p in enumerate(self.planes):
            P[i] = _abi.wct_plane_t(p.n_wires, p.n_impact_per_pitch, p.n_ticks, p.pitch_mm, p.origin_mm,
                                    p.wire_angle_rad, p.tick_us, p.t_window0_us)
        self._resp_keep = [np.ascontiguousarray(r, dtype=np.float32) for r in responses]
        R = (_abi.wct_response_t * n)()
        for i, r in enumerate(self._resp_keep):
            R[i] = _abi.wct_response_t(r.shape[0], r.shape[1], r.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        D = _abi.wct_diffusion_t(diffusion.DL_cm2_s, diffusion.DT_cm2_s, diffusion.v_drift_mm_us, diffusion.nsigma,
                                 int(bool(diffusion.fluctuate)), int(diffusion.seed) & 0xFFFFFFFFFFFFFFFF)
        O = _abi.wct_opts_t(int(hbm_budget_bytes), int(schedule_id), int(bool(deterministic)))
        h = ctypes.c_void_p()
        rc = self._lib.wct_sim_create(P, n, R, ctypes.byref(D), ctypes.byref(O), ctypes.byref(h))
        if rc != 0:
            raise WctError(rc, "wct_sim_create failed")
        self._h = h
        self.diffusion = diffusion

    # -- helpers --------------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise WctError(rc, self._lib.wct_sim_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.wct_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plane_info(self, plane: int) -> dict:
        info = (ctypes.c_int64 * 9)()
        self._check(self._lib.wct_sim_plane_info(self._h, plane, info))
        keys = ("n_wires", "n_ticks", "fft_length", "spectrum_bins", "spectrum_row_stride", "tile_wires",
                "tile_ticks", "n_tiles", "spectrum_bins_used")
        return dict(zip(keys, (int(v) for v in info)))

    def _grid(self, plane: int, out=None):
        torch = _torch()
        p = self.planes[plane]
        if out is None:
            return torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, device="cuda")
        if out.shape != (p.n_wires, p.n_ticks) or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("grid / waveform must be contiguous float32 [n_wires, n_ticks]")
        return out

    # -- the ABI, one call each -----------------------------------------------------------
    def rasterize(self, plane: int, depos: DeviceDepos, with_patches: bool = True, stream=None):
        """wct_sim_rasterize: returns (patch_desc [n,5] int64, patches float32 or None)."""
        torch = _torch()
        desc = torch.empty((max(depos.n, 1), 5), dtype=torch.int64, device="cuda")
        total = ctypes.c_int64()
        ds = depos.c_struct()
        sh = _stream_handle(stream)
        self._check(self._lib.wct_sim_rasterize(self._h, plane, ctypes.byref(ds), None, 0, _ptr(desc),
                                                ctypes.byref(total), sh))
        if not with_patches:
            return desc[: depos.n], None
        patches = torch.empty(max(total.value, 1), dtype=torch.float32, device="cuda")
        self._check(self._lib.wct_sim_rasterize(self._h, plane, ctypes.byref(ds), _ptr(patches), patches.numel(),
                                                _ptr(desc), ctypes.byref(total), sh))
        return desc[: depos.n], patches[: total.value]

    def rasterize_fixed(self, plane: int, depos: DeviceDepos, slot_bins: int, stream=None):
        """wct_sim_rasterize_fixed: scan-free patches, depo i at offset i * slot_bins; returns
        (patch_desc [n,5] int64, patches float32 [n * slot_bins])."""
        torch = _torch()
        desc = torch.empty((max(depos.n, 1), 5), dtype=torch.int64, device="cuda")
        patches = torch.empty(max(depos.n * int(slot_bins), 1), dtype=torch.float32, device="cuda")
        ds = depos.c_struct()
        self._check(self._lib.wct_sim_rasterize_fixed(self._h, plane, ctypes.byref(ds), _ptr(patches), int(slot_bins),
                                                      _ptr(desc), _stream_handle(stream)))
        return desc[: depos.n], patches

    def patch_slot_bins(self, plane: int, x_max_mm: float) -> int:
        """wct_sim_patch_slot_bins: the fixed slot (bins) of rasterize_fixed for depos that drift
        at most x_max_mm on this plane."""
        out = ctypes.c_int64()
        self._check(self._lib.wct_sim_patch_slot_bins(self._h, plane, float(x_max_mm), ctypes.byref(out)))
        return int(out.value)

    def scatter(self, plane: int, depos: DeviceDepos, patches=None, patch_desc=None, out=None, stream=None):
        """wct_sim_scatter: fused (patches None) or from given patches; returns the grid."""
        grid = self._grid(plane, out)
        ds = depos.c_struct()
        self._check(self._lib.wct_sim_scatter(self._h, plane, ctypes.byref(ds), _ptr(patches), _ptr(patch_desc),
                                              _ptr(grid), _stream_handle(stream)))
        return grid

    def convolve(self, plane: int, grid, out=None, stream=None):
        """wct_sim_convolve: returns the waveform (may be `grid` itself if out is grid)."""
        wf = self._grid(plane, out)
        self._check(self._lib.wct_sim_convolve(self._h, plane, _ptr(grid), _ptr(wf), _stream_handle(stream)))
        return wf

    def run_event(self, depos: DeviceDepos, outs: Optional[List] = None, stream=None) -> List:
        """wct_sim_run_event: all planes of one event; returns one waveform per plane."""
        wfs = [self._grid(p, None if outs is None else outs[p]) for p in range(len(self.planes))]
        arr = (ctypes.c_void_p * len(wfs))(*[_ptr(w) for w in wfs])
        ds = depos.c_struct()
        self._check(self._lib.wct_sim_run_event(self._h, ctypes.byref(ds), arr, _stream_handle(stream)))
        return wfs

    def run_batch(self, events: Sequence[DeviceDepos], outs: Optional[List[List]] = None, stream=None):
        """wct_sim_run_batch: several events; returns [event][plane] waveforms."""
        npl = len(self.planes)
        wfs = [[self._grid(p, None if outs is None else outs[e][p]) for p in range(npl)] for e in range(len(events))]
        arr = (ctypes.c_void_p * (len(events) * npl))(*[_ptr(w) for ev in wfs for w in ev])
        evs = (_abi.wct_depos_t * max(len(events), 1))(*[e.c_struct() for e in events])
        self._check(self._lib.wct_sim_run_batch(self._h, evs, len(events), arr, _stream_handle(stream)))
        return wfs

    def digitize(self, plane: int, waveform, gain: float, baseline: float, noise_rms: float, bits: int = 12,
                 add_noise: bool = True, event_id: int = 0, out=None, stream=None):
        """wct_sim_digitize: noise + ADC codes (int16 CUDA tensor [n_wires, n_ticks])."""
        torch = _torch()
        wf = self._grid(plane, waveform)
        pl = self.planes[plane]
        if out is None:
            out = torch.empty((pl.n_wires, pl.n_ticks), dtype=torch.int16, device="cuda")
        elif out.shape != (pl.n_wires, pl.n_ticks) or out.dtype != torch.int16 or not out.is_contiguous():
            raise ValueError("adc output must be contiguous int16 [n_wires, n_ticks]")
        a = _abi.wct_adc_t(float(gain), float(baseline), float(noise_rms), int(bits), int(bool(add_noise)))
        self._check(self._lib.wct_sim_digitize(self._h, plane, _ptr(wf), _ptr(out), ctypes.byref(a),
                                               int(event_id) & 0xFFFFFFFFFFFFFFFF, _stream_handle(stream)))
        return out

    def set_noise_spectrum(self, plane: int, amplitude: Optional[np.ndarray]):
        """wct_sim_set_noise_spectrum: coloured-noise amplitudes per spectrum bin (None: white)."""
        if amplitude is None:
            self._check(self._lib.wct_sim_set_noise_spectrum(self._h, plane, None, 0))
            return
        a = np.ascontiguousarray(amplitude, dtype=np.float32)
        self._check(self._lib.wct_sim_set_noise_spectrum(self._h, plane, a.ctypes.data, int(a.size)))

    def set_lifetime(self, lifetime_us: float, fluctuate: bool = False):
        """wct_sim_set_lifetime: electron-lifetime attenuation of the drifting charge (<= 0: off)."""
        self._check(self._lib.wct_sim_set_lifetime(self._h, float(lifetime_us), int(bool(fluctuate))))

    def set_impact_responses(self, plane: int, responses: Optional[np.ndarray]):
        """wct_sim_set_impact_responses: per-impact-position responses [phase][wire][tick] for one
        plane (None: back to the folded mode)."""
        if responses is None:
            self._check(self._lib.wct_sim_set_impact_responses(self._h, plane, None, 0))
            return
        r = np.ascontiguousarray(responses, dtype=np.float32)
        if r.ndim != 3:
            raise ValueError("impact responses must be [phase][wire][tick]")
        R = (_abi.wct_response_t * r.shape[0])()
        for p in range(r.shape[0]):
            R[p] = _abi.wct_response_t(r.shape[1], r.shape[2], r[p].ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        self._check(self._lib.wct_sim_set_impact_responses(self._h, plane, R, r.shape[0]))

    def convolve_impact(self, plane: int, phase_grids, out=None, stream=None):
        """wct_sim_convolve_impact: phase grids [phase][wire][tick] (CUDA float32) -> waveform."""
        pl = self.planes[plane]
        if not (phase_grids.is_cuda and phase_grids.is_contiguous() and phase_grids.dim() == 3 and
                tuple(phase_grids.shape[1:]) == (pl.n_wires, pl.n_ticks)):
            raise ValueError("phase grids must be a contiguous CUDA float32 [phase, n_wires, n_ticks] tensor")
        wf = self._grid(plane, out)
        self._check(self._lib.wct_sim_convolve_impact(self._h, plane, _ptr(phase_grids), _ptr(wf),
                                                      _stream_handle(stream)))
        return wf

    def run_host(self, events: Sequence, outs: Optional[List[List]] = None) -> List[List]:
        """wct_sim_run_host: events whose depos are in host memory (objects with t0, x, y, z, q
        float32 arrays -- numpy arrays or CPU tensors, pinned for overlapped uploads -- and
        event_id) to waveforms in host memory.  outs: [event][plane] host float32 tensors or
        arrays [n_wires, n_ticks] (pinned tensors download at full speed); allocated pinned when
        None.  Synchronous; returns outs."""
        import torch
        npl = len(self.planes)
        if outs is None:
            outs = [[torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, pin_memory=True) for p in self.planes]
                    for _ in events]
        keep = []

        def host_ptr(a, shape=None):
            if isinstance(a, torch.Tensor):
                if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
                    raise ValueError("host arrays must be contiguous float32 CPU tensors")
                t = a
            else:
                t = np.ascontiguousarray(a, dtype=np.float32)
                if shape is not None and (t is not a or t.shape != shape or not t.flags.writeable):
                    raise ValueError("waveform arrays must be writable contiguous float32 [n_wires, n_ticks]")
            keep.append(t)
            return t.data_ptr() if isinstance(t, torch.Tensor) else t.ctypes.data

        hev = (_abi.wct_host_depos_t * max(len(events), 1))()
        for i, e in enumerate(events):
            ptrs = [host_ptr(getattr(e, k)) for k in ("t0", "x", "y", "z", "q")]
            n = len(e.t0)
            hev[i] = _abi.wct_host_depos_t(*ptrs, n, int(e.event_id) & 0xFFFFFFFFFFFFFFFF)
        wf = []
        for i in range(len(events)):
            for p, pl in enumerate(self.planes):
                o = outs[i][p]
                if isinstance(o, torch.Tensor) and tuple(o.shape) != (pl.n_wires, pl.n_ticks):
                    raise ValueError("waveform tensors must be [n_wires, n_ticks]")
                wf.append(host_ptr(o, (pl.n_wires, pl.n_ticks)))
        arr = (ctypes.c_void_p * max(len(wf), 1))(*wf)
        self._check(self._lib.wct_sim_run_host(self._h, hev, len(events), arr))
        del keep
        return outs

    def sync(self, stream=None):
        """wct_sim_sync: wait for the stream and raise on a device-side error."""
        self._check(self._lib.wct_sim_sync(self._h, _stream_handle(stream)))

    def selftest_wait(self, limit_cycles: int = 2_000_000, stream=None):
        """wct_sim_selftest_wait: a bounded wait that must time out (status WCT_ETIMEOUT)."""
        self._check(self._lib.wct_sim_selftest_wait(self._h, int(limit_cycles), _stream_handle(stream)))

    def set_timing(self, enable: bool = True):
        self._check(self._lib.wct_sim_set_timing(self._h, int(bool(enable))))

    STAGES = ("prep_binning", "raster_scatter", "row_r2c", "wire_stage", "row_c2r")

    def stage_times(self) -> dict:
        """Mean microseconds per run_event of each stage since set_timing(True), and per
        run_batch call its raster launches' and convolutions' durations."""
        us = (ctypes.c_float * 9)()
        self._check(self._lib.wct_sim_stage_times(self._h, us, 9))
        out = dict(zip(self.STAGES, (float(v) for v in us[:5])))
        out["events"] = int(us[5])
        out["batch_raster"] = float(us[6])
        out["batch_convolve"] = float(us[7])
        out["batches"] = int(us[8])
        return out

    def counters(self) -> dict:
        c = (ctypes.c_int64 * 3)()
        self._check(self._lib.wct_sim_counters(self._h, c, 3))
        return {"kernel_launches": int(c[0]), "device_bytes": int(c[1]), "graph_launches": int(c[2])}


def philox4x32_10(ctr, seed: int, stream=None):
    """wct_philox4x32_10 on a [n,4] uint32-as-int32 CUDA tensor; returns [n,4] (int32 view)."""
    torch = _torch()
    out = torch.empty_like(ctr)
    L = load()
    rc = L.wct_philox4x32_10(_ptr(ctr), int(seed) & 0xFFFFFFFFFFFFFFFF, ctr.shape[0], _ptr(out), _stream_handle(stream))
    if rc != 0:
        raise WctError(rc, "wct_philox4x32_10 failed")
    return out


# --------------------------------------------------------------------------------------------
# Field-response ingestion
# --------------------------------------------------------------------------------------------

@dataclass
class FieldResponse:
    """Currents induced on one wire by a unit charge drifting along paths across the pitch:
    path_pos_mm [n_paths] (strictly increasing, relative to the wire centre; all >= 0 means a
    mirror-symmetric field given on one side), current [n_paths, n_samples] in unit charges
    per microsecond, sampled every period_us from a common origin."""
    path_pos_mm: np.ndarray
    current: np.ndarray
    period_us: float


FIELD_FORMAT = "wct-gb300-field-response/1"


def load_field_response(path: str) -> FieldResponse:
    """Read a field response from a JSON file of the form

        {"format": "wct-gb300-field-response/1", "period_us": 0.1,
         "paths": [{"pos_mm": 0.0, "current": [...]}, {"pos_mm": 0.3, "current": [...]}, ...]}

    (every path with the same number of samples, positions strictly increasing; currents in
    unit charges per microsecond)."""
    import json
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != FIELD_FORMAT:
        raise ValueError(f"{path}: not a {FIELD_FORMAT} file")
    paths = doc["paths"]
    pos = np.array([float(q["pos_mm"]) for q in paths], dtype=np.float64)
    cur = np.array([np.asarray(q["current"], dtype=np.float64) for q in paths])
    if cur.ndim != 2:
        raise ValueError(f"{path}: paths have different sample counts")
    return FieldResponse(pos, cur, float(doc["period_us"]))


def save_field_response(path: str, field: FieldResponse) -> None:
    """Write `field` in the JSON form load_field_response reads."""
    import json
    doc = {"format": FIELD_FORMAT, "period_us": float(field.period_us),
           "paths": [{"pos_mm": float(p), "current": [float(v) for v in c]}
                     for p, c in zip(field.path_pos_mm, field.current)]}
    with open(path, "w") as f:
        json.dump(doc, f)


def response_from_field(field: FieldResponse, electronics, pitch_mm: float, n_impact: int, tick_us: float,
                        n_wires_resp: int = 21, n_ticks_resp: int = 200):
    """wct_response_from_field: (per-impact-position responses float32 [n_impact, n_wires_resp,
    n_ticks_resp], their average over the phases float32 [n_wires_resp, n_ticks_resp]) from a
    field response and an electronics impulse response sampled at the field's period.  The
    first feeds Simulator.set_impact_responses, the second Simulator's create-time response."""
    pos = np.ascontiguousarray(field.path_pos_mm, dtype=np.float64)
    cur = np.ascontiguousarray(field.current, dtype=np.float64)
    el = np.ascontiguousarray(electronics, dtype=np.float64).ravel()
    if cur.ndim != 2 or cur.shape[0] != pos.shape[0]:
        raise ValueError("current must be [n_paths, n_samples] with one row per position")
    imp = np.empty((n_impact, n_wires_resp, n_ticks_resp), dtype=np.float32)
    fold = np.empty((n_wires_resp, n_ticks_resp), dtype=np.float32)
    fr = _abi.wct_field_response_t(pos.shape[0], cur.shape[1], float(field.period_us), pos.ctypes.data,
                                   cur.ctypes.data)
    rc = load().wct_response_from_field(ctypes.byref(fr), el.ctypes.data, el.shape[0], float(pitch_mm),
                                        int(n_impact), float(tick_us), int(n_wires_resp), int(n_ticks_resp),
                                        imp.ctypes.data, fold.ctypes.data)
    if rc != 0:
        raise WctError(rc, "wct_response_from_field: invalid field, electronics or sizes")
    return imp, fold
