"""Seeded synthetic inputs for the LArTPC signal-simulation hot path.

This module is the one thing the FP64 oracle and the GPU library both consume:
plane / diffusion parameter records, the synthetic field x electronics
response, and track-shaped ionisation-deposit ("depo") generators.  It holds
none of the simulation's own arithmetic (drift, diffusion windows, erf bin
integrals, fluctuation, scatter-add, convolution); those live separately in the
oracle and in the CUDA library.

Units throughout: mm, microseconds, electrons.

The paper (arXiv 2304.01841 §2) names the three steps (rasterization of ionisation
groups into O(20x20) patches, scatter-add onto an O(10^4 x 10^4) wire x tick grid,
FFT convolution with an O(100 x 100) detector response) but states no workload.
The workloads below are synthetic stand-ins with the shapes of MicroBooNE- and
DUNE-like planes; the recipes are written out next to each generator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Plane", "Diffusion", "Depos", "Workload", "make_response", "make_track_depos",
    "make_isolated_depos", "concat_depos", "workload", "WORKLOADS", "batch_depo_counts",
    "serving_depo_counts", "smooth_pad",
]


@dataclass(frozen=True)
class Plane:
    """One wire plane: n_wires x n_ticks readout grid.

    Wire w covers pitch coordinate [origin + w*pitch, origin + (w+1)*pitch);
    impact sub-bin j covers [origin + j*pitch/n_imp, origin + (j+1)*pitch/n_imp)
    and belongs to wire j // n_imp.  Tick k covers [t_window0 + k*tick,
    t_window0 + (k+1)*tick).  The pitch coordinate of a point is
    p = z*cos(angle) + y*sin(angle).
    """
    n_wires: int
    n_ticks: int
    n_impact_per_pitch: int = 10
    pitch_mm: float = 3.0
    pitch_origin_mm: Optional[float] = None   # default: plane centred, -n_wires*pitch/2
    wire_angle_rad: float = 0.0
    tick_us: float = 0.5
    t_window0_us: float = 0.0
    response_kind: str = "bipolar"            # "bipolar" (induction) or "unipolar" (collection)

    @property
    def origin_mm(self) -> float:
        if self.pitch_origin_mm is not None:
            return float(self.pitch_origin_mm)
        return -0.5 * self.n_wires * self.pitch_mm


@dataclass(frozen=True)
class Diffusion:
    """Drift / diffusion / fluctuation parameters (LArTPC values used by the workloads)."""
    DL_cm2_s: float = 4.0
    DT_cm2_s: float = 8.8
    v_drift_mm_us: float = 1.6
    nsigma: float = 3.0
    fluctuate: bool = False
    seed: int = 0


@dataclass
class Depos:
    """Structure-of-arrays ionisation deposits (float32), plus the event id that keys the RNG."""
    t0: np.ndarray
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    q: np.ndarray
    event_id: int = 0

    def __post_init__(self):
        for name in ("t0", "x", "y", "z", "q"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name), dtype=np.float32))
        n = self.t0.shape[0]
        assert all(getattr(self, k).shape == (n,) for k in ("x", "y", "z", "q"))

    @property
    def n(self) -> int:
        return int(self.t0.shape[0])

    def subset(self, idx) -> "Depos":
        return Depos(self.t0[idx], self.x[idx], self.y[idx], self.z[idx], self.q[idx], self.event_id)


def concat_depos(parts: Sequence[Depos], event_id: int = 0) -> Depos:
    return Depos(*(np.concatenate([getattr(p, k) for p in parts]) for k in ("t0", "x", "y", "z", "q")),
                 event_id=event_id)


# --------------------------------------------------------------------------------------------
# Synthetic response
# --------------------------------------------------------------------------------------------

def make_response(kind: str = "bipolar", n_wires: int = 21, n_ticks: int = 200, tick_us: float = 0.5,
                  falloff_wires: float = 2.0, shaping_us: float = 1.0) -> np.ndarray:
    """Synthetic 2D field x electronics response, row-major [wire offset][tick], float32.

    Row r is the response seen on wire offset k = r - n_wires//2 from the wire the charge
    arrives on.  Field part: exp(-|k|/falloff) times, in time, a Gaussian of centre
    40 + 4|k| ticks and width 4 + 0.5|k| ticks (unipolar, collection) or its negative
    time-derivative scaled by the width (bipolar, induction).  The width and centre depend
    on |k| on purpose so the response is not separable in wire x time.  Electronics:
    CR-RC^2 shaping h(t) = (t/ts)^2 exp(-t/ts) with ts = 1 us (peak at 2 us), unit sum,
    convolved in time with the field part and truncated to n_ticks.  Computed in FP64.
    """
    if n_wires % 2 != 1:
        raise ValueError("response wire extent must be odd (centre wire at n_wires//2)")
    tau = np.arange(n_ticks, dtype=np.float64)
    s = tau * tick_us / shaping_us
    h = s * s * np.exp(-s)
    h /= h.sum()
    out = np.zeros((n_wires, n_ticks), dtype=np.float64)
    for r in range(n_wires):
        k = abs(r - n_wires // 2)
        c = 40.0 + 4.0 * k
        b = 4.0 + 0.5 * k
        g = np.exp(-0.5 * ((tau - c) / b) ** 2) / (b * math.sqrt(2.0 * math.pi))
        if kind == "bipolar":
            fr = -((tau - c) / b) * g
        elif kind == "unipolar":
            fr = g
        else:
            raise ValueError(kind)
        fr = fr * math.exp(-k / falloff_wires)
        out[r] = np.convolve(fr, h)[:n_ticks]
    return out.astype(np.float32)


def make_response_impact(kind: str = "bipolar", n_impact: int = 10, n_wires: int = 21, n_ticks: int = 200,
                         tick_us: float = 0.5, falloff_wires: float = 2.0, shaping_us: float = 1.0) -> np.ndarray:
    """Per-impact-position responses, float32 [phase][wire offset][tick].

    A charge in sub-bin `phase` of its wire sits (phase + 1/2) / n_impact - 1/2 pitches from
    the wire centre, so wire offset k sees it at distance d = k - ((phase + 1/2) / n_impact -
    1/2) pitches.  The field part is that of make_response with |k| replaced by |d| (centre
    40 + 4|d|, width 4 + 0.5|d|, amplitude exp(-|d|/falloff)), so the response varies smoothly
    across the pitch and phases mirror each other (phase p at k equals phase n-1-p at -k);
    the same CR-RC^2 shaping follows.  Computed in FP64.
    """
    if n_wires % 2 != 1:
        raise ValueError("response wire extent must be odd (centre wire at n_wires//2)")
    tau = np.arange(n_ticks, dtype=np.float64)
    s = tau * tick_us / shaping_us
    h = s * s * np.exp(-s)
    h /= h.sum()
    out = np.zeros((n_impact, n_wires, n_ticks), dtype=np.float64)
    for p in range(n_impact):
        frac = (p + 0.5) / n_impact - 0.5
        for r in range(n_wires):
            d = abs((r - n_wires // 2) - frac)
            c = 40.0 + 4.0 * d
            b = 4.0 + 0.5 * d
            g = np.exp(-0.5 * ((tau - c) / b) ** 2) / (b * math.sqrt(2.0 * math.pi))
            if kind == "bipolar":
                fr = -((tau - c) / b) * g
            elif kind == "unipolar":
                fr = g
            else:
                raise ValueError(kind)
            out[p, r] = np.convolve(fr * math.exp(-d / falloff_wires), h)[:n_ticks]
    return out.astype(np.float32)


def make_field_response(kind: str = "unipolar", pitch_mm: float = 3.0, path_step_mm: float = 0.3,
                        reach_pitches: float = 10.5, period_us: float = 0.1, duration_us: float = 100.0):
    """Synthetic field response in the form a field calculation produces: the current induced on
    one wire by a unit charge drifting along paths at 0, path_step, ..., reach pitches from the
    wire (one side; the field is mirror-symmetric), sampled every period_us.

    Returns (path_pos_mm [n_paths], current [n_paths, n_samples] in unit charges per us).  At a
    distance of d pitches the pulse is centred at 20 + 2d us with width 2 + d/4 us and area
    exp(-d/2): a Gaussian (unipolar, collection) or its time derivative scaled by the width
    (bipolar, induction), the continuous counterpart of make_response's field part."""
    pos = np.arange(0.0, reach_pitches * pitch_mm + 1e-9, path_step_mm)
    t = np.arange(int(round(duration_us / period_us))) * period_us
    cur = np.zeros((pos.shape[0], t.shape[0]))
    for j, x in enumerate(pos):
        d = x / pitch_mm
        c, b = 20.0 + 2.0 * d, 2.0 + 0.25 * d
        g = np.exp(-0.5 * ((t - c) / b) ** 2) / (b * math.sqrt(2.0 * math.pi))
        if kind == "unipolar":
            f = g
        elif kind == "bipolar":
            f = -((t - c) / b) * g
        else:
            raise ValueError(kind)
        cur[j] = f * math.exp(-0.5 * d)
    return pos, cur


def electronics_crrc2(period_us: float = 0.1, shaping_us: float = 1.0, n_samples: int = 200, gain: float = 1.0):
    """CR-RC^2 shaper impulse response h(t) = (t / ts)^2 exp(-t / ts) sampled every period_us,
    scaled to unit area (sum h * period = 1) times gain."""
    s = np.arange(n_samples) * period_us / shaping_us
    h = s * s * np.exp(-s)
    return gain * h / (h.sum() * period_us)


# --------------------------------------------------------------------------------------------
# Depo generators
# --------------------------------------------------------------------------------------------

def _lognormal_mean(rng: np.random.Generator, mean: float, sigma_log: float, n: int) -> np.ndarray:
    # sigma_log is the log-space standard deviation; `mean` is the arithmetic mean.
    return rng.lognormal(math.log(mean) - 0.5 * sigma_log * sigma_log, sigma_log, n)


def _split_counts(weights: np.ndarray, total: int) -> np.ndarray:
    # Largest-remainder apportionment: integer counts proportional to weights, summing to total.
    raw = weights / weights.sum() * total
    cnt = np.floor(raw).astype(np.int64)
    rem = total - int(cnt.sum())
    if rem > 0:
        order = np.argsort(-(raw - cnt), kind="stable")
        cnt[order[:rem]] += 1
    return cnt


def make_track_depos(rng: np.random.Generator, n_depos: int, n_tracks: int, lengths_mm,
                     box_lo, box_hi, dim3: bool, q_mean: float = 6000.0, q_sigma_log: float = 0.3
                     ) -> Depos:
    """Straight tracks of equally spaced depos inside an axis-aligned box (x = drift).

    Directions are uniform on the circle in the x-z plane (dim3=False, y = 0) or uniform
    on the sphere (dim3=True).  Each track is placed by rejection so that it lies fully in
    the box (after 200 rejected starts its length is halved).  Depo counts per track are
    proportional to track length and sum to n_depos; charges are lognormal with the given
    arithmetic mean and log-space sigma.  t0 = 0 for every depo.
    """
    box_lo = np.asarray(box_lo, dtype=np.float64)
    box_hi = np.asarray(box_hi, dtype=np.float64)
    lengths = np.broadcast_to(np.asarray(lengths_mm, dtype=np.float64), (n_tracks,)).copy()
    counts = _split_counts(lengths, n_depos)
    xs, ys, zs = [], [], []
    for t in range(n_tracks):
        L = lengths[t]
        for attempt in range(10_000):
            if dim3:
                d = rng.normal(size=3)
                d /= np.linalg.norm(d)
            else:
                a = rng.uniform(0.0, 2.0 * math.pi)
                d = np.array([math.cos(a), 0.0, math.sin(a)])
            start = rng.uniform(box_lo, box_hi)
            if not dim3:
                start[1] = 0.0
            end = start + L * d
            if np.all(end >= box_lo) and np.all(end <= box_hi):
                break
            if attempt % 200 == 199:
                L *= 0.5
        n = int(counts[t])
        f = (np.arange(n, dtype=np.float64) + 0.5) / max(n, 1)
        pts = start[None, :] + (f * L)[:, None] * d[None, :]
        xs.append(pts[:, 0]); ys.append(pts[:, 1]); zs.append(pts[:, 2])
    x = np.concatenate(xs) if xs else np.zeros(0)
    y = np.concatenate(ys) if ys else np.zeros(0)
    z = np.concatenate(zs) if zs else np.zeros(0)
    q = _lognormal_mean(rng, q_mean, q_sigma_log, n_depos)
    return Depos(np.zeros(n_depos), x, y, z, q)


def make_isolated_depos(rng: np.random.Generator, n_depos: int, box_lo, box_hi,
                        q_mean: float = 500.0, q_sigma_log: float = 0.3) -> Depos:
    """Isolated low-charge depos, uniform in the box."""
    p = rng.uniform(np.asarray(box_lo, float), np.asarray(box_hi, float), size=(n_depos, 3))
    q = _lognormal_mean(rng, q_mean, q_sigma_log, n_depos)
    return Depos(np.zeros(n_depos), p[:, 0], p[:, 1], p[:, 2], q)


# --------------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    planes: List[Plane]
    diffusion: Diffusion
    n_depos: int
    seed: int
    description: str
    gen: dict = field(default_factory=dict)

    def responses(self) -> List[np.ndarray]:
        return [make_response(p.response_kind, tick_us=p.tick_us) for p in self.planes]

    def depos(self, n_depos: Optional[int] = None, event_id: int = 0, seed: Optional[int] = None) -> Depos:
        """Generate one event.  n_depos / seed override the workload's defaults."""
        n = self.n_depos if n_depos is None else int(n_depos)
        rng = np.random.default_rng(self.seed if seed is None else seed)
        g = self.gen
        lo, hi = g["box_lo"], g["box_hi"]
        n_iso = int(round(n * g.get("isolated_frac", 0.0)))
        n_trk = n - n_iso
        if g.get("length_mm") is not None:
            lengths = g["length_mm"]
        else:
            lengths = rng.uniform(g["length_range_mm"][0], g["length_range_mm"][1], g["n_tracks"])
        parts = [make_track_depos(rng, n_trk, g["n_tracks"], lengths, lo, hi, g["dim3"],
                                  g.get("q_mean", 6000.0), 0.3)]
        if n_iso:
            parts.append(make_isolated_depos(rng, n_iso, lo, hi, g.get("iso_q_mean", 500.0), 0.3))
        d = concat_depos(parts, event_id=event_id)
        return d


def _box_for(planes: Sequence[Plane], drift_mm: float, half_height_mm: float):
    zmax = 0.5 * planes[-1].n_wires * planes[-1].pitch_mm
    return [0.0, -half_height_mm, -zmax], [drift_mm, half_height_mm, zmax]


def smooth_pad(n: int, radices=(2, 3, 5, 7), even: bool = True) -> int:
    """Smallest integer >= n whose prime factors are all in `radices` (and even, if asked)."""
    m = max(int(n), 1)
    while True:
        if not even or m % 2 == 0:
            r = m
            for p in radices:
                while r % p == 0:
                    r //= p
            if r == 1:
                return m
        m += 1


def workload(name: str) -> Workload:
    """Named synthetic workloads (sizes from the hot-path scope; seeds 20230404 + index).

    - "tiny": 1 plane, 256 wires (3 mm, 10 impact bins/pitch) x 1024 ticks (0.5 us),
      1000 depos on 2 straight 0.5 m tracks in the drift-pitch plane, drift 0-1 ms,
      lognormal charge (mean 6000 e-, log-sigma 0.3), fluctuation off, bipolar response.
    - "tiny_inside": as "tiny" but drift 0-0.45 ms so every depo lands inside the window.
    - "uboone_plane": one MicroBooNE-sized collection plane, 3456 wires x 9600 ticks,
      100k depos on 20 tracks of 0.3-3 m, drift 0-2.3 ms, fluctuation on.
    - "three_plane": U/V/W planes of 2400/2400/3456 wires (+60, -60, 0 degrees) x 9600
      ticks, 1M depos: 800k on 200 tracks (3D directions) + 200k isolated depos of mean
      500 e-; induction planes bipolar, collection unipolar; fluctuation on.
    - "dune_apa": 800/800/960 wires x 6000 ticks, 3 planes, fluctuation on; depo counts
      come from `serving_depo_counts`.
    """
    D = Diffusion
    if name in ("tiny", "tiny_inside"):
        planes = [Plane(256, 1024, response_kind="bipolar")]
        drift = 1600.0 if name == "tiny" else 720.0
        lo, hi = _box_for(planes, drift, 0.0)
        return Workload(name, planes, D(fluctuate=False, seed=20230405), 1000, 20230405,
                        "1 plane 256x1024, 1000 depos, 2 tracks", dict(
                            box_lo=lo, box_hi=hi, n_tracks=2, length_mm=500.0, dim3=False))
    if name == "uboone_plane":
        planes = [Plane(3456, 9600, response_kind="bipolar")]
        lo, hi = _box_for(planes, 3680.0, 0.0)
        return Workload(name, planes, D(fluctuate=True, seed=20230406), 100_000, 20230406,
                        "1 plane 3456x9600, 100k depos, 20 tracks, fluctuation on", dict(
                            box_lo=lo, box_hi=hi, n_tracks=20, length_range_mm=(300.0, 3000.0),
                            dim3=False))
    if name == "three_plane":
        a = math.radians(60.0)
        planes = [Plane(2400, 9600, wire_angle_rad=a, response_kind="bipolar"),
                  Plane(2400, 9600, wire_angle_rad=-a, response_kind="bipolar"),
                  Plane(3456, 9600, wire_angle_rad=0.0, response_kind="unipolar")]
        lo, hi = _box_for(planes, 3680.0, 1160.0)
        return Workload(name, planes, D(fluctuate=True, seed=20230407), 1_000_000, 20230407,
                        "3 planes 2400/2400/3456x9600, 1M depos (200 tracks + 20% isolated)", dict(
                            box_lo=lo, box_hi=hi, n_tracks=200, length_range_mm=(300.0, 3000.0),
                            dim3=True, isolated_frac=0.2))
    if name == "dune_apa":
        a = math.radians(60.0)
        planes = [Plane(800, 6000, wire_angle_rad=a, response_kind="bipolar"),
                  Plane(800, 6000, wire_angle_rad=-a, response_kind="bipolar"),
                  Plane(960, 6000, wire_angle_rad=0.0, response_kind="unipolar")]
        lo, hi = _box_for(planes, 4600.0, 550.0)
        return Workload(name, planes, D(fluctuate=True, seed=20230409), 50_000, 20230409,
                        "3 planes 800/800/960x6000 (APA-like), heavy-tailed depo counts", dict(
                            box_lo=lo, box_hi=hi, n_tracks=20, length_range_mm=(300.0, 3000.0),
                            dim3=True, isolated_frac=0.2))
    raise KeyError(name)


WORKLOADS = ("tiny", "tiny_inside", "uboone_plane", "three_plane", "dune_apa")


def batch_depo_counts(n_events: int = 64, lo: int = 10_000, hi: int = 500_000, seed: int = 20230408
                      ) -> np.ndarray:
    """Per-event depo counts for the batched workload: ln N ~ Normal with lo / hi at the
    1st / 99th percentiles, clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    z99 = 2.3263478740408408
    mu = 0.5 * (math.log(lo) + math.log(hi))
    sig = (math.log(hi) - math.log(lo)) / (2.0 * z99)
    return np.clip(np.exp(rng.normal(mu, sig, n_events)), lo, hi).astype(np.int64)


def serving_depo_counts(n_events: int, seed: int = 20230409, small=(5_000, 50_000),
                        large=(1_000_000, 3_000_000), large_frac: float = 0.10) -> np.ndarray:
    """Heavy-tailed serving mix: 90% log-uniform in `small`, 10% uniform in `large`."""
    rng = np.random.default_rng(seed)
    big = rng.random(n_events) < large_frac
    n_small = np.exp(rng.uniform(math.log(small[0]), math.log(small[1]), n_events))
    n_large = rng.uniform(large[0], large[1], n_events)
    return np.where(big, n_large, n_small).astype(np.int64)


def slice_events(pool: Sequence[Depos], counts, rng: np.random.Generator, first_event_id: int) -> List[Depos]:
    """Events of the given depo counts cut from a pool of large generated events: each a
    contiguous slice of one pool event (whole track segments, plus the isolated depos the slice
    covers), with consecutive event ids from first_event_id."""
    out = []
    for i, n in enumerate(counts):
        base = pool[int(rng.integers(len(pool)))]
        n = int(min(n, base.n))
        s0 = int(rng.integers(0, base.n - n + 1))
        d = base.subset(slice(s0, s0 + n))
        out.append(Depos(d.t0, d.x, d.y, d.z, d.q, event_id=first_event_id + i))
    return out


def batch_events(n_events: int = 64, pool_seed: Optional[int] = None, first_event_id: int = 5000,
                 slice_seed: int = 7) -> List[Depos]:
    """The batched workload: n_events three-plane events (the "three_plane" geometry), depo
    counts from batch_depo_counts, each cut from one of three generated 500k-depo events (200
    tracks + 20% isolated low-charge depos, as the single three-plane event)."""
    wl = workload("three_plane")
    seed = wl.seed if pool_seed is None else pool_seed
    pool = [wl.depos(n_depos=500_000, seed=seed + k) for k in range(3)]
    return slice_events(pool, batch_depo_counts(n_events), np.random.default_rng(slice_seed), first_event_id)
