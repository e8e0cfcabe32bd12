"""FP64 CPU oracle for the LArTPC signal-simulation hot path (arXiv 2304.01841, §2).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the package smoke check and by
the benchmark's CPU-baseline / reference arm.  The GPU library never imports it.  The
rasterize / scatter steps are plain C loops in FP64 (oracle/wct_oracle.c, built with gcc
into oracle/_build/); the convolution is scipy's FP64 FFT (oracle/convolve.py) plus a
literal quadruple loop for small grids.

Parity status of each function (what pins it; see tests/test_oracle_*.py):
  windows / weights    pinned: mpmath Gaussian bin integrals, brute-force window sets,
                       hand-computed drift / diffusion values, moments of the patch.
  rasterize (no fluct) pinned: patch sums to q, outer-product structure, shift invariance;
                       hypothesis-drawn edge cases (bin edges, sigma = 0, off-grid depos).
  rasterize (fluct)    pinned statistically: per-bin mean / variance of the multinomial,
                       large-q limit; the Philox4x32-10 stream by the published Random123
                       known-answer vectors (tests/golden).
  scatter              pinned: charge conservation, hand-built folding cases.
  convolve             pinned: delta response = identity, delta grid = placed response,
                       direct quadruple loop, no circular wrap, linearity.
  digitise             pinned: noise-free codes against exact rounding of hand values,
                       clamping, the noise's normality and its keying.
  all-core variants    rasterize_all_cores / scatter_all_cores (timing only) are checked
                       bit-identical to the serial functions.
  drift attenuation    pinned: closed form q exp(-t_d / lifetime); fluctuated mean and
                       variance of the binomial; the same charge for every plane.
  impact-resolution    pinned: phase-independent responses reduce to the folded path,
  scatter / convolve   FFT form = literal loops, a single sub-bin charge places its phase's
                       response, the impact grid folds to the wire grid.
  response from field  (oracle/response.py) pinned: delta electronics returns the sampled
                       current, exact interpolation of a field linear in x, mirror symmetry,
                       two-sided = mirrored one-sided, zero beyond the field's reach, an
                       impulse current places the electronics response, literal loops.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

from .convolve import convolve_fft, convolve_direct_np, convolve_impact, convolve_impact_direct  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wct_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libwctoracle.so")
_lock = threading.Lock()
_lib = None

# Largest window the library accepts (ticks x impact bins); depos beyond are invalid.
MAX_NT = 128
MAX_NP = 512


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no floating-point contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC]
        try:   # OpenMP for the all-core timing variants; without it they run on one thread
            subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The compiled oracle (built on first use).  $WCT_ORACLE_LIB names another build of the
    same source instead (the sanitizer test loads an ASan / UBSan build this way)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("WCT_ORACLE_LIB")
            if not path:
                path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            L.or_philox_batch.argtypes = [i64, P, P, P]
            L.or_philox_batch.restype = None
            L.or_bin_normal.argtypes = [u64, ctypes.c_uint32, i64, i64, i32, i32, u64]
            L.or_bin_normal.restype = dbl
            L.or_axis_weights.argtypes = [dbl, dbl, dbl, P, P, P, i64]
            L.or_axis_weights.restype = None
            L.or_windows.argtypes = [i64, P, P, P, P, P, P, P, i64, i64, P, P, P]
            L.or_windows.restype = i64
            L.or_rasterize.argtypes = [i64, P, P, P, P, P, P, P, P, i32, u64, i32, u64, P]
            L.or_rasterize.restype = ctypes.c_int
            L.or_scatter.argtypes = [i64, P, P, i32, i64, i64, P]
            L.or_scatter.restype = None
            L.or_convolve_direct.argtypes = [P, i64, i64, P, i64, i64, P]
            L.or_convolve_direct.restype = None
            L.or_omp_threads.argtypes = [i32]
            L.or_omp_threads.restype = i32
            L.or_rasterize_omp.argtypes = [i64, P, P, P, P, P, P, P, P, i32, u64, i32, u64, P, i32]
            L.or_rasterize_omp.restype = ctypes.c_int
            L.or_scatter_omp.argtypes = [i64, P, P, i32, i64, i64, P, i32]
            L.or_scatter_omp.restype = None
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _plane_vec(plane) -> np.ndarray:
    return np.array([plane.pitch_mm, plane.origin_mm, plane.wire_angle_rad, plane.tick_us,
                     plane.t_window0_us, float(plane.n_impact_per_pitch)], dtype=np.float64)


def _diff_vec(diff) -> np.ndarray:
    return np.array([diff.DL_cm2_s, diff.DT_cm2_s, diff.v_drift_mm_us, diff.nsigma], dtype=np.float64)


# ------------------------------------------------------------------------------------------
# Philox / normals
# ------------------------------------------------------------------------------------------

def philox4x32_10(ctr: np.ndarray, key: Tuple[int, int]) -> np.ndarray:
    """Philox4x32-10 of each 4-word counter row under one key (uint32 [n,4] -> [n,4])."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.array(key, dtype=np.uint32)
    out = np.empty_like(ctr)
    lib().or_philox_batch(ctr.shape[0], _p(ctr), _p(k), _p(out))
    return out


def bin_normal(seed: int, depo_index: int, tick: int, impact: int, n_imp: int, plane: int,
               event_id: int) -> float:
    """The fluctuation pool's normal deviate for one absolute (tick, impact) bin."""
    return lib().or_bin_normal(seed, depo_index, tick, impact, n_imp, plane, event_id)


def axis_weights(mu: float, s: float, nsigma: float = 3.0, cap: int = 4096):
    """(lo, weights) of one axis: erf-difference bin integrals over the +-nsigma window."""
    lo = ctypes.c_int64()
    n = ctypes.c_int64()
    w = np.zeros(cap, dtype=np.float64)
    lib().or_axis_weights(mu, s, nsigma, ctypes.byref(lo), ctypes.byref(n), _p(w), cap)
    if n.value > cap:
        raise ValueError("window larger than cap")
    return int(lo.value), w[: n.value].copy()


# ------------------------------------------------------------------------------------------
# Rasterize / scatter / convolve
# ------------------------------------------------------------------------------------------

class Patches:
    """Oracle patches of one plane: desc [n,5] = (offset, lo_t, lo_p, n_t, n_p), values FP64."""

    def __init__(self, desc, values, mus, n_invalid):
        self.desc = desc
        self.values = values
        self.mus = mus
        self.n_invalid = n_invalid

    def patch(self, i: int) -> np.ndarray:
        off, _, _, nt, npp = (int(v) for v in self.desc[i])
        return self.values[off: off + nt * npp].reshape(nt, npp)


def windows(depos, plane, diff, max_nt: int = MAX_NT, max_np: int = MAX_NP):
    n = depos.n
    desc = np.zeros((n, 5), dtype=np.int64)
    mus = np.zeros((n, 4), dtype=np.float64)
    total = ctypes.c_int64()
    pv, dv = _plane_vec(plane), _diff_vec(diff)
    bad = lib().or_windows(n, _p(depos.t0), _p(depos.x), _p(depos.y), _p(depos.z), _p(depos.q),
                           _p(pv), _p(dv), max_nt, max_np, _p(desc), _p(mus), ctypes.byref(total))
    return desc, mus, int(total.value), int(bad)


def rasterize(depos, plane, diff, plane_index: int = 0, fluctuate: Optional[bool] = None,
              max_nt: int = MAX_NT, max_np: int = MAX_NP) -> Patches:
    """All patches of one plane in FP64 (the reading of §2's rasterization step)."""
    desc, mus, total, bad = windows(depos, plane, diff, max_nt, max_np)
    vals = np.zeros(max(total, 1), dtype=np.float64)
    fl = diff.fluctuate if fluctuate is None else fluctuate
    pv, dv = _plane_vec(plane), _diff_vec(diff)
    rc = lib().or_rasterize(depos.n, _p(depos.t0), _p(depos.x), _p(depos.y), _p(depos.z),
                            _p(depos.q), _p(pv), _p(dv), _p(desc), int(bool(fl)),
                            int(diff.seed) & 0xFFFFFFFFFFFFFFFF, plane_index,
                            int(depos.event_id), _p(vals))
    if rc != 0:
        raise RuntimeError(f"oracle rasterize failed ({rc})")
    return Patches(desc, vals[:total], mus, bad)


def scatter(patches: Patches, plane) -> np.ndarray:
    """Scatter-add of the patches onto the plane's wire x tick grid (FP64)."""
    grid = np.zeros((plane.n_wires, plane.n_ticks), dtype=np.float64)
    vals = patches.values if patches.values.size else np.zeros(1)
    lib().or_scatter(patches.desc.shape[0], _p(patches.desc), _p(vals), plane.n_impact_per_pitch,
                     plane.n_wires, plane.n_ticks, _p(grid))
    return grid


def omp_threads(n_threads: int = 0) -> int:
    """Threads the all-core variants use (1 if the oracle was built without OpenMP)."""
    return int(lib().or_omp_threads(int(n_threads)))


def rasterize_all_cores(depos, plane, diff, plane_index: int = 0, n_threads: int = 0) -> Patches:
    """rasterize() with the depos spread over the host cores (each patch computed by one
    thread at its own offset): the same patches, bit for bit.  For timing the oracle."""
    desc, mus, total, bad = windows(depos, plane, diff)
    vals = np.zeros(max(total, 1), dtype=np.float64)
    pv, dv = _plane_vec(plane), _diff_vec(diff)
    rc = lib().or_rasterize_omp(depos.n, _p(depos.t0), _p(depos.x), _p(depos.y), _p(depos.z),
                                _p(depos.q), _p(pv), _p(dv), _p(desc), int(bool(diff.fluctuate)),
                                int(diff.seed) & 0xFFFFFFFFFFFFFFFF, plane_index,
                                int(depos.event_id), _p(vals), int(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle rasterize failed ({rc})")
    return Patches(desc, vals[:total], mus, bad)


def scatter_all_cores(patches: Patches, plane, n_threads: int = 0) -> np.ndarray:
    """scatter() with each host thread owning a band of wires (every bin summed in the serial
    depo order): the same grid, bit for bit.  For timing the oracle."""
    grid = np.zeros((plane.n_wires, plane.n_ticks), dtype=np.float64)
    vals = patches.values if patches.values.size else np.zeros(1)
    lib().or_scatter_omp(patches.desc.shape[0], _p(patches.desc), _p(vals), plane.n_impact_per_pitch,
                         plane.n_wires, plane.n_ticks, _p(grid), int(n_threads))
    return grid


def simulate_event_all_cores(depos, planes, diff, responses, n_threads: int = 0):
    """The whole hot path of one event on every host core: per plane the all-core rasterize and
    scatter, then scipy's FP64 FFT convolution with one worker per thread.  Returns the
    waveforms (FP64)."""
    workers = omp_threads(n_threads)
    out = []
    for p, (plane, resp) in enumerate(zip(planes, responses)):
        pt = rasterize_all_cores(depos, plane, diff, p, n_threads)
        out.append(convolve_fft(scatter_all_cores(pt, plane, n_threads), resp, workers=workers))
    return out


def convolve_direct(grid: np.ndarray, resp: np.ndarray) -> np.ndarray:
    """Literal quadruple-loop linear convolution in C (small grids only)."""
    g = np.ascontiguousarray(grid, dtype=np.float64)
    r = np.ascontiguousarray(resp, dtype=np.float64)
    out = np.zeros_like(g)
    lib().or_convolve_direct(_p(g), g.shape[0], g.shape[1], _p(r), r.shape[0], r.shape[1], _p(out))
    return out


def simulate_plane(depos, plane, diff, resp, plane_index: int = 0):
    """Whole hot path for one plane: (patches, grid, waveform), all FP64."""
    pt = rasterize(depos, plane, diff, plane_index)
    grid = scatter(pt, plane)
    wf = convolve_fft(grid, resp)
    return pt, grid, wf


def scatter_impact(patches: Patches, plane) -> np.ndarray:
    """Scatter-add at impact resolution: grid[j, t] over impact sub-bins j (wire j // n_imp,
    phase j % n_imp) and ticks, (n_wires * n_imp) x n_ticks, FP64; bins outside are dropped.
    The transverse grid of the paper's scatter-add step (§2 step 2) kept at the resolution of
    the patches instead of folded onto wires."""
    n_imp = plane.n_impact_per_pitch
    ni, nt = plane.n_wires * n_imp, plane.n_ticks
    grid = np.zeros((ni, nt), dtype=np.float64)
    desc = patches.desc
    for k in range(desc.shape[0]):
        off, lo_t, lo_p, n_t, n_p = (int(v) for v in desc[k])
        if n_t == 0:
            continue
        patch = patches.values[off: off + n_t * n_p].reshape(n_t, n_p)   # [tick][impact]
        t0, t1 = max(lo_t, 0), min(lo_t + n_t, nt)
        j0, j1 = max(lo_p, 0), min(lo_p + n_p, ni)
        if t0 >= t1 or j0 >= j1:
            continue
        grid[j0:j1, t0:t1] += patch[t0 - lo_t: t1 - lo_t, j0 - lo_p: j1 - lo_p].T
    return grid


def simulate_plane_impact(depos, plane, diff, resp_impact, plane_index: int = 0):
    """Whole hot path with per-impact-position responses: (patches, impact grid, waveform).
    resp_impact[phase][wire offset][tick]."""
    pt = rasterize(depos, plane, diff, plane_index)
    g = scatter_impact(pt, plane)
    wf = convolve_impact(g, resp_impact)
    return pt, g, wf


def absorption_normals(seed: int, n: int, event_id: int) -> np.ndarray:
    """z for the drift attenuation of depos 0..n-1: the first Box-Muller normal of Philox4x32-10
    at counter (depo, 0, 0, 0xFF << 24 | event id mod 2^24) under the seed's key, in FP64
    (u = (word + 1/2) 2^-32, z = sqrt(-2 ln u_0) cos(2 pi u_1))."""
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint64).astype(np.uint32)
    ctr[:, 3] = np.uint32((0xFF << 24) | (int(event_id) & 0xFFFFFF))
    w = philox4x32_10(ctr, (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)).astype(np.float64)
    u0 = (w[:, 0] + 0.5) * 2.0 ** -32
    u1 = (w[:, 1] + 0.5) * 2.0 ** -32
    return np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)


def drift_depos(depos, diff, lifetime_us: float, fluctuate: bool = False):
    """The drift step before rasterization: each depo's charge attenuated by the electron
    lifetime, surviving fraction p = exp(-t_d / lifetime), t_d = x / v.  Without fluctuation the
    mean q p; with it the normal approximation to Binomial(q, p), max(0, q p + sqrt(q p (1-p)) z)
    (absorption_normals).  FP64, returned as a copy of the depos with the new charges (float32,
    the input precision of the later steps)."""
    import copy
    x = depos.x.astype(np.float64)
    q = depos.q.astype(np.float64)
    p = np.exp(-(x / diff.v_drift_mm_us) / lifetime_us)
    m = q * p
    if fluctuate:
        z = absorption_normals(diff.seed, depos.n, depos.event_id)
        m = np.maximum(m + np.sqrt(m * (1.0 - p)) * z, 0.0)
    out = copy.copy(depos)
    out.q = m.astype(np.float32)
    return out


def noise_normals(seed: int, n_wires: int, n_ticks: int, plane_index: int, event_id: int) -> np.ndarray:
    """White-noise z[wire][tick] of the digitiser (FP64): Philox4x32-10 at counter
    (tick // 4, wire, 0, (0x80 | plane) << 24 | event id mod 2^24) under the seed's key; words
    (0, 1) and (2, 3) give the Box-Muller pairs of ticks 4k, 4k+1 and 4k+2, 4k+3
    (u = (word + 1/2) 2^-32, (r cos 2 pi u_1, r sin 2 pi u_1), r = sqrt(-2 ln u_0))."""
    nq = (n_ticks + 3) // 4
    w, qd = np.meshgrid(np.arange(n_wires), np.arange(nq), indexing="ij")
    ctr = np.zeros((n_wires * nq, 4), dtype=np.uint32)
    ctr[:, 0] = qd.ravel().astype(np.uint32)
    ctr[:, 1] = w.ravel().astype(np.uint32)
    ctr[:, 3] = np.uint32(((0x80 | plane_index) << 24) | (int(event_id) & 0xFFFFFF))
    x = philox4x32_10(ctr, (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)).astype(np.float64)
    u = (x + 0.5) * 2.0 ** -32
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.stack([r01 * np.cos(2 * np.pi * u[:, 1]), r01 * np.sin(2 * np.pi * u[:, 1]),
                  r23 * np.cos(2 * np.pi * u[:, 3]), r23 * np.sin(2 * np.pi * u[:, 3])], axis=1)
    return z.reshape(n_wires, nq * 4)[:, :n_ticks]


def coloured_noise(seed: int, n_wires: int, n_ticks: int, fft_length: int, amplitude: np.ndarray,
                   noise_rms: float, plane_index: int, event_id: int) -> np.ndarray:
    """Coloured noise [wire][tick] (FP64): the first n_ticks samples of the inverse real DFT of
    length fft_length (numpy's normalisation, 1 / fft_length) of
        N[w][f] = noise_rms * amplitude[f] * (z_re + i z_im) / sqrt(2),   f = 0 .. fft_length / 2,
    z_im = 0 at f = 0 and f = fft_length / 2; z from Philox4x32-10 at counter
    (f // 2, wire, 1, (0x80 | plane) << 24 | event id mod 2^24) under the seed's key, words
    (0, 1) for bin 2k and (2, 3) for bin 2k+1 as Box-Muller pairs."""
    F = fft_length // 2 + 1
    pairs = (F + 1) // 2
    w, k = np.meshgrid(np.arange(n_wires), np.arange(pairs), indexing="ij")
    ctr = np.zeros((n_wires * pairs, 4), dtype=np.uint32)
    ctr[:, 0] = k.ravel().astype(np.uint32)
    ctr[:, 1] = w.ravel().astype(np.uint32)
    ctr[:, 2] = 1
    ctr[:, 3] = np.uint32(((0x80 | plane_index) << 24) | (int(event_id) & 0xFFFFFF))
    x = philox4x32_10(ctr, (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)).astype(np.float64)
    u = (x + 0.5) * 2.0 ** -32
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    zr = np.stack([r01 * np.cos(2 * np.pi * u[:, 1]), r23 * np.cos(2 * np.pi * u[:, 3])], axis=1)
    zi = np.stack([r01 * np.sin(2 * np.pi * u[:, 1]), r23 * np.sin(2 * np.pi * u[:, 3])], axis=1)
    zr = zr.reshape(n_wires, 2 * pairs)[:, :F]
    zi = zi.reshape(n_wires, 2 * pairs)[:, :F].copy()
    zi[:, 0] = 0.0
    if fft_length % 2 == 0:
        zi[:, F - 1] = 0.0
    N = noise_rms * np.asarray(amplitude, dtype=np.float64)[None, :] * (zr + 1j * zi) / np.sqrt(2.0)
    return np.fft.irfft(N, n=fft_length, axis=1)[:, :n_ticks]


def digitize(waveform: np.ndarray, gain: float, baseline: float, noise_rms: float, bits: int, add_noise: bool,
             seed: int, plane_index: int, event_id: int, noise_wave: Optional[np.ndarray] = None):
    """ADC codes of a float32 waveform: code = clamp(floor(gain v + baseline + noise + 1/2),
    0, 2^bits - 1), the integer decided in FP32 with each operation rounded separately in that
    order (as the device does).  noise = noise_rms z with z = noise_normals(...) rounded to FP32
    (white), or the given noise waveform rounded to FP32 (coloured, see coloured_noise).
    Returns (codes int16, the FP32 value before rounding)."""
    f32 = np.float32
    v = np.asarray(waveform, dtype=np.float32)
    nw, nt = v.shape
    if add_noise and noise_wave is not None:
        nz = np.asarray(noise_wave, dtype=np.float32)
    elif add_noise and noise_rms > 0:
        nz = f32(noise_rms) * noise_normals(seed, nw, nt, plane_index, event_id).astype(np.float32)
    else:
        nz = np.zeros_like(v)
    with np.errstate(invalid="ignore", over="ignore"):
        s = (f32(gain) * v + f32(baseline)) + nz
        code = np.floor(s + f32(0.5))
        code = np.where(np.isnan(code), f32(0), code)
        code = np.clip(code, f32(0), f32((1 << bits) - 1))
    return code.astype(np.int16), s
