"""Oracle of the field-response ingestion (the detector response of §2 step 3 built from a
field response and an electronics response).  TEST INFRASTRUCTURE ONLY.

Definition (the paper takes the response as given; the reading is stated with the C entry
point): a charge in impact sub-bin p of its wire sits at y_p = ((p + 1/2)/n_imp - 1/2) pitch
from that wire's centre; the wire at offset d = r - K (K = n_wires // 2) sees it at
x = y_p - d pitch, and its current is the field's I(x, t): linear interpolation in x between
the two paths around x (|x| if every path position is >= 0: a mirror-symmetric field given on
one side), zero beyond the outermost path.  In time it is convolved with the electronics
response on the fine grid and sampled every m = tick / period samples:

    R_p[r][tau] = period * sum_s I(x, s) E[tau m - s].

The folded response is the mean over p.  FP64.  Parity pinned by tests/test_oracle_response.py
(delta electronics, fields constant or linear in x, mirror symmetry, outer-range zeros, a
literal loop on tiny inputs).
"""
from __future__ import annotations

import numpy as np


def field_at(pos: np.ndarray, current: np.ndarray, x: float):
    """I(x, .) by linear interpolation between paths; None beyond the covered range."""
    if pos[0] >= 0.0:
        x = abs(x)
    if x < pos[0] or x > pos[-1]:
        return None
    j = int(np.searchsorted(pos, x, side="right")) - 1
    j = min(max(j, 0), len(pos) - 2)
    a = (x - pos[j]) / (pos[j + 1] - pos[j])
    return (1.0 - a) * current[j] + a * current[j + 1]


def response_from_field(pos, current, period_us: float, electronics, pitch_mm: float, n_impact: int,
                        tick_us: float, n_wires: int = 21, n_ticks: int = 200):
    """(impact [n_impact, n_wires, n_ticks], folded [n_wires, n_ticks]) in FP64."""
    pos = np.asarray(pos, dtype=np.float64)
    current = np.asarray(current, dtype=np.float64)
    e = np.asarray(electronics, dtype=np.float64)
    m = int(round(tick_us / period_us))
    if m < 1 or abs(tick_us / period_us - m) > 1e-9 * tick_us / period_us:
        raise ValueError("tick must be a whole number of field periods")
    K = n_wires // 2
    out = np.zeros((n_impact, n_wires, n_ticks))
    for p in range(n_impact):
        y = ((p + 0.5) / n_impact - 0.5) * pitch_mm
        for r in range(n_wires):
            cur = field_at(pos, current, y - (r - K) * pitch_mm)
            if cur is None:
                continue
            full = np.convolve(cur, e) * period_us          # fine-grid samples 0 .. ns + ne - 2
            idx = np.arange(n_ticks) * m
            ok = idx < full.shape[0]
            out[p, r, ok] = full[idx[ok]]
    return out, out.mean(axis=0)


def response_from_field_loops(pos, current, period_us: float, electronics, pitch_mm: float, n_impact: int,
                              tick_us: float, n_wires: int, n_ticks: int):
    """The same definition as literal loops (tiny inputs only)."""
    m = int(round(tick_us / period_us))
    K = n_wires // 2
    ns, ne = len(current[0]), len(electronics)
    out = [[[0.0] * n_ticks for _ in range(n_wires)] for _ in range(n_impact)]
    for p in range(n_impact):
        for r in range(n_wires):
            x = ((p + 0.5) / n_impact - 0.5) * pitch_mm - (r - K) * pitch_mm
            if pos[0] >= 0.0:
                x = abs(x)
            j = None
            for i in range(len(pos) - 1):
                if pos[i] <= x <= pos[i + 1]:
                    j = i
                    break
            if j is None:
                continue
            a = (x - pos[j]) / (pos[j + 1] - pos[j])
            for t in range(n_ticks):
                acc = 0.0
                for s in range(ns):
                    k = t * m - s
                    if 0 <= k < ne:
                        acc += ((1.0 - a) * current[j][s] + a * current[j + 1][s]) * electronics[k]
                out[p][r][t] = acc * period_us
    return np.array(out)
