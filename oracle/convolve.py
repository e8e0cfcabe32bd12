"""FP64 convolution of the wire x tick grid with the detector response (arXiv 2304.01841, §2
step 3, "the large grid is then convolved with the detector response ... the main computation
here is FFT").  TEST INFRASTRUCTURE ONLY.

Definition (linear, not circular; response centred in wire, causal in time, output cropped to
the grid):
    out[w, t] = sum_r sum_tau grid[w - (r - kc), t - tau] * resp[r, tau],   kc = n_resp_wires // 2
with the grid zero outside its extent.  convolve_fft evaluates it with scipy's FP64 2D real FFT
on a zero-padded (n_wires + n_resp_wires - 1) x (n_ticks + n_resp_ticks - 1) array, which holds
the full linear convolution without wrap-around; convolve_direct_np is the same sum written as
explicit shifted adds (small grids).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def convolve_fft(grid: np.ndarray, resp: np.ndarray, workers: int = 1) -> np.ndarray:
    g = np.asarray(grid, dtype=np.float64)
    r = np.asarray(resp, dtype=np.float64)
    nw, nt = g.shape
    kw, kt = r.shape
    kc = kw // 2
    pw, pt = nw + kw - 1, nt + kt - 1
    G = sfft.rfft2(g, s=(pw, pt), workers=workers)
    R = sfft.rfft2(r, s=(pw, pt), workers=workers)
    full = sfft.irfft2(G * R, s=(pw, pt), workers=workers)
    # full[a, b] = sum over w' + r = a, t' + tau = b; out[w, t] sits at a = w + kc, b = t.
    return full[kc: kc + nw, :nt].copy()


def convolve_direct_np(grid: np.ndarray, resp: np.ndarray) -> np.ndarray:
    g = np.asarray(grid, dtype=np.float64)
    r = np.asarray(resp, dtype=np.float64)
    nw, nt = g.shape
    kw, kt = r.shape
    kc = kw // 2
    out = np.zeros_like(g)
    for row in range(kw):
        dw = row - kc                       # out[w] takes grid[w - dw]
        for tau in range(kt):
            if tau >= nt:
                break
            c = r[row, tau]
            if c == 0.0:
                continue
            w_lo, w_hi = max(0, dw), min(nw, nw + dw)
            if w_lo >= w_hi:
                continue
            out[w_lo:w_hi, tau:] += c * g[w_lo - dw: w_hi - dw, : nt - tau]
    return out


# Per-impact-position responses.  The transverse grid is kept at impact resolution: row
# j = n_imp * w' + phase holds the charge arriving in sub-bin `phase` of wire w', and the
# response seen on wire w depends on both the wire offset k = w - w' and the phase:
#     out[w, t] = sum_{w', phase} sum_tau g[n_imp w' + phase, t - tau] * resp[phase][k + kc][tau]
# (the detector response of §2 step 3 resolved by impact position, as the toolkit's
# per-impact field responses are).  With the same response for every phase this is the
# folded convolution of the summed sub-bins.

def convolve_impact(g_imp: np.ndarray, resp_impact: np.ndarray, workers: int = 1) -> np.ndarray:
    r = np.asarray(resp_impact, dtype=np.float64)
    n_imp = r.shape[0]
    g = np.asarray(g_imp, dtype=np.float64)
    if g.shape[0] % n_imp:
        raise ValueError("impact grid rows must be a multiple of the phase count")
    out = None
    for phase in range(n_imp):
        part = convolve_fft(g[phase::n_imp], r[phase], workers=workers)
        out = part if out is None else out + part
    return out


def convolve_impact_direct(g_imp: np.ndarray, resp_impact: np.ndarray) -> np.ndarray:
    """The same sum as literal loops over charge rows, response rows and ticks (small grids)."""
    r = np.asarray(resp_impact, dtype=np.float64)
    n_imp, kw, kt = r.shape
    kc = kw // 2
    g = np.asarray(g_imp, dtype=np.float64)
    ni, nt = g.shape
    nw = ni // n_imp
    out = np.zeros((nw, nt))
    for j in range(ni):
        wq, phase = divmod(j, n_imp)
        for row in range(kw):
            w = wq + row - kc
            if not 0 <= w < nw:
                continue
            for tau in range(min(kt, nt)):
                c = r[phase, row, tau]
                if c != 0.0:
                    out[w, tau:] += c * g[j, : nt - tau]
    return out
