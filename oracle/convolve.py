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
