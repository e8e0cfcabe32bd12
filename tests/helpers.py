"""Shared helpers for the GPU parity tests (tolerances, simulator construction)."""
import numpy as np

# Tolerances stated by the hot-path contract: patch / grid bins within 1e-5 of the largest
# bin (FP32 GPU vs FP64 oracle); waveforms within 1e-4 relative L2.
BIN_TOL = 1e-5
WAVE_RTOL = 1e-4


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


def max_rel_bin(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / m) if m > 0 else float(np.abs(a).max() if a.size else 0.0)


def make_sim(planes, responses, diffusion, **kw):
    import paper_2304_01841_gb300 as g
    return g.Simulator(planes, responses, diffusion, **kw)


def to_np(t):
    return t.detach().cpu().numpy()
