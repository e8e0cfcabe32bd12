"""Pins of the oracle's drift step (electron-lifetime attenuation before rasterization)."""
import math

import numpy as np

import oracle
import synth


def _depos(x, q):
    n = len(x)
    d = synth.Depos(np.zeros(n), np.asarray(x, float), np.zeros(n), np.zeros(n), np.asarray(q, float))
    d.event_id = 5
    return d


def test_attenuation_closed_forms():
    diff = synth.Diffusion()
    tau = 3000.0                                        # us
    half = diff.v_drift_mm_us * tau * math.log(2.0)    # one half-life of drift, in mm
    d = _depos([0.0, half, 2 * half], [6000.0, 6000.0, 6000.0])
    q = oracle.drift_depos(d, diff, tau).q
    assert q[0] == 6000.0
    assert abs(q[1] - 3000.0) <= 1e-3 and abs(q[2] - 1500.0) <= 1e-3


def test_fluctuated_survival_is_binomial_like():
    diff = synth.Diffusion(seed=123)
    tau = 1000.0
    n = 200_000
    x = np.full(n, diff.v_drift_mm_us * tau)            # t_d = lifetime: p = 1/e
    d = _depos(x, np.full(n, 6000.0))
    q = oracle.drift_depos(d, diff, tau, fluctuate=True).q.astype(np.float64)
    p = math.exp(-1.0)
    mean, var = 6000.0 * p, 6000.0 * p * (1 - p)
    assert abs(q.mean() - mean) <= 5 * math.sqrt(var / n)
    assert abs(q.var() / var - 1.0) <= 0.02
    # the draw is keyed by depo index and event: another event id gives other charges
    d2 = _depos(x[:1000], np.full(1000, 6000.0))
    d2.event_id = 6
    assert np.any(oracle.drift_depos(d2, diff, tau, fluctuate=True).q != q[:1000].astype(np.float32))


def test_absorption_normals_are_standard_normal():
    z = oracle.absorption_normals(99, 100_000, 3)
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.02
    assert abs(np.mean(z ** 3)) < 0.05 and abs(np.mean(z ** 4) - 3.0) < 0.1
