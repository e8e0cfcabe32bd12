"""Pins for the oracle's diffusion windows and erf-difference bin weights (CPU only).

The weights are pinned against Gaussian bin integrals computed independently by mpmath
quadrature of the density (no erf involved), against brute-force window sets, against
hand-computed drift / diffusion numbers, and against the moments of a Gaussian.
"""
import math

import numpy as np
import pytest

import oracle
import synth

mpmath = pytest.importorskip("mpmath")


def _mp_bin_weights(mu, s, lo, n):
    mpmath.mp.dps = 30
    f = lambda x: mpmath.exp(-(x - mu) ** 2 / (2 * s * s)) / (s * mpmath.sqrt(2 * mpmath.pi))
    vals = [mpmath.quad(f, [lo + i, lo + i + 1]) for i in range(n)]
    tot = mpmath.fsum(vals)
    return np.array([float(v / tot) for v in vals])


@pytest.mark.parametrize("case", range(24))
def test_weights_match_quadrature(case):
    rng = np.random.default_rng(1000 + case)
    s = float(np.exp(rng.uniform(np.log(0.05), np.log(8.0))))
    mu = float(rng.uniform(-40.0, 40.0))
    lo, w = oracle.axis_weights(mu, s, 3.0)
    ref = _mp_bin_weights(mu, s, lo, len(w))
    np.testing.assert_allclose(w, ref, rtol=0, atol=2e-14)
    assert abs(w.sum() - 1.0) < 1e-14


def test_window_is_set_of_bins_overlapping_nsigma_interval():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        s = float(np.exp(rng.uniform(np.log(1e-3), np.log(20.0))))
        mu = float(rng.uniform(-100.0, 100.0))
        ns = float(rng.choice([1.0, 2.5, 3.0, 4.0]))
        lo, w = oracle.axis_weights(mu, s, ns)
        a, b = mu - ns * s, mu + ns * s
        brute = [i for i in range(-200, 200) if i <= b and i + 1 > a]
        assert list(range(lo, lo + len(w))) == brute


def test_point_charge_goes_to_containing_bin():
    for mu, want in [(3.25, 3), (-0.5, -1), (7.0, 7), (-2.0, -2), (0.0, 0)]:
        for s in (0.0, 1e-7, 9.9e-7):
            lo, w = oracle.axis_weights(mu, s, 3.0)
            assert lo == want and list(w) == [1.0]


def test_centred_depo_is_symmetric_and_shift_invariant():
    for s in (0.3, 1.0, 2.7, 6.1):
        lo, w = oracle.axis_weights(10.5, s, 3.0)
        np.testing.assert_allclose(w, w[::-1], rtol=0, atol=1e-15)
        lo2, w2 = oracle.axis_weights(10.5 + 7.0, s, 3.0)
        assert lo2 == lo + 7
        np.testing.assert_allclose(w2, w, rtol=0, atol=1e-15)


@pytest.mark.parametrize("s", [3.0, 5.0, 11.0])
def test_weight_moments_are_gaussian(s):
    # With a wide window the binned Gaussian has mean mu and variance s^2 + 1/12 (Sheppard).
    mu = 0.37
    lo, w = oracle.axis_weights(mu, s, 9.0)
    centres = lo + np.arange(len(w)) + 0.5
    m = float((centres * w).sum())
    v = float(((centres - m) ** 2 * w).sum())
    assert abs(m - mu) < 1e-9
    assert abs(v - (s * s + 1.0 / 12.0)) < 1e-6 * s * s


def test_drift_diffusion_hand_values():
    # x = 160 mm at 1.6 mm/us -> t_d = 100 us -> tick 200 at 0.5 us/tick.
    # sigma_L = sqrt(2 * 4.0 cm^2/s * 100 us) = sqrt(2 * 4e-4 mm^2/us * 100 us) = sqrt(0.08) mm
    #         = 0.28284271 mm -> / 1.6 mm/us / 0.5 us = 0.35355339 ticks.
    # sigma_T = sqrt(2 * 8.8e-4 * 100) = sqrt(0.176) = 0.41952354 mm -> / 0.3 mm = 1.39841180 bins.
    # p = z = 1.5 mm, origin = -384 mm -> (1.5 + 384) / 0.3 = 1285.0 impact bins.
    plane = synth.Plane(256, 1024)
    diff = synth.Diffusion()
    d = synth.Depos([0.0], [160.0], [0.0], [1.5], [1000.0])
    desc, mus, total, bad = oracle.windows(d, plane, diff)
    assert bad == 0
    mu_t, s_t, mu_p, s_p = mus[0]
    assert abs(mu_t - 200.0) < 1e-9
    assert abs(s_t - 0.35355339059327373) < 1e-12
    assert abs(mu_p - 1285.0) < 1e-9
    assert abs(s_p - 1.3984117975602022) < 1e-12
    # window: ticks floor(200 - 1.0607) .. floor(200 + 1.0607) = 198 .. 201
    assert tuple(desc[0, 1:]) == (198, int(math.floor(1285.0 - 3 * 1.3984117975602022)), 4,
                                  int(math.floor(1285.0 + 3 * 1.39841179756)) -
                                  int(math.floor(1285.0 - 3 * 1.39841179756)) + 1)


def test_time_offset_and_wire_angle():
    # t0 shifts the arrival; the pitch coordinate is z cos(a) + y sin(a).
    a = math.radians(60.0)
    plane = synth.Plane(100, 1000, wire_angle_rad=a, pitch_origin_mm=0.0, t_window0_us=10.0)
    diff = synth.Diffusion()
    d = synth.Depos([25.0], [16.0], [10.0], [0.0], [1.0])
    _, mus, _, _ = oracle.windows(d, plane, diff)
    # arrival = 25 + 16/1.6 = 35 us -> (35 - 10) / 0.5 = 50 ticks
    assert abs(mus[0, 0] - 50.0) < 1e-9
    # p = 10 * sin(60 deg) = 8.660254 mm -> / 0.3 = 28.867513 bins
    assert abs(mus[0, 2] - 28.867513459481287) < 1e-9


def test_invalid_depos_are_flagged():
    plane = synth.Plane(64, 256)
    diff = synth.Diffusion()
    d = synth.Depos([0, 0, 0, 0, np.nan, 0], [10, -1, 10, 10, 10, 1e7], [0] * 6, [0] * 6,
                    [1, 1, -1, np.inf, 1, 1])
    desc, _, total, bad = oracle.windows(d, plane, diff)
    # depos 1 (x<0), 2 (q<0), 3 (q inf), 4 (t0 nan), 5 (window > limits) are invalid
    assert bad == 5
    assert desc[0, 3] > 0 and all(desc[i, 3] == 0 for i in range(1, 6))
