"""Pins of the oracle's noise + digitisation (the steps after the convolution)."""
import numpy as np

import oracle


def test_noise_free_codes_round_half_up_and_clamp():
    v = np.array([[0.49, 0.5, 1.5, 2.4999, -3.0, 1e9, np.nan, 4094.6]], dtype=np.float32)
    codes, _ = oracle.digitize(v, 1.0, 0.0, 0.0, 12, False, seed=1, plane_index=0, event_id=0)
    assert codes.tolist() == [[0, 1, 2, 2, 0, 4095, 0, 4095]]
    # gain and baseline: 2 * 10.25 + 100 = 120.5 -> 121
    c2, _ = oracle.digitize(np.array([[10.25]], np.float32), 2.0, 100.0, 0.0, 12, False, 1, 0, 0)
    assert c2[0, 0] == 121


def test_noise_is_standard_normal_white_and_keyed():
    z = oracle.noise_normals(7, 64, 1000, plane_index=1, event_id=3)
    assert z.shape == (64, 1000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.02
    # white: neighbouring ticks (same and different Philox calls) uncorrelated
    assert abs(np.mean(z[:, 1:] * z[:, :-1])) < 0.01
    assert not np.allclose(z, oracle.noise_normals(7, 64, 1000, plane_index=2, event_id=3))
    assert not np.allclose(z, oracle.noise_normals(7, 64, 1000, plane_index=1, event_id=4))


def test_noise_adds_its_variance_to_the_codes():
    v = np.zeros((200, 2000), np.float32)
    codes, s = oracle.digitize(v, 1.0, 2000.0, 3.0, 12, True, seed=11, plane_index=0, event_id=0)
    # rounding adds 1/12 to the variance of the code
    assert abs(codes.astype(float).var() - (9.0 + 1.0 / 12.0)) < 0.15
    assert abs(codes.astype(float).mean() - 2000.0) < 0.05


def test_coloured_noise_variance_and_spectrum():
    # flat amplitude 1 with noise_rms sqrt(P): Var(noise[t]) = (P - 1) / P (closed form of the
    # real inverse DFT of a circular complex Gaussian spectrum with real DC / Nyquist bins)
    P = 1024
    F = P // 2 + 1
    n = oracle.coloured_noise(5, 400, P, P, np.ones(F), np.sqrt(P), 0, 1)
    assert abs(n.var() - (P - 1) / P) < 0.02
    # shaped amplitude: the spectrum of the full-length noise follows (rms * amp)^2 per bin
    amp = np.exp(-np.arange(F) / 80.0)
    m = oracle.coloured_noise(6, 2000, P, P, amp, 2.0, 1, 2)
    pw = (np.abs(np.fft.rfft(m, axis=1)) ** 2).mean(axis=0)
    ratio = pw[1:200] / (2.0 * amp[1:200]) ** 2
    assert abs(ratio.mean() - 1.0) < 0.02 and np.all(np.abs(ratio - 1.0) < 0.25)


def test_coloured_noise_is_keyed_apart_from_white_noise():
    P, F = 256, 129
    c = oracle.coloured_noise(9, 8, P, P, np.ones(F), 1.0, 0, 3)
    c2 = oracle.coloured_noise(9, 8, P, P, np.ones(F), 1.0, 0, 4)
    assert not np.allclose(c, c2)
    # digitise adds the given noise waveform instead of the white noise
    v = np.zeros((8, P), np.float32)
    codes, s = oracle.digitize(v, 1.0, 1000.0, 1.0, 12, True, 9, 0, 3, noise_wave=c * 50.0)
    assert np.allclose(s, 1000.0 + (c * 50.0).astype(np.float32), atol=1e-3)
