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
