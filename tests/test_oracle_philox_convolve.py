"""Pins for the oracle's Philox4x32-10 stream, its normal deviates, and the FP64 convolution.

No published known-answer vectors for Philox are available here, so the generator is
pinned by its statistical properties (uniformity, avalanche, independence) and, in the GPU
tests, by bit-equality with the separately written CUDA generator.  The convolution is
pinned by closed forms (delta response, delta grid), by the literal quadruple loop, by
linearity and by the absence of circular wrap-around.
"""
import os

import numpy as np
import pytest

import oracle
import synth

scipy_stats = pytest.importorskip("scipy.stats")


def _kat_vectors():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], (v[4], v[5]), v[6:10]))
    return rows


def test_philox_known_answer_vectors():
    # the published known-answer vectors of Philox4x32-10 (tests/golden, cited there)
    for ctr, key, want in _kat_vectors():
        got = oracle.philox4x32_10(np.array([ctr], dtype=np.uint32), key)
        assert [int(v) for v in np.asarray(got).ravel()] == want


def test_philox_words_are_uniform():
    n = 1 << 17
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    out = oracle.philox4x32_10(ctr, (0x12345678, 0x9ABCDEF0)).ravel()
    for shift in (0, 8, 16, 24):
        byte = (out >> np.uint32(shift)) & np.uint32(0xFF)
        cnt = np.bincount(byte.astype(np.int64), minlength=256)
        chi2 = ((cnt - cnt.mean()) ** 2 / cnt.mean()).sum()
        p = scipy_stats.chi2.sf(chi2, 255)
        assert 1e-5 < p
    # each of the 32 bits is set half of the time
    bits = ((out[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(out.size))


def test_philox_avalanche():
    rng = np.random.default_rng(3)
    base = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    key = (0xDEADBEEF, 0x01234567)
    y0 = oracle.philox4x32_10(base, key)
    flips = []
    for word in range(4):
        for bit in range(32):
            c = base.copy()
            c[:, word] ^= np.uint32(1 << bit)
            y = oracle.philox4x32_10(c, key)
            diff = np.unpackbits((y ^ y0).view(np.uint8), axis=None).reshape(256, -1).sum(1)
            flips.append(diff.mean())
    flips = np.array(flips)
    assert np.all(np.abs(flips - 64.0) < 3.0)
    # key bits too
    for kb in range(64):
        k = (key[0] ^ (1 << kb), key[1]) if kb < 32 else (key[0], key[1] ^ (1 << (kb - 32)))
        y = oracle.philox4x32_10(base, k)
        assert abs(np.unpackbits((y ^ y0).view(np.uint8)).reshape(256, -1).sum(1).mean() - 64) < 3


def test_philox_counter_words_decorrelate():
    n = 1 << 14
    outs = []
    for w in range(4):
        ctr = np.zeros((n, 4), dtype=np.uint32)
        ctr[:, w] = np.arange(n, dtype=np.uint32)
        outs.append(oracle.philox4x32_10(ctr, (1, 2)).astype(np.float64))
    for o in outs:
        u = o / 2**32
        # lag-1 correlation along the counter and cross-word correlation
        assert abs(np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]) < 0.05
        assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 0.05


def test_bin_normals_are_standard_normal():
    z = np.array([oracle.bin_normal(77, d, t, j, 10, 1, 5)
                  for d in range(4) for t in range(-20, 30) for j in range(-30, 70)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.03
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    # the four lanes of one Philox call are uncorrelated
    zz = np.array([[oracle.bin_normal(9, 0, t, 10 * w + l, 10, 0, 0) for l in range(4)]
                   for t in range(60) for w in range(40)])
    c = np.corrcoef(zz.T)
    assert np.all(np.abs(c - np.eye(4)) < 0.06)


# ------------------------------------------------------------------------------------------
# Convolution
# ------------------------------------------------------------------------------------------

def _rand_grid(seed, nw, nt):
    return np.random.default_rng(seed).normal(size=(nw, nt))


def test_delta_response_is_identity():
    g = _rand_grid(0, 30, 80)
    r = np.zeros((21, 200)); r[10, 0] = 1.0
    np.testing.assert_allclose(oracle.convolve_fft(g, r), g, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(oracle.convolve_direct(g, r), g)


def test_delta_grid_places_the_response():
    resp = synth.make_response("bipolar").astype(np.float64)
    g = np.zeros((40, 400)); g[17, 33] = 1.0
    out = oracle.convolve_fft(g, resp)
    want = np.zeros_like(g)
    for r in range(21):
        w = 17 + (r - 10)
        want[w, 33:233] = resp[r]
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,rshape", [((12, 50), (5, 13)), ((32, 256), (21, 200)),
                                          ((7, 300), (21, 200)), ((25, 64), (3, 64))])
def test_fft_matches_direct_loops(shape, rshape):
    g = _rand_grid(1, *shape)
    r = np.random.default_rng(2).normal(size=rshape)
    a = oracle.convolve_fft(g, r)
    b = oracle.convolve_direct(g, r)
    c = oracle.convolve_direct_np(g, r)
    scale = np.abs(b).max()
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(c, b, rtol=0, atol=1e-12 * scale)


def test_no_circular_wrap():
    resp = synth.make_response("unipolar").astype(np.float64)
    g = np.zeros((30, 300)); g[0, 299] = 1.0; g[29, 299] = 1.0
    out = oracle.convolve_fft(g, resp)
    # a spike at the last tick must leave earlier ticks untouched, and a spike on the
    # first / last wire must not reach the far side of the plane
    assert np.abs(out[:, :299]).max() < 1e-14
    assert np.abs(out[11:19]).max() < 1e-14


def test_convolution_is_linear():
    resp = synth.make_response("bipolar").astype(np.float64)
    a, b = _rand_grid(4, 24, 300), _rand_grid(5, 24, 300)
    lhs = oracle.convolve_fft(2.5 * a - 0.5 * b, resp)
    rhs = 2.5 * oracle.convolve_fft(a, resp) - 0.5 * oracle.convolve_fft(b, resp)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())
