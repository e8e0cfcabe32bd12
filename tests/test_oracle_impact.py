"""Pins of the oracle's impact-resolution path (per-impact-position responses, §2 step 3 with
the transverse grid kept at the patches' resolution)."""
import numpy as np

import oracle
import synth


def _rand_impact_grid(rng, nw, nt, n_imp):
    return rng.normal(size=(nw * n_imp, nt))


def test_phase_independent_response_reduces_to_folded():
    # the same response for every phase: the impact-resolution convolution equals the folded
    # convolution of the per-wire sums of the sub-bins
    rng = np.random.default_rng(1)
    n_imp = 10
    g = _rand_impact_grid(rng, 40, 300, n_imp)
    r = synth.make_response("bipolar").astype(np.float64)
    r_imp = np.repeat(r[None], n_imp, axis=0)
    folded = g.reshape(40, n_imp, 300).sum(axis=1)
    want = oracle.convolve_fft(folded, r)
    got = oracle.convolve_impact(g, r_imp)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_fft_form_equals_literal_loops():
    rng = np.random.default_rng(2)
    for n_imp, nw, nt, kw, kt in [(10, 12, 90, 21, 40), (4, 7, 33, 5, 37), (1, 9, 50, 3, 60)]:
        g = _rand_impact_grid(rng, nw, nt, n_imp)
        r = rng.normal(size=(n_imp, kw, kt))
        got = oracle.convolve_impact(g, r)
        want = oracle.convolve_impact_direct(g, r)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_single_subbin_charge_places_its_phase_response():
    # one unit charge in sub-bin (wire w0, phase p0) at tick t0: wire w0 + k sees
    # resp[p0][k + kc] delayed by t0, nothing else
    n_imp, nw, nt = 10, 30, 400
    r = synth.make_response_impact("unipolar", n_impact=n_imp).astype(np.float64)
    kc = r.shape[1] // 2
    w0, p0, t0 = 13, 7, 25
    g = np.zeros((nw * n_imp, nt))
    g[w0 * n_imp + p0, t0] = 1.0
    out = oracle.convolve_impact(g, r)
    want = np.zeros((nw, nt))
    for row in range(r.shape[1]):
        w = w0 + row - kc
        if 0 <= w < nw:
            want[w, t0:t0 + r.shape[2]] = r[p0, row, : nt - t0]
    assert np.abs(out - want).max() <= 1e-12
    # a different phase of the same wire gives a different waveform (the response depends on it)
    g2 = np.zeros_like(g)
    g2[w0 * n_imp + 2, t0] = 1.0
    assert np.abs(oracle.convolve_impact(g2, r) - out).max() > 1e-4 * np.abs(out).max()


def test_impact_grid_folds_to_the_wire_grid_and_conserves_charge():
    wl = synth.workload("tiny")
    d = wl.depos()
    pl = wl.planes[0]
    pt = oracle.rasterize(d, pl, wl.diffusion)
    g_imp = oracle.scatter_impact(pt, pl)
    g = oracle.scatter(pt, pl)
    folded = g_imp.reshape(pl.n_wires, pl.n_impact_per_pitch, pl.n_ticks).sum(axis=1)
    assert np.abs(folded - g).max() <= 1e-9 * np.abs(g).max()
    assert g_imp.sum() > 0 and abs(g_imp.sum() - g.sum()) <= 1e-9 * g.sum()


def test_impact_responses_mirror_and_vary_across_the_pitch():
    r = synth.make_response_impact("bipolar", n_impact=10)
    assert r.shape == (10, 21, 200)
    assert np.array_equal(r[3], r[6][::-1])                  # phase p at k == phase n-1-p at -k
    # near the wire the response changes with the phase, far away hardly at all
    near = np.abs(r[0, 10] - r[9, 10]).max() / np.abs(r[0, 10]).max()
    assert near < 1e-6                                       # symmetric distances +-0.45
    assert np.abs(r[0, 11] - r[9, 11]).max() > 1e-2 * np.abs(r[0, 11]).max()
