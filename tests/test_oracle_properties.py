"""Property tests of the oracle's rasterize + scatter on geometry edge cases (a depo on a bin
edge, sigma = 0, partly or wholly off the grid, a single depo, an empty event), with inputs
drawn by hypothesis (CPU only; derandomized so a run is reproducible)."""
import math

import numpy as np
import pytest

import oracle
import synth

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

PL = synth.Plane(40, 400)                  # 40 wires x 3 mm, 400 ticks x 0.5 us, 10 impacts / wire
DIFF = synth.Diffusion(fluctuate=False)
EDGE = st.sampled_from([0.0, 0.25, 0.5, 0.999999, 1.0])
SETTINGS = settings(max_examples=60, deadline=None, derandomize=True)


def _one(t0, x, z, q=5000.0):
    f = np.float32
    return synth.Depos(np.array([t0], f), np.array([x], f), np.array([0.0], f), np.array([z], f),
                       np.array([q], f))


def _in_grid_sum(pt, plane):
    """Charge of the patch bins that fall on the grid, summed bin by bin from the window."""
    tot = 0.0
    off, lo_t, lo_p, nt, npp = (int(v) for v in pt.desc[0])
    p = pt.values[off: off + nt * npp].reshape(nt, npp)
    for a in range(nt):
        for j in range(npp):
            tick, imp = lo_t + a, lo_p + j
            if 0 <= tick < plane.n_ticks and 0 <= imp < plane.n_wires * plane.n_impact_per_pitch:
                tot += p[a, j]
    return tot


@SETTINGS
@given(t0=st.floats(-30.0, 230.0), x=st.floats(0.0, 400.0), z=st.floats(-80.0, 80.0),
       q=st.floats(1.0, 1e6))
def test_patch_keeps_its_charge_and_the_grid_keeps_what_lands_on_it(t0, x, z, q):
    d = _one(t0, x, z, q)
    pt = oracle.rasterize(d, PL, DIFF)
    assert pt.n_invalid == 0
    qf = float(np.float32(q))
    assert abs(pt.values.sum() - qf) <= 1e-9 * qf                   # normalised over the window
    assert (pt.values >= 0).all()
    g = oracle.scatter(pt, PL)
    assert abs(g.sum() - _in_grid_sum(pt, PL)) <= 1e-9 * qf          # off-grid bins dropped


@SETTINGS
@given(k=st.integers(0, 300), frac=EDGE, w=st.integers(2, 37), sub=st.integers(0, 9), sfrac=EDGE)
def test_point_charge_on_a_bin_edge_lands_in_the_bin_above(k, frac, w, sub, sfrac):
    # x = 0: no drift, sigma = 0 in both directions; t0 and z placed on or near bin edges
    t0 = (k + frac) * PL.tick_us
    z = PL.origin_mm + (w * PL.n_impact_per_pitch + sub + sfrac) * PL.pitch_mm / PL.n_impact_per_pitch
    d = _one(t0, 0.0, z)
    pt = oracle.rasterize(d, PL, DIFF)
    off, lo_t, lo_p, nt, npp = (int(v) for v in pt.desc[0])
    assert nt == 1 and npp == 1
    # the bin containing the (float32) coordinates, an edge belonging to the bin above
    t32, z32 = float(np.float32(t0)), float(np.float32(z))
    assert lo_t == math.floor(t32 / PL.tick_us)
    assert lo_p == math.floor((z32 - PL.origin_mm) / (PL.pitch_mm / PL.n_impact_per_pitch))
    g = oracle.scatter(pt, PL)
    if 0 <= lo_t < PL.n_ticks:
        assert g[lo_p // PL.n_impact_per_pitch, lo_t] == pytest.approx(5000.0)


@SETTINGS
@given(t0=st.floats(10.0, 60.0), x=st.floats(1.0, 200.0), z=st.floats(-40.0, 30.0), shift=st.integers(1, 4))
def test_moving_a_depo_by_whole_pitches_moves_the_grid_by_whole_wires(t0, x, z, shift):
    # arrival t0 + x / v stays inside the 200 us window, the depo inside the plane
    a = oracle.scatter(oracle.rasterize(_one(t0, x, z), PL, DIFF), PL)
    b = oracle.scatter(oracle.rasterize(_one(t0, x, z + shift * PL.pitch_mm), PL, DIFF), PL)
    assert a.max() > 0
    # compare where both grids are defined; float32 coordinates move the window by < 1e-5 bin
    np.testing.assert_allclose(b[shift:], a[:-shift], rtol=0, atol=1e-4 * a.max())


def test_empty_event_gives_an_empty_grid():
    f = np.zeros(0, np.float32)
    pt = oracle.rasterize(synth.Depos(f, f, f, f, f), PL, DIFF)
    assert pt.values.size == 0 and not oracle.scatter(pt, PL).any()
