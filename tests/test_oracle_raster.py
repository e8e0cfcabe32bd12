"""Pins for the oracle's rasterization, fluctuation and scatter-add (CPU only)."""
import numpy as np
import pytest

import oracle
import synth


def _one_depo(x=800.0, z=1.35, q=6000.0, n=1):
    return synth.Depos(np.zeros(n), np.full(n, x), np.zeros(n), np.full(n, z), np.full(n, q))


def test_patches_sum_to_charge_inside_grid():
    wl = synth.workload("tiny_inside")
    d = wl.depos()
    pl = wl.planes[0]
    pt = oracle.rasterize(d, pl, wl.diffusion)
    sums = np.array([pt.patch(i).sum() for i in range(d.n)])
    np.testing.assert_allclose(sums, d.q.astype(np.float64), rtol=1e-12, atol=0)
    grid = oracle.scatter(pt, pl)
    assert abs(grid.sum() - d.q.astype(np.float64).sum()) < 1e-9 * d.q.sum()


def test_patch_is_outer_product_of_gaussian_bin_integrals():
    mpmath = pytest.importorskip("mpmath")
    pl = synth.Plane(64, 2048, pitch_origin_mm=0.0)
    diff = synth.Diffusion()
    d = _one_depo(x=1500.0, z=90.0, q=5000.0)
    pt = oracle.rasterize(d, pl, diff)
    P = pt.patch(0)
    _, lo_t, lo_p, nt, npp = pt.desc[0]
    mu_t, s_t, mu_p, s_p = pt.mus[0]
    mpmath.mp.dps = 30

    def binint(mu, s, lo, n):
        f = lambda x: mpmath.exp(-(x - mu) ** 2 / (2 * s * s))
        v = np.array([float(mpmath.quad(f, [lo + i, lo + i + 1])) for i in range(n)])
        return v / v.sum()

    wt = binint(mu_t, s_t, int(lo_t), int(nt))
    wp = binint(mu_p, s_p, int(lo_p), int(npp))
    np.testing.assert_allclose(P, 5000.0 * np.outer(wt, wp), rtol=0, atol=1e-10)


def test_fluctuated_patch_sums_to_charge_and_is_nonnegative():
    wl = synth.workload("tiny_inside")
    d = wl.depos()
    diff = synth.Diffusion(fluctuate=True, seed=99)
    pt = oracle.rasterize(d, wl.planes[0], diff)
    for i in range(0, d.n, 37):
        P = pt.patch(i)
        assert (P >= 0).all()
        assert abs(P.sum() - float(d.q[i])) < 1e-9 * float(d.q[i])


@pytest.mark.parametrize("x", [50.0, 200.0, 1000.0])
def test_fluctuation_moments(x):
    # Many copies of one depo (distinct depo index => independent counters).  Each bin is
    # X_i ~ N(q w_i, q w_i (1 - w_i)), clamped at 0, then the patch is rescaled to sum to q.
    # Where the clamp never acts, the delta method gives the rescaled bin
    #   mean q w_i,   variance q [w_i (1 - w_i)(1 - 2 w_i) + w_i^2 (1 - sum_j w_j^2)].
    # Short drifts (x = 50 mm) give bins with w ~ 0.5, where a dropped (1 - w) or a
    # missing rescale changes the variance by tens of percent.
    n = 8000
    pl = synth.Plane(64, 2048, pitch_origin_mm=0.0)
    d = _one_depo(x=x, z=90.15, q=6000.0, n=n)
    base = oracle.rasterize(d.subset(slice(0, 1)), pl, synth.Diffusion()).patch(0)
    pt = oracle.rasterize(d, pl, synth.Diffusion(fluctuate=True, seed=12345))
    stack = np.stack([pt.patch(i) for i in range(n)])
    q = 6000.0
    w = base / q
    mean = stack.mean(0)
    var = stack.var(0, ddof=1)
    pred = q * (w * (1 - w) * (1 - 2 * w) + w * w * (1 - (w * w).sum()))
    sel = base > 20.0               # bins where the clamp at zero never matters
    assert sel.sum() >= 5
    se = np.sqrt(pred / n)
    assert np.all(np.abs(mean - base)[sel] < 5 * se[sel])
    ratio = var[sel] / pred[sel]
    assert abs(ratio.mean() - 1.0) < 0.03
    assert np.all(np.abs(ratio - 1.0) < 0.08)


def test_fluctuation_vanishes_for_large_charge():
    pl = synth.Plane(64, 2048, pitch_origin_mm=0.0)
    d = _one_depo(x=1000.0, z=90.15, q=1e12)
    a = oracle.rasterize(d, pl, synth.Diffusion()).patch(0)
    b = oracle.rasterize(d, pl, synth.Diffusion(fluctuate=True, seed=5)).patch(0)
    # relative deviation per bin ~ 1/sqrt(q w): < 1e-4 of the largest bin
    assert np.abs(a - b).max() < 1e-4 * a.max()
    assert np.abs(a - b).max() > 0


def test_fluctuation_pool_is_keyed():
    pl = synth.Plane(64, 2048, pitch_origin_mm=0.0)
    d = _one_depo(x=1000.0, z=90.15, q=6000.0, n=2)
    f = lambda seed, ev=0, plane=0: oracle.rasterize(
        synth.Depos(d.t0, d.x, d.y, d.z, d.q, event_id=ev), pl,
        synth.Diffusion(fluctuate=True, seed=seed), plane_index=plane)
    a, b = f(1), f(1)
    assert np.array_equal(a.values, b.values)
    assert not np.array_equal(a.patch(0), a.patch(1))       # depo index
    assert not np.array_equal(f(2).values, a.values)          # seed
    assert not np.array_equal(f(1, ev=3).values, a.values)    # event id
    assert not np.array_equal(f(1, plane=2).values, a.values)  # plane


def test_bin_normal_uses_absolute_coordinates():
    # The deviate of a bin depends on its absolute (tick, impact) only, so two windows that
    # overlap see identical deviates on the overlap.
    z1 = [oracle.bin_normal(3, 0, 100, j, 10, 0, 0) for j in range(-25, 25)]
    z2 = [oracle.bin_normal(3, 0, 100, j, 10, 0, 0) for j in range(-25, 25)]
    assert z1 == z2
    assert len(set(z1)) == len(z1)


def test_scatter_folds_impact_bins_onto_wires_by_hand():
    pl = synth.Plane(4, 6, n_impact_per_pitch=10)
    # depo 0: ticks 1..2, impact bins 8..12 (wires 0 and 1); depo 1: ticks 5..6 (6 off grid),
    # impact -2..1 (wire -1 dropped, wire 0 kept); depo 2: impact 39..40 (wire 3, wire 4 dropped)
    desc = np.array([[0, 1, 8, 2, 5], [10, 5, -2, 2, 4], [18, 0, 39, 1, 2]], dtype=np.int64)
    vals = np.arange(1, 21, dtype=np.float64)
    pt = oracle.Patches(desc, vals, None, 0)
    g = oracle.scatter(pt, pl)
    want = np.zeros((4, 6))
    # depo 0, tick 1 row = [1,2,3,4,5] over impacts 8,9 | 10,11,12
    want[0, 1] += 1 + 2; want[1, 1] += 3 + 4 + 5
    want[0, 2] += 6 + 7; want[1, 2] += 8 + 9 + 10
    # depo 1, tick 5 row = [11,12,13,14] over impacts -2,-1 | 0,1 ; tick 6 dropped
    want[0, 5] += 13 + 14
    # depo 2, tick 0 row = [19, 20] over impacts 39 | 40
    want[3, 0] += 19
    np.testing.assert_array_equal(g, want)


def test_scatter_conserves_in_range_charge():
    wl = synth.workload("tiny")
    d = wl.depos()
    pl = wl.planes[0]
    pt = oracle.rasterize(d, pl, wl.diffusion)
    g = oracle.scatter(pt, pl)
    tot = 0.0
    for i in range(d.n):
        _, lt, lp, nt, npp = (int(v) for v in pt.desc[i])
        P = pt.patch(i)
        ticks = lt + np.arange(nt)
        wires = np.floor_divide(lp + np.arange(npp), 10)
        m = np.outer((ticks >= 0) & (ticks < pl.n_ticks), (wires >= 0) & (wires < pl.n_wires))
        tot += P[m].sum()
    assert abs(g.sum() - tot) < 1e-9 * max(tot, 1.0)


def test_all_core_variants_are_bit_identical_to_the_serial_oracle():
    # the all-core timing variants (depos spread over threads; each thread owning a band of
    # wires for the scatter) compute exactly the serial oracle's patches and grid
    import oracle
    import synth
    wl = synth.workload("tiny")
    d = wl.depos(n_depos=3000)
    pl = wl.planes[0]
    for fl in (False, True):
        diff = synth.Diffusion(fluctuate=fl, seed=91)
        ref = oracle.rasterize(d, pl, diff)
        for threads in (1, 3, 0):
            pt = oracle.rasterize_all_cores(d, pl, diff, n_threads=threads)
            assert np.array_equal(pt.desc, ref.desc) and np.array_equal(pt.values, ref.values)
            assert np.array_equal(oracle.scatter_all_cores(pt, pl, n_threads=threads), oracle.scatter(ref, pl))
    assert oracle.omp_threads(3) in (1, 3)
    wf = oracle.simulate_event_all_cores(d, [pl], synth.Diffusion(fluctuate=True, seed=91), [wl.responses()[0]])
    _, _, w_ref = oracle.simulate_plane(d, pl, synth.Diffusion(fluctuate=True, seed=91), wl.responses()[0])
    assert np.allclose(wf[0], w_ref, rtol=0, atol=1e-9 * np.abs(w_ref).max())
