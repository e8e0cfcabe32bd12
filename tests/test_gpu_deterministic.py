"""GPU tests of the deterministic mode (fixed-point integer accumulation of the scatter-add):
bitwise-identical results whatever the order in which contributions land, and parity with
the oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import BIN_TOL, WAVE_RTOL, make_sim, max_rel_bin, rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_01841_gb300 as g
    g.load(build_if_missing=True)


def _dev(d):
    import paper_2304_01841_gb300 as g
    return g.DeviceDepos.from_host(d)


def _permuted(d, seed):
    p = np.random.default_rng(seed).permutation(d.n)
    out = synth.Depos(d.t0[p], d.x[p], d.y[p], d.z[p], d.q[p])
    out.event_id = d.event_id
    return out


def test_depo_order_does_not_change_a_bit():
    # fluctuation off: the same multiset of contributions in another order (other warps, other
    # atomics) gives bit-identical grids and waveforms on every plane
    wl = synth.workload("three_plane")
    d = wl.depos(n_depos=60000)
    dp = _permuted(d, 1)
    diff = synth.Diffusion(fluctuate=False)
    sim = make_sim(wl.planes, wl.responses(), diff, deterministic=True)
    a = [w.clone() for w in sim.run_event(_dev(d))]
    b = [w.clone() for w in sim.run_event(_dev(dp))]
    ga = [sim.scatter(p, _dev(d)).clone() for p in range(len(wl.planes))]
    gb = [sim.scatter(p, _dev(dp)).clone() for p in range(len(wl.planes))]
    sim.sync()
    for p in range(len(wl.planes)):
        assert torch.equal(a[p], b[p]), p
        assert torch.equal(ga[p], gb[p]), p
        _, grid, wf = oracle.simulate_plane(d, wl.planes[p], diff, wl.responses()[p], plane_index=p)
        assert max_rel_bin(to_np(ga[p]), grid) <= BIN_TOL
        assert rel_l2(to_np(a[p]), wf) <= WAVE_RTOL


def test_patch_scatter_is_order_independent():
    # the unfused path (patches, then the tile scatter) in the deterministic mode
    wl = synth.workload("tiny")
    d = wl.depos()
    dp = _permuted(d, 2)
    diff = synth.Diffusion(fluctuate=False)
    sim = make_sim(wl.planes, wl.responses(), diff, deterministic=True)
    grids = []
    for dd in (d, dp):
        dev = _dev(dd)
        desc, patches = sim.rasterize(0, dev)
        grids.append(sim.scatter(0, dev, patches=patches, patch_desc=desc).clone())
    sim.sync()
    assert torch.equal(grids[0], grids[1])
    ref = oracle.scatter(oracle.rasterize(d, wl.planes[0], diff), wl.planes[0])
    assert max_rel_bin(to_np(grids[0]), ref) <= BIN_TOL


def test_batch_and_repeats_are_bit_identical_with_fluctuation():
    wl = synth.workload("uboone_plane")
    diff = synth.Diffusion(fluctuate=True, seed=77)
    sim = make_sim(wl.planes, wl.responses(), diff, deterministic=True)
    evs = []
    for e, n in enumerate((100000, 30000, 5000)):
        d = wl.depos(n_depos=n, seed=500 + e)
        d.event_id = 900 + e
        evs.append(d)
    dev = [_dev(e) for e in evs]
    batch = [[w.clone() for w in ev] for ev in sim.run_batch(dev)]
    again = [[w.clone() for w in ev] for ev in sim.run_batch(dev)]
    singles = [sim.run_event(e)[0].clone() for e in dev]
    sim.sync()
    for e in range(len(evs)):
        assert torch.equal(batch[e][0], again[e][0]), e
        assert torch.equal(batch[e][0], singles[e]), e
    _, _, ref = oracle.simulate_plane(evs[0], wl.planes[0], diff, wl.responses()[0])
    assert rel_l2(to_np(singles[0]), ref) <= WAVE_RTOL


def test_impact_mode_is_order_independent():
    wl = synth.workload("tiny")
    pl = wl.planes[0]
    r_imp = synth.make_response_impact(pl.response_kind, n_impact=pl.n_impact_per_pitch)
    diff = synth.Diffusion(fluctuate=False)
    d = wl.depos()
    dp = _permuted(d, 3)
    sim = make_sim([pl], [synth.make_response(pl.response_kind)], diff, deterministic=True)
    sim.set_impact_responses(0, r_imp)
    a = sim.run_event(_dev(d))[0].clone()
    b = sim.run_event(_dev(dp))[0].clone()
    sim.sync()
    assert torch.equal(a, b)
    _, _, ref = oracle.simulate_plane_impact(d, pl, diff, r_imp)
    assert rel_l2(to_np(a), ref) <= WAVE_RTOL
