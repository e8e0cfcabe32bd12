"""GPU parity of the impact mode (per-impact-position responses) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import WAVE_RTOL, make_sim, rel_l2, to_np

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


@pytest.mark.parametrize("nw,nt,kind", [(256, 1024, "bipolar"), (700, 9600, "unipolar"), (37, 1000, "bipolar")])
def test_convolve_impact_random_phase_grids(nw, nt, kind):
    pl = synth.Plane(nw, nt, response_kind=kind)
    r_imp = synth.make_response_impact(kind, n_impact=pl.n_impact_per_pitch)
    sim = make_sim([pl], [synth.make_response(kind)], synth.Diffusion())
    sim.set_impact_responses(0, r_imp)
    g = np.random.default_rng(nw + nt).normal(size=(pl.n_impact_per_pitch, nw, nt)).astype(np.float32)
    out = sim.convolve_impact(0, torch.from_numpy(g).cuda())
    sim.sync()
    # phase-major grids [p][w'] are the impact rows n_imp w' + p
    g_imp = np.transpose(g, (1, 0, 2)).reshape(nw * pl.n_impact_per_pitch, nt)
    ref = oracle.convolve_impact(g_imp, r_imp, workers=4)
    assert rel_l2(to_np(out), ref) <= WAVE_RTOL


def test_run_event_impact_tiny_and_reduced_uboone():
    for name, n in (("tiny", None), ("uboone_plane", 20000)):
        wl = synth.workload(name)
        pl = wl.planes[0]
        d = wl.depos(n_depos=n) if n else wl.depos()
        r_imp = synth.make_response_impact(pl.response_kind, n_impact=pl.n_impact_per_pitch)
        diff = synth.Diffusion(fluctuate=True, seed=31)
        sim = make_sim([pl], [synth.make_response(pl.response_kind)], diff)
        sim.set_impact_responses(0, r_imp)
        wf = sim.run_event(_dev(d))[0]
        sim.sync()
        _, _, ref = oracle.simulate_plane_impact(d, pl, diff, r_imp)
        assert rel_l2(to_np(wf), ref) <= WAVE_RTOL, name


def test_phase_independent_responses_match_folded_mode_and_switch_back():
    wl = synth.workload("tiny")
    pl = wl.planes[0]
    r = synth.make_response(pl.response_kind)
    d = wl.depos()
    sim = make_sim([pl], [r], wl.diffusion)
    folded = to_np(sim.run_event(_dev(d))[0])
    sim.set_impact_responses(0, np.repeat(r[None], pl.n_impact_per_pitch, axis=0))
    imp = to_np(sim.run_event(_dev(d))[0])
    sim.set_impact_responses(0, None)
    back = to_np(sim.run_event(_dev(d))[0])
    sim.sync()
    assert rel_l2(imp, folded) <= WAVE_RTOL
    assert np.abs(back - folded).max() <= 1e-5 * np.abs(folded).max()


def test_run_batch_and_run_host_in_impact_mode():
    wl = synth.workload("tiny")
    pl = wl.planes[0]
    r_imp = synth.make_response_impact(pl.response_kind, n_impact=pl.n_impact_per_pitch)
    diff = synth.Diffusion(fluctuate=True, seed=9)
    sim = make_sim([pl], [synth.make_response(pl.response_kind)], diff)
    sim.set_impact_responses(0, r_imp)
    rng = np.random.default_rng(4)
    evs = []
    for e in range(3):
        d = wl.depos()
        keep = rng.random(d.n) < 0.7
        ev = synth.Depos(d.t0[keep], d.x[keep], d.y[keep], d.z[keep], d.q[keep])
        ev.event_id = 40 + e
        evs.append(ev)
    dev = [_dev(e) for e in evs]
    batch = sim.run_batch(dev)
    hosts = sim.run_host(evs)
    sim.sync()
    for e, ev in enumerate(evs):
        _, _, ref = oracle.simulate_plane_impact(ev, pl, diff, r_imp)
        assert rel_l2(to_np(batch[e][0]), ref) <= WAVE_RTOL
        assert rel_l2(hosts[e][0].numpy(), ref) <= WAVE_RTOL


def test_impact_responses_are_validated():
    import paper_2304_01841_gb300 as g
    pl = synth.Plane(64, 500)
    sim = make_sim([pl], [synth.make_response("bipolar")], synth.Diffusion())
    with pytest.raises(g.WctError):
        sim.set_impact_responses(0, synth.make_response_impact("bipolar", n_impact=4))     # phases != n_imp
    with pytest.raises(g.WctError):
        sim.convolve_impact(0, torch.zeros((10, 64, 500), device="cuda"))                  # not in impact mode


def test_responses_ingested_from_a_field_response():
    # field response -> tick responses through the C ABI; the folded and the impact modes with
    # them against the oracle given the same arrays
    import paper_2304_01841_gb300 as g
    wl = synth.workload("tiny")
    pl = wl.planes[0]
    pos, cur = synth.make_field_response(pl.response_kind, pitch_mm=pl.pitch_mm)
    e = synth.electronics_crrc2(0.1, 1.0, 200)
    imp, fold = g.response_from_field(g.FieldResponse(pos, cur, 0.1), e, pl.pitch_mm, pl.n_impact_per_pitch,
                                      pl.tick_us)
    d = wl.depos()
    diff = synth.Diffusion(fluctuate=True, seed=12)
    sim = make_sim([pl], [fold], diff)
    folded = to_np(sim.run_event(_dev(d))[0])
    sim.set_impact_responses(0, imp)
    resolved = to_np(sim.run_event(_dev(d))[0])
    sim.sync()
    _, _, ref_f = oracle.simulate_plane(d, pl, diff, fold)
    _, _, ref_i = oracle.simulate_plane_impact(d, pl, diff, imp)
    assert rel_l2(folded, ref_f) <= WAVE_RTOL
    assert rel_l2(resolved, ref_i) <= WAVE_RTOL
    # the field varies across the pitch, so resolving the impact position changes the answer
    assert rel_l2(resolved, folded) > 10 * WAVE_RTOL
