"""GPU tests of the batched and served forms: every event gives the result it gives alone."""
import numpy as np
import pytest

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


def _small_three_plane():
    a = np.radians(60.0)
    planes = [synth.Plane(96, 1200, wire_angle_rad=a, pitch_origin_mm=-144.0, response_kind="bipolar"),
              synth.Plane(96, 1200, wire_angle_rad=-a, pitch_origin_mm=-144.0, response_kind="bipolar"),
              synth.Plane(120, 1200, pitch_origin_mm=-180.0, response_kind="unipolar")]
    responses = [synth.make_response(p.response_kind) for p in planes]
    return planes, responses


def _events(n_events, seed=0, lo=50, hi=4000, id0=0):
    rng = np.random.default_rng(seed)
    out = []
    for e in range(n_events):
        n = int(rng.integers(lo, hi))
        d = synth.make_track_depos(rng, n, 3, rng.uniform(50, 250, 3), [0, -40, -150], [900, 40, 150], True)
        d.event_id = id0 + e
        out.append(d)
    return out


def _close(a, b, scale):
    return float(np.abs(a - b).max()) <= 1e-5 * max(scale, 1.0)


def test_batch_multiplane_matches_single_and_graph_replay():
    import paper_2304_01841_gb300 as g
    planes, responses = _small_three_plane()
    diff = synth.Diffusion(fluctuate=True, seed=77)
    sim = make_sim(planes, responses, diff)
    evs = _events(7, seed=1)
    dev = [g.DeviceDepos.from_host(e) for e in evs]
    outs = [[torch.empty((p.n_wires, p.n_ticks), device="cuda") for p in planes] for _ in evs]
    singles = [[w.clone() for w in sim.run_event(d)] for d in dev]
    for rep in range(3):                      # direct, recorded, replayed
        sim.run_batch(dev, outs)
        sim.sync()
        for e in range(len(evs)):
            for p in range(len(planes)):
                s = to_np(singles[e][p])
                assert _close(to_np(outs[e][p]), s, np.abs(s).max()), (rep, e, p)
    assert sim.counters()["graph_launches"] >= 2
    # same pointers, new depo values: the replayed graph reads the new values
    new = _events(7, seed=2)
    for e, (d, n) in enumerate(zip(dev, new)):
        m = min(d.n, n.n)
        for name in ("t0", "x", "y", "z", "q"):
            src = np.zeros(d.n, np.float32)
            src[:m] = getattr(n, name)[:m]
            getattr(d, name).copy_(torch.from_numpy(src))
    sim.run_batch(dev, outs)
    want = [[w.clone() for w in sim.run_event(d)] for d in dev]
    sim.sync()
    for e in range(len(evs)):
        for p in range(len(planes)):
            s = to_np(want[e][p])
            assert _close(to_np(outs[e][p]), s, np.abs(s).max())


def test_batch_with_empty_off_plane_and_single_depo_events():
    # degenerate members of a batch: an empty event, events whose depos all fall outside the
    # planes (beyond the wires, beyond the ticks), a one-depo event and one event passed twice,
    # mixed with ordinary ones; every waveform is written (outputs start at 7), the degenerate
    # ones are exactly zero, and every event matches the FP64 oracle
    import oracle
    import paper_2304_01841_gb300 as g
    planes, responses = _small_three_plane()
    diff = synth.Diffusion(fluctuate=True, seed=91)
    sim = make_sim(planes, responses, diff)
    base = _events(3, seed=5, lo=300, hi=900, id0=40)
    empty = base[0].subset(slice(0, 0))
    empty.event_id = 50
    beyond_wires = base[1].subset(slice(None))
    beyond_wires.z = beyond_wires.z + np.float32(5000.0)     # pitch far beyond every plane's wires
    beyond_wires.y = beyond_wires.y + np.float32(5000.0)
    beyond_wires.event_id = 51
    beyond_ticks = base[2].subset(slice(None))
    beyond_ticks.t0 = beyond_ticks.t0 + np.float32(1e4)      # arrivals after the last tick
    beyond_ticks.event_id = 52
    one = base[0].subset(slice(3, 4))
    one.event_id = 53
    evs = [base[0], empty, beyond_wires, one, base[1], beyond_ticks, base[2]]
    dev = [g.DeviceDepos.from_host(e) for e in evs]
    evs.append(base[0])                                       # the same device arrays twice
    dev.append(dev[0])
    outs = [[torch.full((p.n_wires, p.n_ticks), 7.0, device="cuda") for p in planes] for _ in evs]
    sim.run_batch(dev, outs)
    sim.sync()
    for e, d in enumerate(evs):
        for p in range(len(planes)):
            got = to_np(outs[e][p])
            if e in (1, 2, 5):
                assert float(np.abs(got).max()) == 0.0, (e, p)
                continue
            _, _, ref = oracle.simulate_plane(d, planes[p], diff, responses[p], plane_index=p)
            assert rel_l2(got, ref) <= WAVE_RTOL, (e, p)


def test_batch_schedules_and_memory_limit_match_single_events():
    # one persistent raster launch for the whole batch (the default), chunks of 2 events that
    # pipeline with the previous chunk's convolutions, a single convolution stream, and a budget
    # that leaves room for only two batch grid sets (chunks of one event, alternating): every
    # event equals run_event, and the default issues exactly one raster launch per batch
    import paper_2304_01841_gb300 as g
    planes, responses = _small_three_plane()
    diff = synth.Diffusion(fluctuate=True, seed=78)
    evs = _events(7, seed=5)
    evs[3] = synth.Depos(*(np.zeros(0, np.float32) for _ in range(5)))
    evs[3].event_id = 3
    ref_sim = make_sim(planes, responses, diff)
    dev = [g.DeviceDepos.from_host(e) for e in evs]
    singles = [[to_np(w) for w in ref_sim.run_event(d)] for d in dev]
    ref_sim.sync()
    # the handle's memory for one event at a time, less the spectra of run_event's second
    # convolution stream (the one-stream batch below takes none)
    infos = [ref_sim.plane_info(i) for i in range(len(planes))]
    fork_bytes = 2 * 8 * max(i["n_wires"] * i["spectrum_row_stride"] for i in infos) + 2 * max(p.n_wires for p in planes)
    base = ref_sim.counters()["device_bytes"] - fork_bytes
    set_bytes = sum(4 * p.n_wires * p.n_ticks + 4 * (2 * ref_sim.plane_info(i)["n_tiles"] + 2)
                    for i, p in enumerate(planes))
    ref_sim.close()

    def check(sim, label):
        outs = [[torch.full((p.n_wires, p.n_ticks), float("nan"), device="cuda") for p in planes] for _ in evs]
        for rep in range(2):
            sim.run_batch(dev, outs)
            sim.sync()
            for e in range(len(evs)):
                for p in range(len(planes)):
                    assert _close(to_np(outs[e][p]), singles[e][p], np.abs(singles[e][p]).max()), (label, rep, e, p)

    sim = make_sim(planes, responses, diff)
    n0 = sim.counters()["kernel_launches"]
    outs = [[torch.empty((p.n_wires, p.n_ticks), device="cuda") for p in planes] for _ in evs]
    sim.run_batch(dev, outs)
    sim.sync()
    # one raster launch; per (event, plane) pair: row activity, forward transform, wire stage,
    # inverse transform
    assert sim.counters()["kernel_launches"] - n0 == 1 + 4 * len(evs) * len(planes)
    check(sim, "default")
    sim.close()
    for sched, label in ((8 | (2 << 4), "chunks of 2"), (8 | 256, "one convolution stream")):
        sim = make_sim(planes, responses, diff, schedule_id=sched)
        check(sim, label)
        sim.close()
    sim = make_sim(planes, responses, diff, schedule_id=8 | 256, hbm_budget_bytes=base + int(2.5 * set_bytes))
    check(sim, "two grid sets")
    assert sim.counters()["device_bytes"] <= base + int(2.5 * set_bytes)
    sim.close()


def test_server_results_same_alone_and_in_mix():
    import paper_2304_01841_gb300 as g
    from paper_2304_01841_gb300.serve import EventServer
    planes, responses = _small_three_plane()
    diff = synth.Diffusion(fluctuate=True, seed=5)
    evs = _events(24, seed=3, lo=10, hi=6000, id0=300)
    evs[7] = evs[7].subset(slice(0, 0))        # an empty request among the others
    srv = EventServer(planes, responses, diff, n_slots=3, max_batch=4, hbm_budget_bytes=64 << 20,
                      keep_results=True)
    reqs = [srv.submit(e) for e in evs[:10]]
    srv.step()                                 # some requests start while others still arrive
    reqs += [srv.submit(e) for e in evs[10:]]
    srv.drain()
    sim = make_sim(planes, responses, diff)
    for r, e in zip(reqs, evs):
        alone = [to_np(w) for w in sim.run_event(g.DeviceDepos.from_host(e))]
        for p in range(len(planes)):
            assert _close(r.waveforms[p], alone[p], np.abs(alone[p]).max()), (r.rid, p)
        assert r.latency > 0
    srv.close()


def test_server_respects_hbm_budget():
    from paper_2304_01841_gb300.serve import EventServer
    planes, responses = _small_three_plane()
    evs = _events(12, seed=4, lo=100, hi=2000, id0=500)
    one = 20 * 2000 + sum(4 * p.n_wires * p.n_ticks for p in planes)
    srv = EventServer(planes, responses, synth.Diffusion(), n_slots=4, max_batch=4, hbm_budget_bytes=2 * one)
    for e in evs:
        srv.submit(e)
    peak = 0
    while srv.step() > 0:
        peak = max(peak, srv.in_use)
    assert 0 < peak <= 2 * one
    assert len(srv.completed) == len(evs)
    srv.close()


def test_run_host_matches_run_event():
    # host depos -> host waveforms through the pipelined entry point: pinned tensors and plain
    # numpy inputs, an empty event, more events than staging buffers, then a larger event that
    # grows the staging
    import paper_2304_01841_gb300 as g
    planes, responses = _small_three_plane()
    diff = synth.Diffusion(fluctuate=True, seed=11)
    sim = make_sim(planes, responses, diff)
    evs = _events(5, seed=7, lo=100, hi=3000, id0=900)
    evs.append(synth.Depos(*(np.zeros(0, np.float32) for _ in range(5))))
    evs[-1].event_id = 950
    pinned = []
    for i, e in enumerate(evs):
        if i % 2 == 0:
            o = type("P", (), {})()
            for k in ("t0", "x", "y", "z", "q"):
                setattr(o, k, torch.from_numpy(np.ascontiguousarray(getattr(e, k), dtype=np.float32)).pin_memory())
            o.event_id = e.event_id
            pinned.append(o)
        else:
            pinned.append(e)
    outs = sim.run_host(pinned)
    for e, ev in enumerate(evs):
        want = [to_np(w) for w in sim.run_event(g.DeviceDepos.from_host(ev))]
        sim.sync()
        for p in range(len(planes)):
            got = outs[e][p].numpy()
            assert _close(got, want[p], np.abs(want[p]).max()), (e, p)
    big = _events(1, seed=8, lo=20000, hi=20001, id0=990)
    out_np = [[np.empty((p.n_wires, p.n_ticks), np.float32) for p in planes]]
    sim.run_host(big, outs=out_np)
    want = [to_np(w) for w in sim.run_event(g.DeviceDepos.from_host(big[0]))]
    sim.sync()
    for p in range(len(planes)):
        assert _close(out_np[0][p], want[p], np.abs(want[p]).max())


def test_benchmarked_batch_of_64_three_plane_events_sampled():
    # the batched configuration the benchmark times: 64 three-plane events (2400/2400/3456 x
    # 9600), depo counts lognormal 10k..500k cut from track pools, one run_batch replayed from
    # its graph; one event in 16 against the oracle on every plane
    import bench
    import oracle
    import paper_2304_01841_gb300 as g
    wl = synth.workload("three_plane")
    evs = bench.rank_events(0, 64)
    sim = make_sim(wl.planes, wl.responses(), wl.diffusion)
    dev = [g.DeviceDepos.from_host(e) for e in evs]
    outs = [[torch.empty((p.n_wires, p.n_ticks), dtype=torch.float32, device="cuda") for p in wl.planes]
            for _ in evs]
    sim.run_batch(dev, outs)
    sim.run_batch(dev, outs)
    sim.sync()
    for e in range(0, 64, 16):
        for p, pl in enumerate(wl.planes):
            _, _, ref = oracle.simulate_plane(evs[e], pl, wl.diffusion, wl.responses()[p], plane_index=p)
            assert rel_l2(to_np(outs[e][p]), ref) <= 1e-4, (e, p)


def test_served_apa_mix_sampled():
    # the served configuration: APA-like planes (800/800/960 x 6000), a heavy-tailed mix of
    # small events and a 1M-depo one through the event server; the large event and a small one
    # against the oracle
    import oracle
    from paper_2304_01841_gb300.serve import EventServer, pin_depos
    wl = synth.workload("dune_apa")
    pool = [wl.depos(n_depos=1_000_000, seed=wl.seed + 1)]
    counts = [20_000, 1_000_000, 8_000, 45_000, 5_000, 30_000]
    evs = synth.slice_events(pool, counts, np.random.default_rng(11), 9000)
    srv = EventServer(wl.planes, wl.responses(), wl.diffusion, n_slots=4, max_batch=8, hbm_budget_bytes=24 << 30,
                      keep_results=True)
    reqs = [srv.submit(pin_depos(e)) for e in evs]
    srv.drain()
    for i in (1, 2):
        for p, pl in enumerate(wl.planes):
            _, _, ref = oracle.simulate_plane(evs[i], pl, wl.diffusion, wl.responses()[p], plane_index=p)
            assert rel_l2(np.asarray(reqs[i].waveforms[p]), ref) <= 1e-4, (i, p)
    srv.close()
