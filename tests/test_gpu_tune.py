"""The schedule autotuner measured on the GPU: it times every candidate schedule, caches the
choice, and the chosen schedule gives the oracle's waveforms."""
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


def test_autotune_measures_caches_and_stays_exact(tmp_path):
    import paper_2304_01841_gb300 as g
    from paper_2304_01841_gb300 import tune
    wl = synth.workload("uboone_plane")
    d = wl.depos(n_depos=20000)
    dev = g.DeviceDepos.from_host(d)
    cache = tune.TuneCache(str(tmp_path / "tune.json"))
    best = tune.autotune(wl.planes, wl.responses(), wl.diffusion, dev, reps=3, cache=cache)
    assert best in tune.CANDIDATES
    entry = cache.entries[tune.tune_key(torch.cuda.get_device_name(), wl.planes)]
    assert set(int(k) for k in entry["ms"]) == set(tune.CANDIDATES)
    assert all(v > 0 for v in entry["ms"].values())
    assert tune.TuneCache(cache.path).get(tune.tune_key(torch.cuda.get_device_name(), wl.planes)) == best
    sim = make_sim(wl.planes, wl.responses(), wl.diffusion, schedule_id=best)
    wf = to_np(sim.run_event(dev)[0])
    sim.sync()
    _, _, ref = oracle.simulate_plane(d, wl.planes[0], wl.diffusion, wl.responses()[0])
    assert rel_l2(wf, ref) <= WAVE_RTOL


def test_batch_autotune_measures_and_stays_exact(tmp_path):
    import numpy as np
    import paper_2304_01841_gb300 as g
    from paper_2304_01841_gb300 import tune
    wl = synth.workload("three_plane")
    evs = [wl.depos(n_depos=n, seed=40 + i, event_id=60 + i) for i, n in enumerate((6000, 15000, 3000, 9000))]
    dev = [g.DeviceDepos.from_host(e) for e in evs]
    cache = tune.TuneCache(str(tmp_path / "tune.json"))
    best = tune.autotune_batch(wl.planes, wl.responses(), wl.diffusion, dev, reps=2, cache=cache)
    assert best in tune.BATCH_CANDIDATES
    sim = make_sim(wl.planes, wl.responses(), wl.diffusion, schedule_id=best)
    out = sim.run_batch(dev)
    sim.sync()
    for p in range(3):
        _, _, ref = oracle.simulate_plane(evs[1], wl.planes[p], wl.diffusion, wl.responses()[p], plane_index=p)
        assert rel_l2(to_np(out[1][p]), ref) <= WAVE_RTOL
