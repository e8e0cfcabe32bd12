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
