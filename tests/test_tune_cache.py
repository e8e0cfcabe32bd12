"""CPU tests of the schedule autotuner's selection and its persistent cache (fake handles and
timer; the measured path runs in tests/test_gpu_tune.py)."""
import json

import synth
from paper_2304_01841_gb300 import tune

PLANES = [synth.Plane(64, 500), synth.Plane(80, 500)]


class FakeSim:
    def __init__(self, sched, log):
        self.sched, self.closed = sched, False
        log.append(sched)

    def close(self):
        self.closed = True


def _run(tmp_path, speeds, deterministic=False, device="GB300"):
    made = []
    cache = tune.TuneCache(str(tmp_path / "tune.json"))
    best = tune.autotune(PLANES, None, None, object(), candidates=(-1, 4, 1, 0, 6), deterministic=deterministic,
                         cache=cache, device=device, make_sim=lambda s: FakeSim(s, made),
                         timer=lambda sim, d, reps: speeds[sim.sched])
    return best, made


def test_picks_the_fastest_and_persists(tmp_path):
    speeds = {-1: 0.40, 4: 0.42, 1: 0.55, 0: 0.61, 6: 0.39}
    best, made = _run(tmp_path, speeds)
    assert best == 6 and made == [-1, 4, 1, 0, 6]
    data = json.load(open(tmp_path / "tune.json"))
    key = tune.tune_key("GB300", PLANES)
    assert data[key]["schedule_id"] == 6 and float(data[key]["ms"]["1"]) == 0.55
    # a later process reads the cache and times nothing
    best2, made2 = _run(tmp_path, {k: 1.0 for k in speeds})
    assert best2 == 6 and made2 == []


def test_keys_separate_devices_geometry_and_mode(tmp_path):
    speeds = {-1: 0.40, 4: 0.42, 1: 0.55, 0: 0.61, 6: 0.39}
    _run(tmp_path, speeds)
    best, made = _run(tmp_path, speeds, device="other")
    assert made and best == 6
    # deterministic handles use the warp-level rasterizer: +2 schedules are not candidates
    best, made = _run(tmp_path, speeds, deterministic=True)
    assert 6 not in made and best == -1
    assert tune.tune_key("a", PLANES) != tune.tune_key("a", PLANES[:1])


def test_ties_keep_the_earlier_candidate_and_bad_cache_is_ignored(tmp_path):
    (tmp_path / "tune.json").write_text("not json")
    best, made = _run(tmp_path, {-1: 0.5, 4: 0.5, 1: 0.5, 0: 0.5, 6: 0.5})
    assert best == -1 and len(made) == 5


def test_batch_autotune_picks_the_fastest_and_caches_it(tmp_path):
    from paper_2304_01841_gb300 import tune
    planes = [synth.Plane(64, 500)]
    times = {-1: 5.0, 8 | 256: 6.0, 8 | 512: 4.5, 8 | (5 << 4): 4.5, 8 | (4 << 4): 7.0}
    made = []

    class FakeSim:
        def __init__(self, sched):
            self.sched = sched
            made.append(sched)

        def close(self):
            pass

    cache = tune.TuneCache(str(tmp_path / "t.json"))
    best = tune.autotune_batch(planes, None, None, [object()] * 4, cache=cache, device="dev",
                               make_sim=FakeSim, timer=lambda sim, ev, reps: times[sim.sched])
    assert best == 8 | 512 and made == list(tune.BATCH_CANDIDATES)        # ties: the earlier candidate
    made.clear()
    again = tune.autotune_batch(planes, None, None, [object()] * 4, cache=tune.TuneCache(cache.path), device="dev",
                                make_sim=FakeSim, timer=lambda sim, ev, reps: 0.0)
    assert again == best and made == []                                   # from the cache, no timing
    other = tune.autotune_batch(planes, None, None, [object()] * 8, cache=cache, device="dev",
                                make_sim=FakeSim, timer=lambda sim, ev, reps: times[sim.sched])
    assert other == best and len(made) == len(tune.BATCH_CANDIDATES)      # another batch size: measured
