"""CPU tests of the benchmark's host-side arithmetic: algorithmic bytes per stage (the figures
the roofline fractions divide by) and the weak-scaling shard plan."""
import bench
import synth


def test_stage_bytes_of_the_benchmarked_plane():
    pl = synth.workload("uboone_plane").planes[0]
    sb = bench.stage_bytes(pl, 100_000, spec_bins=2150)
    grid = 4 * 3456 * 9600
    spec = 8 * 3456 * 2150
    assert sb["raster_scatter"] == 20 * 100_000 + grid
    assert sb["row_r2c"] == grid + spec == sb["row_c2r"]
    assert sb["wire_stage"] == 2 * spec
    assert sb["convolve"] == 2 * grid + 2 * spec == 384_307_200
    # the spectrum is never counted beyond the unpadded half length (n_ticks + 199) / 2 + 1
    full = bench.stage_bytes(pl, 100_000, spec_bins=10**6)
    assert full["wire_stage"] == 2 * 8 * 3456 * ((9600 + 199) // 2 + 1)


def test_shard_plan_gives_disjoint_events_per_rank():
    plans = [bench.shard_plan(r, 4, 16, 20230405) for r in range(4)]
    seeds = [s for p in plans for s, _ in p]
    ids = [e for p in plans for _, e in p]
    assert len(set(seeds)) == len(seeds) == 64 and sorted(ids) == list(range(64))
    assert bench.shard_plan(0, 1, 16, 20230405) == plans[0]     # rank 0 is the same at any N


def test_unpruned_and_classical_bytes_of_the_three_planes():
    # the unpruned byte model: grid read + waveform write + one spectrum round trip at every bin
    # of the unpadded half spectrum (1286 MB for the three-plane event); the classical
    # three-pass 2D-FFT schedule moves three more spectra
    planes = synth.workload("three_plane").planes
    unp = sum(bench.unpruned_convolve_bytes(p)[0] for p in planes)
    cls = sum(bench.unpruned_convolve_bytes(p)[1] for p in planes)
    spec = sum(8 * p.n_wires * ((p.n_ticks + 199) // 2 + 1) for p in planes)
    grid = sum(4 * p.n_wires * p.n_ticks for p in planes)
    assert unp == 2 * grid + 2 * spec and abs(unp / 1e6 - 1286) < 5
    assert cls - unp == 3 * spec


def test_benchmarked_batch_recipe():
    # 64 events, counts lognormal 10k..500k, distinct event ids, per-rank pools disjoint
    counts = synth.batch_depo_counts(64)
    assert counts.min() >= 10_000 and counts.max() <= 500_000 and 60_000 < counts.mean() < 160_000
    a = bench.rank_events(0, 4)
    b = bench.rank_events(1, 4)
    assert [e.event_id for e in a] == [5000, 5001, 5002, 5003] and [e.event_id for e in b] == [5004, 5005, 5006, 5007]
    assert not any(np_equal(x.x, y.x) for x, y in zip(a, b))


def np_equal(u, v):
    import numpy as np
    return u.shape == v.shape and bool(np.array_equal(u, v))
