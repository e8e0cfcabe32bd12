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
