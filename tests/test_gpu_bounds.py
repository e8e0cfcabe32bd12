"""The bounds-checked build (-DWCT_BOUNDS_CHECK) run over every kernel path on representative
workloads: no index is ever out of range, and the results still match the oracle.  It runs in a
child process that loads the checked library ($WCT_LIB)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes, os, sys
sys.path.insert(0, ROOT); sys.path.insert(0, os.path.join(ROOT, "tests"))
import numpy as np, torch
import oracle, synth
import paper_2304_01841_gb300 as g
from helpers import WAVE_RTOL, BIN_TOL, rel_l2, max_rel_bin, to_np
lib = g.load()
assert lib._name == os.environ["WCT_LIB"], lib._name
rec = (ctypes.c_int64 * 3)()
def clean(sim):
    sim.sync()
    assert lib.wct_debug_bounds(sim._h, rec) == 0
    assert list(rec) == [0, 0, 0], list(rec)
dev = g.DeviceDepos.from_host
# three planes, fluctuation, fused path + batch + host path
wl = synth.workload("three_plane")
evs = [wl.depos(n_depos=n, seed=300 + i, event_id=10 + i) for i, n in enumerate((40000, 3000, 12000))]
evs.append(synth.Depos(*(np.zeros(0, np.float32) for _ in range(5))))
for det in (False, True):
    sim = g.Simulator(wl.planes, wl.responses(), wl.diffusion, deterministic=det)
    wfs = [[w.clone() for w in sim.run_event(dev(e))] for e in evs]
    batch = sim.run_batch([dev(e) for e in evs])
    host = sim.run_host(evs[:2])
    clean(sim)
    for p in range(3):
        _, _, ref = oracle.simulate_plane(evs[0], wl.planes[p], wl.diffusion, wl.responses()[p], plane_index=p)
        assert rel_l2(to_np(wfs[0][p]), ref) <= WAVE_RTOL
        assert rel_l2(to_np(batch[0][p]), ref) <= WAVE_RTOL
        assert rel_l2(host[0][p].numpy(), ref) <= WAVE_RTOL
    sim.close()
# unfused patches (scanned and fixed slots) + tile scatter, wide windows, CTA-level rasterizer
tiny = synth.workload("tiny")
d = tiny.depos()
for sched in (-1, 6, 0, 1):
    sim = g.Simulator(tiny.planes, tiny.responses(), synth.Diffusion(fluctuate=True, seed=4), schedule_id=sched)
    dd = dev(d)
    desc, patches = sim.rasterize(0, dd)
    grid = sim.scatter(0, dd, patches=patches, patch_desc=desc)
    fused = sim.scatter(0, dd)
    slot = sim.patch_slot_bins(0, float(d.x.max()))
    desc_f, patches_f = sim.rasterize_fixed(0, dd, slot)
    grid_f = sim.scatter(0, dd, patches=patches_f, patch_desc=desc_f)
    wf = sim.run_event(dd)[0]
    clean(sim)
    ref = oracle.scatter(oracle.rasterize(d, tiny.planes[0], synth.Diffusion(fluctuate=True, seed=4)), tiny.planes[0])
    assert max_rel_bin(to_np(grid), ref) <= BIN_TOL and max_rel_bin(to_np(fused), ref) <= BIN_TOL
    assert max_rel_bin(to_np(grid_f), ref) <= BIN_TOL
    # an undersized slot: the skipped depos are reported (WCT_EINVAL), no index goes out of range
    desc_x, patches_x = sim.rasterize_fixed(0, dd, 24)
    sim.scatter(0, dd, patches=patches_x, patch_desc=desc_x)
    try:
        sim.sync()
        raise AssertionError("undersized slots were not reported")
    except g.WctError as e:
        assert e.code == 1
    assert lib.wct_debug_bounds(sim._h, rec) == 0 and list(rec) == [0, 0, 0], list(rec)
    sim.close()
# impact mode, both accumulation modes
pl = tiny.planes[0]
r_imp = synth.make_response_impact(pl.response_kind, n_impact=pl.n_impact_per_pitch)
for det in (False, True):
    sim = g.Simulator([pl], [synth.make_response(pl.response_kind)], tiny.diffusion, deterministic=det)
    sim.set_impact_responses(0, r_imp)
    wf = to_np(sim.run_event(dev(d))[0])
    clean(sim)
    _, _, ref = oracle.simulate_plane_impact(d, pl, tiny.diffusion, r_imp)
    assert rel_l2(wf, ref) <= WAVE_RTOL
    sim.close()
# the benchmark's plane at full size, one event
u = synth.workload("uboone_plane")
sim = g.Simulator(u.planes, u.responses(), u.diffusion)
du = u.depos()
wf = to_np(sim.run_event(dev(du))[0])
clean(sim)
_, _, ref = oracle.simulate_plane(du, u.planes[0], u.diffusion, u.responses()[0])
assert rel_l2(wf, ref) <= WAVE_RTOL
print("bounds ok")
"""


def test_checked_build_sees_no_out_of_range_index():
    from paper_2304_01841_gb300 import build
    path = build.build(bounds_check=True)
    env = dict(os.environ, WCT_LIB=path)
    code = f"ROOT = {ROOT!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "bounds ok" in r.stdout


def test_release_build_records_nothing():
    import ctypes
    import synth
    import paper_2304_01841_gb300 as g
    lib = g.load(build_if_missing=True)
    sim = g.Simulator([synth.Plane(32, 300)], [synth.make_response("bipolar")], synth.Diffusion())
    rec = (ctypes.c_int64 * 3)()
    assert lib.wct_debug_bounds(sim._h, rec) == 1          # WCT_EINVAL: not a checked build
    sim.close()
