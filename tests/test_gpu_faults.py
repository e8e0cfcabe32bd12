"""Host-side fault injection on the GPU path: every device allocation the library makes can be
made to fail (wct_debug_fail_alloc); each call that hits it returns WCT_ENOMEM, frees what it
had taken, and the handle keeps working.  No kernel is made to fault."""
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


@pytest.fixture()
def arm():
    import paper_2304_01841_gb300 as g
    lib = g.load()
    yield lambda n: lib.wct_debug_fail_alloc(n)
    lib.wct_debug_fail_alloc(-1)


def _free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def _dev(d):
    import paper_2304_01841_gb300 as g
    return g.DeviceDepos.from_host(d)


@pytest.mark.parametrize("deterministic", [False, True])
def test_create_fails_cleanly_at_every_allocation(arm, deterministic):
    import paper_2304_01841_gb300 as g
    wl = synth.workload("three_plane")
    base = _free_bytes()
    failures = 0
    for k in range(200):
        arm(k)
        try:
            sim = make_sim(wl.planes, wl.responses(), wl.diffusion, deterministic=deterministic)
        except g.WctError as e:
            assert "WCT_ENOMEM" in str(e)
            failures += 1
            assert abs(_free_bytes() - base) <= (64 << 20), k      # everything taken was freed
            continue
        arm(-1)
        break
    assert failures >= 5                  # create makes several allocations, each one tested
    d = wl.depos(n_depos=5000)
    wfs = sim.run_event(_dev(d))
    sim.sync()
    _, _, ref = oracle.simulate_plane(d, wl.planes[2], wl.diffusion, wl.responses()[2], plane_index=2)
    assert rel_l2(to_np(wfs[2]), ref) <= WAVE_RTOL
    sim.close()
    del wfs
    torch.cuda.empty_cache()                  # the test's own tensors, held by torch's cache
    assert abs(_free_bytes() - base) <= (64 << 20)


def test_failed_calls_leave_the_handle_usable(arm):
    import paper_2304_01841_gb300 as g
    wl = synth.workload("tiny")
    pl = wl.planes[0]
    sim = make_sim([pl], [synth.make_response(pl.response_kind)], wl.diffusion)
    d = wl.depos()
    folded = to_np(sim.run_event(_dev(d))[0])
    sim.sync()
    # impact responses: the allocation of the phase grids fails, the plane stays folded
    arm(1)
    with pytest.raises(g.WctError, match="WCT_ENOMEM"):
        sim.set_impact_responses(0, synth.make_response_impact(pl.response_kind, n_impact=pl.n_impact_per_pitch))
    arm(-1)
    again = to_np(sim.run_event(_dev(d))[0])
    sim.sync()
    assert np.abs(again - folded).max() <= 1e-5 * np.abs(folded).max()
    # a larger event: the depo scratch grows, and that allocation fails
    big = wl.depos(n_depos=4 * d.n, seed=9)
    arm(0)
    with pytest.raises(g.WctError, match="WCT_ENOMEM"):
        sim.run_event(_dev(big))
    arm(-1)
    wf = to_np(sim.run_event(_dev(big))[0])
    sim.sync()
    _, _, ref = oracle.simulate_plane(big, pl, wl.diffusion, synth.make_response(pl.response_kind))
    assert rel_l2(wf, ref) <= WAVE_RTOL
    # host-to-host: the first call's staging buffers fail
    arm(0)
    with pytest.raises(g.WctError, match="WCT_ENOMEM"):
        sim.run_host([d])
    arm(-1)
    host = sim.run_host([d])[0][0].numpy()
    sim.sync()
    assert np.abs(host - folded).max() <= 1e-5 * np.abs(folded).max()
    sim.close()
