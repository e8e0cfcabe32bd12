"""GPU parity of the noise + digitisation step against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import make_sim, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_01841_gb300 as g
    g.load(build_if_missing=True)


def _sim(nw, nt, seed=5):
    return make_sim([synth.Plane(nw, nt)], [synth.make_response("bipolar")], synth.Diffusion(seed=seed))


@pytest.mark.parametrize("nw,nt", [(64, 1024), (37, 1001)])
def test_noise_free_codes_bit_exact(nw, nt):
    rng = np.random.default_rng(nw)
    v = (rng.normal(size=(nw, nt)) * 300.0).astype(np.float32)
    v[0, :8] = [0.5, 1.5, -0.5, 2.5, 1e9, -1e9, np.nan, 0.49999997]     # ties, clamps, NaN
    sim = _sim(nw, nt)
    got = to_np(sim.digitize(0, torch.from_numpy(v).cuda(), 1.7, 2048.0, 0.0, bits=12, add_noise=False))
    sim.sync()
    want, _ = oracle.digitize(v, 1.7, 2048.0, 0.0, 12, False, seed=5, plane_index=0, event_id=0)
    assert np.array_equal(got, want)


def test_noisy_codes_agree_except_at_rounding_ties():
    nw, nt = 512, 9600
    rng = np.random.default_rng(3)
    v = (rng.normal(size=(nw, nt)) * 50.0).astype(np.float32)
    sim = _sim(nw, nt, seed=77)
    got = to_np(sim.digitize(0, torch.from_numpy(v).cuda(), 1.0, 900.0, 2.5, bits=12, add_noise=True, event_id=12))
    sim.sync()
    want, s = oracle.digitize(v, 1.0, 900.0, 2.5, 12, True, seed=77, plane_index=0, event_id=12)
    diff = got.astype(np.int32) - want.astype(np.int32)
    bad = diff != 0
    # the device's normals differ from the FP64 ones by < 1e-5, so a code may differ only when
    # the value sits within 2.5 * 1e-5 of a rounding boundary, and then by one
    dist = np.abs((s - np.floor(s)) - 0.5)
    assert np.all(np.abs(diff) <= 1)
    assert np.all(dist[bad] < 1e-4)
    assert bad.mean() < 1e-3


def test_event_waveform_digitizes_in_range():
    wl = synth.workload("tiny")
    sim = make_sim(wl.planes, wl.responses(), wl.diffusion)
    import paper_2304_01841_gb300 as g
    wf = sim.run_event(g.DeviceDepos.from_host(wl.depos()))[0]
    codes = to_np(sim.digitize(0, wf, 0.05, 500.0, 1.5, bits=12, event_id=1))
    sim.sync()
    assert codes.dtype == np.int16 and codes.min() >= 0 and codes.max() <= 4095
    assert abs(float(np.median(codes)) - 500.0) <= 2


def test_coloured_noise_codes_match_oracle():
    # a per-plane noise spectrum: the device's noise (spectrum from Philox, inverse row
    # transform) against the FP64 oracle, through the codes of a flat waveform with unit gain:
    # codes may differ only where the value sits within 1e-3 of a rounding boundary
    nw, nt = 300, 9600
    pl = synth.Plane(nw, nt)
    sim = make_sim([pl], [synth.make_response("bipolar")], synth.Diffusion(seed=41))
    info = sim.plane_info(0)
    F, P = info["spectrum_bins"], info["fft_length"]
    f = np.arange(F)
    amp = (1.0 / (1.0 + (f / 300.0) ** 2)).astype(np.float32)          # low-pass shape
    sim.set_noise_spectrum(0, amp)
    rms = 2000.0                                                       # noise std ~ 6 counts
    v = np.random.default_rng(8).normal(size=(nw, nt)).astype(np.float32) * 20.0
    got = to_np(sim.digitize(0, torch.from_numpy(v).cuda(), 1.0, 1500.0, rms, bits=12, event_id=77))
    sim.sync()
    noise = oracle.coloured_noise(41, nw, nt, P, amp, rms, 0, 77)
    assert noise.std() > 3.0                                           # the noise is there
    want, s = oracle.digitize(v, 1.0, 1500.0, rms, 12, True, 41, 0, 77, noise_wave=noise)
    diff = got.astype(np.int32) - want.astype(np.int32)
    bad = diff != 0
    dist = np.abs((s - np.floor(s)) - 0.5)
    assert np.all(np.abs(diff) <= 1) and np.all(dist[bad] < 1e-3) and bad.mean() < 1e-3
    # back to white noise
    sim.set_noise_spectrum(0, None)
    w = to_np(sim.digitize(0, torch.from_numpy(v).cuda(), 1.0, 1500.0, 2.0, bits=12, event_id=77))
    sim.sync()
    ww, _ = oracle.digitize(v, 1.0, 1500.0, 2.0, 12, True, 41, 0, 77)
    assert (w != ww).mean() < 1e-3
