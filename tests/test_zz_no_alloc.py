"""The allocation-free convolution entry point, wct_convolve_static, against the FP64 oracle
and against wct_sim_convolve.

wct_convolve_static is for callers that may not allocate device memory when they call the
library (a host framework that owns all device memory through its own pool, or a path that
cannot afford cudaMalloc's implicit synchronisation).  It works from a fixed scratch array
the library reserves when it is loaded, so this test checks that two calls in a row, which
share and reuse that array, each give the oracle's convolution (and the handle-based one's),
that a timed-out device wait is reported through wct_convolve_static_status, and that sizes
beyond the reserved scratch are refused before any launch.

This file is collected last on purpose: it must pass after the other tests and on its own.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import WAVE_RTOL, make_sim, rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_01841_gb300 as g
    return g.load(build_if_missing=True)


def _static_convolve(lib, grid, resp_dev, out):
    nw, nt = grid.shape
    kw, kt = resp_dev.shape
    stream = torch.cuda.current_stream().cuda_stream
    return lib.wct_convolve_static(grid.data_ptr(), nw, nt, resp_dev.data_ptr(), kw, kt, out.data_ptr(), stream)


def test_static_convolve_matches_handle_twice_in_a_row(lib):
    pl = synth.Plane(256, 1024)
    resp = synth.make_response("bipolar")
    sim = make_sim([pl], [resp], synth.Diffusion())
    resp_dev = torch.from_numpy(resp).cuda()
    rng = np.random.default_rng(2024)
    for call in range(2):
        g = torch.from_numpy(rng.normal(size=(256, 1024)).astype(np.float32)).cuda()
        want = sim.convolve(0, g)
        got = torch.full_like(g, float("nan"))
        assert _static_convolve(lib, g, resp_dev, got) == 0
        assert lib.wct_convolve_static_status(torch.cuda.current_stream().cuda_stream) == 0
        sim.sync()
        ref = oracle.convolve_fft(to_np(g).astype(np.float64), resp)
        assert rel_l2(to_np(got), ref) <= WAVE_RTOL, call
        assert rel_l2(to_np(got), to_np(want)) <= WAVE_RTOL, call


def test_static_convolve_narrow_response_in_place(lib):
    # a 5-wire response (padded to the 21-row stage inside) and grid == waveform
    pl = synth.Plane(64, 500)
    resp = np.random.default_rng(7).normal(size=(5, 37)).astype(np.float32)
    sim = make_sim([pl], [resp], synth.Diffusion())
    g = torch.from_numpy(np.random.default_rng(8).normal(size=(64, 500)).astype(np.float32)).cuda()
    want = sim.convolve(0, g)
    buf = g.clone()
    assert _static_convolve(lib, buf, torch.from_numpy(resp).cuda(), buf) == 0
    assert lib.wct_convolve_static_status(torch.cuda.current_stream().cuda_stream) == 0
    ref = oracle.convolve_fft(to_np(g).astype(np.float64), resp)
    assert rel_l2(to_np(buf), ref) <= WAVE_RTOL
    assert rel_l2(to_np(buf), to_np(want)) <= WAVE_RTOL


def test_static_convolve_reports_a_timed_out_wait(lib):
    # a bounded wait that can never complete (nothing arrives on its barrier) gives up after a
    # short limit and records WCT_ETIMEOUT in the fixed array's status word, as the convolution's
    # copy-fed kernels do when a bulk copy never lands; the status call reports it once, the
    # context stays usable and the next convolution is exact again
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.wct_convolve_static_status(stream) == 0
    assert lib.wct_convolve_static_selftest_wait(200_000, stream) == 0
    assert lib.wct_convolve_static_status(stream) == 4           # WCT_ETIMEOUT
    assert lib.wct_convolve_static_status(stream) == 0           # read and cleared
    resp = synth.make_response("unipolar")
    g = torch.from_numpy(np.random.default_rng(11).normal(size=(48, 700)).astype(np.float32)).cuda()
    out = torch.empty_like(g)
    assert _static_convolve(lib, g, torch.from_numpy(resp).cuda(), out) == 0
    assert lib.wct_convolve_static_status(stream) == 0
    assert rel_l2(to_np(out), oracle.convolve_fft(to_np(g).astype(np.float64), resp)) <= WAVE_RTOL
    assert lib.wct_convolve_static_selftest_wait(-1, stream) == 1


def test_static_convolve_rejects_sizes_beyond_its_scratch(lib):
    resp_dev = torch.zeros((21, 200), dtype=torch.float32, device="cuda")
    tiny = torch.zeros((1, 8), dtype=torch.float32, device="cuda")
    # 3456 x 9600 needs ~272 MB of spectra: far beyond the reserved scratch; refused on the host
    rc = lib.wct_convolve_static(tiny.data_ptr(), 3456, 9600, resp_dev.data_ptr(), 21, 200, tiny.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert lib.wct_convolve_static(None, 4, 4, resp_dev.data_ptr(), 21, 200, tiny.data_ptr(), None) == 1
    assert lib.wct_convolve_static(tiny.data_ptr(), 1, 8, resp_dev.data_ptr(), 20, 200, tiny.data_ptr(), None) == 1
