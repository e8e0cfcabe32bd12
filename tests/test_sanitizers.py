"""The oracle's C code and the library's host-side field-response ingestion built with
AddressSanitizer + UndefinedBehaviorSanitizer and exercised on normal and edge-case inputs
(CPU only; a sanitizer report fails the test)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g", "-O1"]

SCRIPT = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle, synth
wl = synth.workload("tiny")
pl = wl.planes[0]
d = wl.depos()
for fluct in (False, True):
    diff = synth.Diffusion(fluctuate=fluct, seed=3)
    pt = oracle.rasterize(d, pl, diff)
    g = oracle.scatter(pt, pl)
    assert g.sum() > 0
# edge cases: point charges (x = 0), depos off the grid, invalid values, an empty event
n = 64
rng = np.random.default_rng(1)
x = rng.uniform(0, 1600, n).astype(np.float32); x[:8] = 0.0
y = np.zeros(n, np.float32)
z = rng.uniform(-600, 600, n).astype(np.float32); z[8:16] = 1e5
q = rng.uniform(100, 1e4, n).astype(np.float32); q[16] = np.nan; q[17] = -1.0
e = synth.Depos(np.zeros(n, np.float32), x, y, z, q)
oracle.scatter(oracle.rasterize(e, pl, synth.Diffusion(fluctuate=True, seed=5)), pl)
empty = synth.Depos(*(np.zeros(0, np.float32) for _ in range(5)))
oracle.scatter(oracle.rasterize(empty, pl, wl.diffusion), pl)
oracle.convolve_direct(rng.normal(size=(9, 40)), rng.normal(size=(5, 11)))
oracle.philox4x32_10(rng.integers(0, 2**32, size=(100, 4), dtype=np.uint64).astype(np.uint32), (7, 9))
for mu, s in ((0.5, 0.0), (3.25, 1e-9), (10.0, 2.0), (-3.0, 0.7)):
    oracle.axis_weights(mu, s)
# host-side ingestion of the library, sanitized build
L = ctypes.CDLL(RESP)
class FR(ctypes.Structure):
    _fields_ = [("n_paths", ctypes.c_int32), ("n_samples", ctypes.c_int32), ("period_us", ctypes.c_double),
                ("path_pos_mm", ctypes.c_void_p), ("current", ctypes.c_void_p)]
P, I, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
L.wct_response_from_field.argtypes = [ctypes.POINTER(FR), P, I, D, I, D, I, I, P, P]
L.wct_response_from_field.restype = ctypes.c_int
pos, cur = synth.make_field_response("bipolar", reach_pitches=3.0)
el = synth.electronics_crrc2()
imp = np.empty((10, 21, 200), np.float32); fold = np.empty((21, 200), np.float32)
def call(pos, cur, el, pitch=3.0, nimp=10, tick=0.5, nw=21, nt=200, period=0.1, out=True):
    f = FR(len(pos), cur.shape[1], period, pos.ctypes.data, cur.ctypes.data)
    return L.wct_response_from_field(ctypes.byref(f), el.ctypes.data, len(el), pitch, nimp, tick, nw, nt,
                                     imp.ctypes.data if out else None, fold.ctypes.data if out else None)
assert call(pos, cur, el) == 0
assert call(pos, cur, el, out=False) == 0
assert call(pos, cur, el[:1]) == 0                          # one-sample electronics
assert call(pos[::-1].copy(), cur, el) == 1                 # decreasing positions
assert call(pos, cur, el, period=0.15) == 1                 # tick not a whole number of periods
assert call(pos, cur, el, nw=20) == 1
assert call(pos[:2].copy(), cur[:2].copy(), el) == 0        # two paths
bad = cur.copy(); bad[1, 1] = np.inf
assert call(pos, bad, el) == 1
print("sanitized run ok")
"""


def _build(tmp_path):
    so = str(tmp_path / "liboracle_san.so")
    subprocess.check_call(["gcc", *SAN, "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", so,
                           os.path.join(ROOT, "oracle", "wct_oracle.c"), "-lm"])
    resp = str(tmp_path / "libresp_san.so")
    subprocess.check_call(["g++", *SAN, "-x", "c++", "-std=c++17", "-fPIC", "-shared", "-I",
                           os.path.join(ROOT, "include"), "-o", resp,
                           os.path.join(ROOT, "paper_2304_01841_gb300", "csrc", "wct_response.cu")])
    return so, resp


def test_oracle_and_ingestion_under_asan_ubsan(tmp_path):
    asan = subprocess.check_output(["gcc", "-print-file-name=libasan.so"], text=True).strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no AddressSanitizer runtime")
    so, resp = _build(tmp_path)
    env = dict(os.environ, LD_PRELOAD=asan, WCT_ORACLE_LIB=so, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    code = f"ROOT = {ROOT!r}\nRESP = {resp!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "sanitized run ok" in out
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
