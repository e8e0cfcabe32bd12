"""Host-side checks of the C ABI (CPU only): the library builds, loads and exports every
declared entry point; the ctypes structures match the C layout; argument errors are
returned before any CUDA work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wct_sim.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2304_01841_gb300 import _abi, build
    build.build()
    return _abi.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wct_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2304_01841_gb300 import _abi
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_abi.EXPORTS), set(names) - set(_abi.EXPORTS)


def test_struct_layout_matches_header(tmp_path):
    from paper_2304_01841_gb300 import _abi
    c = tmp_path / "layout.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "wct_sim.h"\n'
                 "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(wct_plane_t),"
                 " sizeof(wct_response_t), sizeof(wct_diffusion_t), sizeof(wct_opts_t), sizeof(wct_depos_t),"
                 " offsetof(wct_diffusion_t, seed), offsetof(wct_depos_t, event_id),"
                 " sizeof(wct_field_response_t), offsetof(wct_field_response_t, current)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(_abi.wct_plane_t), ctypes.sizeof(_abi.wct_response_t),
            ctypes.sizeof(_abi.wct_diffusion_t), ctypes.sizeof(_abi.wct_opts_t), ctypes.sizeof(_abi.wct_depos_t),
            _abi.wct_diffusion_t.seed.offset, _abi.wct_depos_t.event_id.offset,
            ctypes.sizeof(_abi.wct_field_response_t), _abi.wct_field_response_t.current.offset]
    assert got == want


def test_header_constants_match_binding():
    from paper_2304_01841_gb300 import _abi
    src = open(HEADER).read()
    for name in ("WCT_MAX_WINDOW_TICKS", "WCT_MAX_WINDOW_IMPACTS", "WCT_MAX_RESPONSE_WIRES"):
        m = re.search(r"#define\s+%s\s+(\d+)" % name, src)
        assert m and int(m.group(1)) == getattr(_abi, name)


def test_oracle_limits_match_library():
    import oracle
    from paper_2304_01841_gb300 import _abi
    assert oracle.MAX_NT == _abi.WCT_MAX_WINDOW_TICKS
    assert oracle.MAX_NP == _abi.WCT_MAX_WINDOW_IMPACTS


def test_argument_errors_return_before_cuda_work(lib):
    from paper_2304_01841_gb300 import _abi
    import numpy as np
    resp = np.zeros((21, 200), dtype=np.float32)
    P = (_abi.wct_plane_t * 1)(_abi.wct_plane_t(256, 10, 1024, 3.0, -384.0, 0.0, 0.5, 0.0))
    R = (_abi.wct_response_t * 1)(_abi.wct_response_t(21, 200, resp.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    D = _abi.wct_diffusion_t(4.0, 8.8, 1.6, 3.0, 0, 1)
    h = ctypes.c_void_p()
    E = _abi.WCT_EINVAL
    assert lib.wct_sim_create(P, 0, R, ctypes.byref(D), None, ctypes.byref(h)) == E
    assert lib.wct_sim_create(P, 1, R, ctypes.byref(D), None, None) == E
    bad = _abi.wct_diffusion_t(4.0, 8.8, 0.0, 3.0, 0, 1)               # zero drift speed
    assert lib.wct_sim_create(P, 1, R, ctypes.byref(bad), None, ctypes.byref(h)) == E
    R2 = (_abi.wct_response_t * 1)(_abi.wct_response_t(20, 200, resp.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    assert lib.wct_sim_create(P, 1, R2, ctypes.byref(D), None, ctypes.byref(h)) == E   # even wire count
    R3 = (_abi.wct_response_t * 1)(_abi.wct_response_t(23, 200, resp.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    assert lib.wct_sim_create(P, 1, R3, ctypes.byref(D), None, ctypes.byref(h)) == E   # wider than 21
    P2 = (_abi.wct_plane_t * 1)(_abi.wct_plane_t(256, 10, 1024, -3.0, -384.0, 0.0, 0.5, 0.0))
    assert lib.wct_sim_create(P2, 1, R, ctypes.byref(D), None, ctypes.byref(h)) == E   # negative pitch
    assert h.value is None
    assert lib.wct_sim_sync(None, None) == E
    assert lib.wct_sim_destroy(None) == E
    assert lib.wct_philox4x32_10(None, 0, -1, None, None) == E


def test_debug_entry_points_without_a_gpu(lib):
    import ctypes
    assert lib.wct_debug_fail_alloc(3) == 0          # arms without device work
    assert lib.wct_debug_fail_alloc(-1) == 0         # disarms
    rec = (ctypes.c_int64 * 3)()
    assert lib.wct_debug_bounds(None, rec) == 1      # WCT_EINVAL: no handle
