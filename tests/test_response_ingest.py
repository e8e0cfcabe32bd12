"""Field-response ingestion through the C ABI (host computation, no GPU) against the oracle,
and its argument checks."""
import numpy as np
import pytest

import synth
from oracle import response as orr

PITCH, NIMP, TICK, PERIOD = 3.0, 10, 0.5, 0.1


@pytest.fixture(scope="module")
def g():
    import paper_2304_01841_gb300 as pkg
    from paper_2304_01841_gb300 import build
    build.build()
    pkg.load()
    return pkg


@pytest.mark.parametrize("kind,reach", [("unipolar", 10.5), ("bipolar", 10.5), ("bipolar", 4.0)])
def test_library_matches_oracle(g, kind, reach):
    pos, cur = synth.make_field_response(kind, reach_pitches=reach)
    e = synth.electronics_crrc2(PERIOD, 1.0, 200, gain=14.0)
    imp, fold = g.response_from_field(g.FieldResponse(pos, cur, PERIOD), e, PITCH, NIMP, TICK)
    ref_imp, ref_fold = orr.response_from_field(pos, cur, PERIOD, e, PITCH, NIMP, TICK)
    scale = np.abs(ref_imp).max()
    assert np.abs(imp - ref_imp).max() <= 1e-6 * scale
    assert np.abs(fold - ref_fold).max() <= 1e-6 * scale


def test_library_matches_oracle_on_an_irregular_two_sided_field(g):
    rng = np.random.default_rng(7)
    pos = np.sort(rng.uniform(-20.0, 20.0, size=40))
    cur = rng.normal(size=(40, 300))
    e = rng.normal(size=57)
    imp, fold = g.response_from_field(g.FieldResponse(pos, cur, 0.125), e, 2.5, 7, 0.5, n_wires_resp=13,
                                      n_ticks_resp=90)
    ref_imp, ref_fold = orr.response_from_field(pos, cur, 0.125, e, 2.5, 7, 0.5, n_wires=13, n_ticks=90)
    scale = np.abs(ref_imp).max()
    assert np.abs(imp - ref_imp).max() <= 1e-6 * scale
    assert np.abs(fold - ref_fold).max() <= 1e-6 * scale


def test_json_round_trip(g, tmp_path):
    pos, cur = synth.make_field_response("bipolar", reach_pitches=2.0)
    f = g.FieldResponse(pos, cur, PERIOD)
    path = str(tmp_path / "field.json")
    g.save_field_response(path, f)
    back = g.load_field_response(path)
    assert back.period_us == PERIOD
    assert np.array_equal(back.path_pos_mm, pos) and np.array_equal(back.current, cur)


def test_argument_errors(g):
    pos, cur = synth.make_field_response("unipolar", reach_pitches=2.0)
    e = synth.electronics_crrc2()
    ok = g.FieldResponse(pos, cur, PERIOD)
    g.response_from_field(ok, e, PITCH, NIMP, TICK)
    bad = [
        (g.FieldResponse(pos[::-1].copy(), cur, PERIOD), e, PITCH, NIMP, TICK, 21),      # positions decreasing
        (g.FieldResponse(pos, cur, 0.15), e, PITCH, NIMP, TICK, 21),                     # tick not whole periods
        (ok, e, PITCH, NIMP, TICK, 20),                                                  # even wire extent
        (ok, e, -PITCH, NIMP, TICK, 21),                                                 # negative pitch
        (g.FieldResponse(pos[:1], cur[:1], PERIOD), e, PITCH, NIMP, TICK, 21),           # one path
    ]
    for f, el, pitch, nimp, tick, nw in bad:
        with pytest.raises(g.WctError):
            g.response_from_field(f, el, pitch, nimp, tick, n_wires_resp=nw)
    nan = cur.copy()
    nan[3, 5] = np.nan
    with pytest.raises(g.WctError):
        g.response_from_field(g.FieldResponse(pos, nan, PERIOD), e, PITCH, NIMP, TICK)
