"""Pins of the oracle's field-response ingestion (the detector response of §2 step 3 built from
a field response and an electronics response)."""
import numpy as np
import pytest

import synth
from oracle import response as orr

PITCH, NIMP, TICK, PERIOD = 3.0, 10, 0.5, 0.1
M = 5   # fine samples per tick


def _positions(reach_pitches=10.5):
    return np.arange(0.0, reach_pitches * PITCH + 1e-9, 0.3)


def _x(p, r, n_wires=21, n_imp=NIMP):
    return ((p + 0.5) / n_imp - 0.5) * PITCH - (r - n_wires // 2) * PITCH


def test_constant_field_with_delta_electronics_is_the_sampled_current():
    rng = np.random.default_rng(1)
    pos = _positions()
    f = rng.normal(size=1000)
    cur = np.repeat(f[None], pos.shape[0], axis=0)
    delta = np.array([1.0 / PERIOD])                    # unit-area impulse
    imp, fold = orr.response_from_field(pos, cur, PERIOD, delta, PITCH, NIMP, TICK)
    want = f[np.arange(200) * M]
    assert np.abs(imp - want).max() <= 1e-12
    assert np.abs(fold - want).max() <= 1e-12


def test_field_linear_in_position_is_interpolated_exactly_and_mirrored():
    rng = np.random.default_rng(2)
    pos = _positions()
    f = rng.normal(size=1000)
    a, b = 0.7, -0.02
    cur = (a + b * pos)[:, None] * f[None]
    imp, _ = orr.response_from_field(pos, cur, PERIOD, np.array([1.0 / PERIOD]), PITCH, NIMP, TICK)
    for p in (0, 3, 9):
        for r in (0, 7, 10, 11, 20):
            want = (a + b * abs(_x(p, r))) * f[np.arange(200) * M]
            assert np.abs(imp[p, r] - want).max() <= 1e-12, (p, r)


def test_mirror_symmetry_of_phases_and_offsets():
    pos, cur = synth.make_field_response("bipolar")
    e = synth.electronics_crrc2()
    imp, _ = orr.response_from_field(pos, cur, PERIOD, e, PITCH, NIMP, TICK)
    # phase p at offset d sees x; phase n-1-p at offset -d sees -x
    assert np.abs(imp - imp[::-1, ::-1]).max() <= 1e-12 * np.abs(imp).max()
    # near the wire the phases differ, so the impact mode has something to resolve
    assert np.abs(imp[0, 10] - imp[4, 10]).max() > 1e-2 * np.abs(imp[:, 10]).max()


def test_two_sided_field_matches_the_mirrored_one_sided_field():
    pos, cur = synth.make_field_response("unipolar", reach_pitches=6.0)
    both = np.concatenate([-pos[:0:-1], pos])
    cur2 = np.concatenate([cur[:0:-1], cur])
    e = synth.electronics_crrc2()
    one, _ = orr.response_from_field(pos, cur, PERIOD, e, PITCH, NIMP, TICK)
    two, _ = orr.response_from_field(both, cur2, PERIOD, e, PITCH, NIMP, TICK)
    assert np.abs(one - two).max() <= 1e-12 * np.abs(one).max()


def test_rows_beyond_the_fields_reach_are_zero():
    pos, cur = synth.make_field_response("unipolar", reach_pitches=5.0)
    imp, _ = orr.response_from_field(pos, cur, PERIOD, synth.electronics_crrc2(), PITCH, NIMP, TICK)
    for p in range(NIMP):
        for r in range(21):
            inside = abs(_x(p, r)) <= 5.0 * PITCH + 1e-9
            assert (np.abs(imp[p, r]).max() > 0) == inside, (p, r)


def test_impulse_current_places_the_electronics_response():
    # I = unit-area impulse at fine sample s0 on every path: R[tau] = E[tau m - s0]
    rng = np.random.default_rng(3)
    pos = _positions()
    s0 = 37
    cur = np.zeros((pos.shape[0], 400))
    cur[:, s0] = 1.0 / PERIOD
    e = rng.normal(size=300)
    imp, _ = orr.response_from_field(pos, cur, PERIOD, e, PITCH, NIMP, TICK, n_ticks=100)
    want = np.zeros(100)
    for t in range(100):
        k = t * M - s0
        if 0 <= k < e.shape[0]:
            want[t] = e[k]
    assert np.abs(imp[2, 13] - want).max() <= 1e-12


def test_vectorised_form_equals_literal_loops():
    rng = np.random.default_rng(4)
    pos = np.array([0.0, 0.4, 1.1, 2.0, 3.5, 4.1])
    cur = rng.normal(size=(6, 23))
    e = rng.normal(size=9)
    got, fold = orr.response_from_field(pos, cur, 0.25, e, 1.5, 3, 0.75, n_wires=5, n_ticks=12)
    want = orr.response_from_field_loops(pos, cur, 0.25, e, 1.5, 3, 0.75, 5, 12)
    assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
    assert np.abs(fold - want.mean(axis=0)).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_tick_must_be_a_whole_number_of_periods():
    pos, cur = synth.make_field_response("unipolar")
    with pytest.raises(ValueError):
        orr.response_from_field(pos, cur, 0.15, synth.electronics_crrc2(0.15), PITCH, NIMP, TICK)
