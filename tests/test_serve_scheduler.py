"""CPU tests of the serving scheduler (admission, HBM budget, continuous batching, FIFO), driven
with a fake device backend whose batches finish after a set number of scheduler passes."""
import numpy as np

import synth
from paper_2304_01841_gb300.serve import EventServer


class FakeBackend:
    log = []

    def __init__(self, passes=2):
        self.passes = passes
        self.left = 0
        self.batch = None

    def launch(self, batch):
        self.batch = [r.rid for r in batch]
        self.left = self.passes
        FakeBackend.log.append(("launch", id(self), tuple(self.batch)))

    def done(self):
        self.left -= 1
        return self.left <= 0

    def retire(self, batch):
        FakeBackend.log.append(("retire", id(self), tuple(r.rid for r in batch)))

    def close(self):
        pass


def _depos(n):
    return synth.Depos(np.zeros(n), np.ones(n), np.zeros(n), np.zeros(n), np.ones(n))


PLANES = [synth.Plane(10, 100)]          # 4 kB of waveform per request
ONE = 4 * 10 * 100


def _server(passes=2, **kw):
    FakeBackend.log = []
    return EventServer(PLANES, None, None, backend_factory=lambda: FakeBackend(passes), **kw)


def test_fifo_and_batching_limits():
    srv = _server(n_slots=2, max_batch=3, hbm_budget_bytes=1 << 30)
    reqs = [srv.submit(_depos(10)) for _ in range(8)]
    srv.drain()
    launches = [b for kind, _, b in FakeBackend.log if kind == "launch"]
    assert all(len(b) <= 3 for b in launches)
    assert [rid for b in launches for rid in b] == list(range(8))          # FIFO, each once
    assert sorted(r.rid for r in srv.completed) == list(range(8))
    assert all(r.done.is_set() for r in reqs)


def test_budget_limits_memory_in_flight():
    need = 20 * 100 + ONE
    srv = _server(n_slots=4, max_batch=4, hbm_budget_bytes=3 * need)
    for _ in range(12):
        srv.submit(_depos(100))
    peak = 0
    while srv.step() > 0:
        peak = max(peak, srv.in_use)
    assert peak <= 3 * need
    assert len(srv.completed) == 12


def test_oversized_request_runs_alone_when_idle():
    srv = _server(n_slots=2, max_batch=4, hbm_budget_bytes=1000)   # every request is over budget
    for _ in range(3):
        srv.submit(_depos(50))
    srv.drain()
    launches = [b for kind, _, b in FakeBackend.log if kind == "launch"]
    assert launches == [(0,), (1,), (2,)]


def test_requests_arriving_later_join_as_slots_free():
    srv = _server(n_slots=1, max_batch=8, hbm_budget_bytes=1 << 30, passes=3)
    srv.submit(_depos(10))
    srv.step()                                  # request 0 launched
    for _ in range(3):
        srv.submit(_depos(10))                  # arrive while the slot is busy
    srv.drain()
    launches = [b for kind, _, b in FakeBackend.log if kind == "launch"]
    assert launches[0] == (0,) and launches[1] == (1, 2, 3)


class FailingBackend(FakeBackend):
    """Raises on the launch (or the retire) of any batch holding a request id in `bad`."""

    def __init__(self, bad, where, passes=2):
        super().__init__(passes)
        self.bad, self.where = set(bad), where

    def launch(self, batch):
        super().launch(batch)
        if self.where == "launch" and self.bad & {r.rid for r in batch}:
            raise RuntimeError("injected launch failure")

    def retire(self, batch):
        super().retire(batch)
        if self.where == "retire" and self.bad & {r.rid for r in batch}:
            raise RuntimeError("injected device error at sync")


def test_cancel_pending_and_in_flight():
    srv = _server(passes=3, n_slots=1, max_batch=1, hbm_budget_bytes=1 << 30)
    reqs = [srv.submit(_depos(10)) for _ in range(4)]
    srv.step()                                       # request 0 on the device
    assert srv.cancel(reqs[2]) is True               # pending: never launched
    assert reqs[2].done.is_set() and reqs[2].cancelled
    assert srv.cancel(reqs[0]) is False              # in flight: finishes, results dropped
    srv.drain()
    launched = [rid for kind, _, b in FakeBackend.log if kind == "launch" for rid in b]
    assert launched == [0, 1, 3]
    assert all(r.done.is_set() for r in reqs)
    assert reqs[0].cancelled and reqs[0].waveforms is None and reqs[0].error is None
    assert not reqs[1].cancelled and not reqs[3].cancelled
    assert srv.in_use == 0


def test_failed_batches_complete_with_their_error_and_the_server_carries_on():
    for where in ("launch", "retire"):
        FakeBackend.log = []
        srv = EventServer(PLANES, None, None, n_slots=2, max_batch=2, hbm_budget_bytes=1 << 30,
                          backend_factory=lambda: FailingBackend({3}, where))
        reqs = [srv.submit(_depos(10)) for _ in range(8)]
        srv.drain()
        assert all(r.done.is_set() for r in reqs)
        failed = [r.rid for r in reqs if r.error is not None]
        batch_of_3 = next(b for kind, _, b in FakeBackend.log if kind == "launch" and 3 in b)
        assert sorted(failed) == sorted(batch_of_3), where      # only the failing batch
        assert all("injected" in str(reqs[i].error) for i in failed)
        assert sorted(r.rid for r in srv.completed) == list(range(8))
        assert srv.in_use == 0


def test_small_requests_never_wait_behind_a_heavy_one():
    # a 1M-depo request at the head of the queue runs alone on the heavy slot; the small
    # requests behind it are batched on the other slots without waiting for it
    srv = _server(passes=6, n_slots=3, max_batch=8, hbm_budget_bytes=1 << 40)
    big = srv.submit(_depos(1_000_000))
    small = [srv.submit(_depos(2000)) for _ in range(5)]
    srv.step()
    launches = [b for kind, _, b in FakeBackend.log if kind == "launch"]
    assert (big.rid,) in launches                                   # alone
    assert any(set(b) == {r.rid for r in small} for b in launches)  # all small ones, same pass
    assert all(r.t_admit > 0 for r in small)                        # admitted while the big one runs
    srv.drain()
    assert all(r.done.is_set() for r in [big] + small)


def test_light_batches_are_capped_in_depos_and_heavy_ones_queue_in_order():
    srv = _server(passes=2, n_slots=2, max_batch=8, hbm_budget_bytes=1 << 40, max_batch_depos=10_000,
                  heavy_depos=500_000)
    heavy = [srv.submit(_depos(600_000)) for _ in range(2)]
    light = [srv.submit(_depos(4000)) for _ in range(5)]
    srv.drain()
    launches = [b for kind, _, b in FakeBackend.log if kind == "launch"]
    light_ids = {r.rid for r in light}
    for b in launches:
        if set(b) & light_ids:
            assert set(b) <= light_ids and 4000 * len(b) <= 10_000       # depo cap, never mixed
    heavy_order = [b[0] for b in launches if b[0] in {r.rid for r in heavy}]
    assert heavy_order == [r.rid for r in heavy] and all(len(b) == 1 for b in launches if b[0] in heavy_order)


def test_single_slot_still_runs_heavy_requests_alone():
    srv = _server(passes=2, n_slots=1, max_batch=8, hbm_budget_bytes=1 << 40)
    a = srv.submit(_depos(10))
    h = srv.submit(_depos(2_000_000))
    b = srv.submit(_depos(10))
    srv.drain()
    launches = [b_ for kind, _, b_ in FakeBackend.log if kind == "launch"]
    assert (h.rid,) in launches and all(len(x) == 1 or h.rid not in x for x in launches)
    assert sorted(r.rid for r in srv.completed) == [a.rid, h.rid, b.rid]
