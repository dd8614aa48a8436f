"""Host-side scheduling of the continuous-batching server, with a fake engine
(no GPU): memory admission, FCFS order, overlap of requests that arrive
while others run, exact step counts, error isolation, latency statistics."""
import itertools

import numpy as np
import pytest

from paper_2205_00686_gb300.serve import Server


@pytest.fixture(autouse=True, params=[1, 2], ids=["pipeline1", "pipeline2"])
def _pipeline(request, monkeypatch):
    """Every test runs with one and with two chunks queued ahead."""
    init = Server.__init__

    def with_depth(self, *a, **k):
        k.setdefault("pipeline", request.param)
        init(self, *a, **k)
    monkeypatch.setattr(Server, "__init__", with_depth)


class FakeCase:
    def __init__(self, nx, ny, tag=0):
        self.nx, self.ny, self.tag = nx, ny, tag
        self.params = {}


class FakeBackend:
    """Steps attached handles at once; wait() reports the error words of a
    chunk's members, as the device engine does one chunk later."""

    def __init__(self, fail_tags=(), fail_open_tags=()):
        self.open_handles = {}
        self.log = []
        self.fail_tags = set(fail_tags)
        self.fail_open_tags = set(fail_open_tags)
        self.peak_bytes = 0
        self._live_bytes = 0

    def bytes_for(self, case):
        return case.nx * case.ny * 100

    def open(self, case, steps):
        if case.tag in self.fail_open_tags:
            raise MemoryError("device allocation failed")
        h = {"case": case, "steps": 0, "target": steps, "attached": True}
        self.open_handles[id(h)] = h
        self._live_bytes += self.bytes_for(case)
        self.peak_bytes = max(self.peak_bytes, self._live_bytes)
        self.log.append(("open", case.tag))
        return h

    def step(self, n):
        live = [h for h in self.open_handles.values() if h["attached"]]
        for h in live:
            h["steps"] = min(h["steps"] + n, h["target"])
        self.log.append(("step", n, sorted(h["case"].tag for h in live)))
        return [id(h) for h in live]

    def wait(self, token):
        return {k: -4 for k in token
                if k in self.open_handles and self.open_handles[k]["case"].tag in self.fail_tags}

    def detach(self, h):
        h["attached"] = False

    def close(self, h, read=True):
        del self.open_handles[id(h)]
        self._live_bytes -= self.bytes_for(h["case"])
        self.log.append(("close", h["case"].tag))
        return h["steps"] if read else None


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def test_memory_budget_is_never_exceeded_and_all_finish():
    be = FakeBackend()
    srv = Server(be, mem_budget=3 * 64 * 64 * 100, chunk=10, clock=Clock())
    reqs = [srv.submit(FakeCase(64, 64, i), steps=25 + 5 * i) for i in range(7)]
    while srv.tick():
        pass
    assert be.peak_bytes <= srv.mem_budget
    assert all(r.result == r.steps for r in reqs)      # exactly `steps`, no overshoot
    assert srv.mem_used == 0 and not srv.active


def test_fcfs_admission_and_continuous_batching():
    """A short request that arrives after a long one starts while the long
    one is still running, and finishes first."""
    be = FakeBackend()
    srv = Server(be, mem_budget=2 * 64 * 64 * 100, chunk=5, clock=Clock())
    long_r = srv.submit(FakeCase(64, 64, "long"), steps=100)
    srv.tick()
    short_r = srv.submit(FakeCase(64, 64, "short"), steps=10)
    while srv.tick():
        pass
    opens = [e for e in be.log if e[0] == "open"]
    assert [o[1] for o in opens] == ["long", "short"]
    assert short_r.finished < long_r.finished
    # the two overlapped in at least one batched step
    assert any(e[0] == "step" and e[2] == ["long", "short"] for e in be.log)


def test_a_request_that_does_not_fit_waits_for_memory():
    be = FakeBackend()
    srv = Server(be, mem_budget=64 * 64 * 100 + 10, chunk=7, clock=Clock())
    a = srv.submit(FakeCase(64, 64, "a"), steps=20)
    b = srv.submit(FakeCase(64, 64, "b"), steps=20)
    while srv.tick():
        pass
    assert b.admitted >= a.finished
    with pytest.raises(ValueError):
        srv.submit(FakeCase(128, 128, "huge"), steps=1)


def test_failed_request_is_isolated():
    be = FakeBackend(fail_tags={"bad"})
    srv = Server(be, mem_budget=10 ** 9, chunk=10, clock=Clock())
    good = [srv.submit(FakeCase(32, 32, "g%d" % i), steps=30) for i in range(3)]
    bad = srv.submit(FakeCase(32, 32, "bad"), steps=30)
    while srv.tick():
        pass
    assert bad.error == -4 and bad.result is None
    assert all(r.error == 0 and r.result == 30 for r in good)
    st = srv.stats()
    assert st["requests"] == 4 and st["failed"] == 1


def test_stats_percentiles():
    be = FakeBackend()
    clk = Clock()
    srv = Server(be, mem_budget=10 ** 9, chunk=10, clock=clk)
    for i in range(5):
        srv.submit(FakeCase(16, 16, i), steps=10 * (i + 1), arrival=0.0)
    while srv.tick():
        pass
    st = srv.stats()
    lat = sorted(r.latency for r in srv.finished)
    assert st["p50_s"] == pytest.approx(np.percentile(lat, 50))
    assert st["p99_s"] == pytest.approx(np.percentile(lat, 99))
    assert st["node_updates"] == sum(16 * 16 * 10 * (i + 1) for i in range(5))


def test_timed_arrivals_are_admitted_while_others_run():
    be = FakeBackend()
    ticks = itertools.count()
    srv = Server(be, mem_budget=10 ** 9, chunk=5, clock=lambda: next(ticks) * 0.01)
    arrivals = [(0.0, FakeCase(16, 16, "first"), 200), (0.2, FakeCase(16, 16, "later"), 20)]
    st = srv.run(arrivals)
    assert st["requests"] == 2
    steps = [e for e in be.log if e[0] == "step"]
    assert any(e[2] == ["first", "later"] for e in steps)


def test_failed_admission_fails_only_that_request():
    """A domain whose creation fails (e.g. device memory exhausted) retires
    its own request with ADMIT_FAILED; the budget is not charged and every
    other request runs to completion."""
    from paper_2205_00686_gb300.serve import ADMIT_FAILED
    be = FakeBackend(fail_open_tags={"b"})
    srv = Server(be, mem_budget=2 * 64 * 64 * 100, chunk=10, clock=Clock())
    reqs = {t: srv.submit(FakeCase(64, 64, t), steps=30) for t in "abcd"}
    while srv.tick():
        pass
    assert reqs["b"].error == ADMIT_FAILED and "allocation" in reqs["b"].detail
    assert reqs["b"].result is None
    for t in "acd":
        assert reqs[t].error == 0 and reqs[t].result == 30
    assert srv.mem_used == 0 and be.peak_bytes <= srv.mem_budget
    st = srv.stats()
    assert st["failed"] == 1 and st["requests"] == 4


def test_cancel_waiting_and_running_requests():
    """Cancelling a running request retires it between chunks without a
    read-back and frees its memory for the queue; cancelling a queued one
    removes it; a finished request cannot be cancelled."""
    from paper_2205_00686_gb300.serve import CANCELLED
    be = FakeBackend()
    srv = Server(be, mem_budget=2 * 64 * 64 * 100, chunk=10, clock=Clock())
    a, b, c, d = (srv.submit(FakeCase(64, 64, t), steps=50) for t in "abcd")
    srv.tick()                      # a, b admitted; c, d waiting
    assert set(srv.active) == {a.rid, b.rid}
    assert srv.cancel(b.rid) and b.error == CANCELLED and b.result is None
    assert ("close", "b") in be.log
    assert srv.cancel(d.rid) and d.error == CANCELLED
    while srv.tick():
        pass
    assert a.result == 50 and c.result == 50
    assert not srv.cancel(a.rid) and not srv.cancel(12345)
    assert ("open", "d") not in be.log
    st = srv.stats()
    assert st["cancelled"] == 2 and st["failed"] == 0 and st["requests"] == 4
