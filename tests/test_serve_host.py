"""Host logic of the relax server (paper_2411_18194_gb300.serve) on CPU:
admission in arrival order under a memory budget, joining between lock
steps, retirement, and the latency statistics.  The batch and the contexts
are fakes: a fake member needs a given number of lock-step attempts."""
import numpy as np
import pytest

from inputs import Problem


class FakeMag:
    def __init__(self, need):
        self.left = need
        self.closed = False

    def close(self):
        self.closed = True


class FakeBatch:
    def __init__(self):
        self.members = []
        self.max_members = 0
        self.advances = 0

    def add(self, mag, goal, a, c):
        assert goal == "relax"
        self.members.append(mag)
        self.max_members = max(self.max_members, len(self.members))

    def remove(self, mag):
        self.members.remove(mag)

    def status(self, mag):
        return mag.left <= 0, 0

    def advance(self, n):
        self.advances += 1
        for m in self.members:
            m.left -= n
        return sum(m.left > 0 for m in self.members)

    def close(self):
        pass


class W:
    def __init__(self, shape, need):
        self.problem = Problem(shape, (4e-9, 4e-9, 2e-9), 1, frozenset({"DEMAG", "EXCH"}))
        self.need = need


@pytest.fixture
def server(monkeypatch):
    from paper_2411_18194_gb300 import serve
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "_make_magnet", lambda w, dt0: FakeMag(w.need))
    return serve


class Clock:
    """Simulated time: every call advances it by 1 ms."""
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


def test_request_bytes_counts_the_spectrum_once(server):
    a = server.request_bytes((256, 256, 2), False)
    b = server.request_bytes((256, 256, 2), True)
    n = 256 * 256 * 2
    assert b >= 9 * 12 * n and a > b
    assert server.request_bytes((64, 64, 1), True) < b


def test_fifo_admission_under_budget_and_release(server):
    reqs = [server.Request(i, W((128, 128, 1), need=8 + i), arrival=0.0, torque_tol=1e-3, max_time=1e-10)
            for i in range(6)]
    one = server.request_bytes((128, 128, 1), False)
    srv = server.RelaxServer(budget_bytes=2.5 * one, attempts_per_round=4)
    done = srv.run(reqs, clock=Clock())
    assert len(done) == 6 and srv.used == pytest.approx(0.0) and not srv.active
    # the budget admits the first request (spectrum built) plus shared-spectrum followers only
    assert srv.batch.max_members >= 2
    assert srv.batch.max_members * server.request_bytes((128, 128, 1), True) <= 2.5 * one + one
    order = [r.id for r in sorted(done, key=lambda r: r.admitted)]
    assert order == sorted(order)                      # admitted in arrival order
    for r in done:
        assert r.admitted >= r.arrival and r.done > r.admitted and r.mag is None


def test_spectrum_charged_per_geometry_and_build_buffers_at_admission_only(server):
    """The shared kernel spectrum stays charged while any request of its
    geometry runs and is released with the last one; the FP64 build buffers
    count only against the admission of the request that builds it."""
    shape = (128, 128, 1)
    reqs = [server.Request(0, W(shape, need=40), 0.0, 1e-3, 1e-10),
            server.Request(1, W(shape, need=8), 0.0, 1e-3, 1e-10)]
    srv = server.RelaxServer(budget_bytes=1e12, attempts_per_round=4)
    for r in reqs:
        srv.submit(r)
    srv._admit(0.0)
    st, sp = server.state_bytes(shape), server.spectrum_bytes(shape)
    assert len(srv.active) == 2
    assert srv.used == pytest.approx(2 * st + sp)       # no build buffers after admission
    for _ in range(3):                                  # request 1 (8 attempts) finishes first
        srv.batch.advance(srv.attempts)
    srv._retire(1.0)
    assert [r.id for r in srv.active] == [0]
    assert srv.used == pytest.approx(st + sp)           # spectrum still resident for request 0
    for _ in range(10):
        srv.batch.advance(srv.attempts)
    srv._retire(2.0)
    assert not srv.active and srv.used == pytest.approx(0.0)
    assert server.request_bytes(shape, False) == st + sp + server.build_bytes(shape)


def test_late_arrivals_join_while_others_run(server):
    reqs = [server.Request(0, W((64, 64, 1), need=400), 0.0, 1e-3, 1e-10),
            server.Request(1, W((64, 64, 1), need=8), 0.05, 1e-3, 1e-10)]
    srv = server.RelaxServer(budget_bytes=1e12, attempts_per_round=4)
    done = {r.id: r for r in srv.run(reqs, clock=Clock())}
    # the short request arrived during the long one, joined it and finished first
    assert done[1].admitted < done[0].done and done[1].done < done[0].done
    assert srv.batch.max_members == 2


def test_latency_stats(server):
    class R:
        def __init__(self, a, d):
            self.arrival, self.done = a, d

        @property
        def latency(self):
            return self.done - self.arrival
    rs = [R(0.0, 1.0), R(0.5, 1.5), R(1.0, 4.0)]
    st = server.latency_stats(rs)
    assert st["solves"] == 3 and st["span_s"] == 4.0 and st["solves_per_s"] == 0.75
    assert st["p50_s"] == 1.0 and st["p99_s"] == pytest.approx(np.percentile([1, 1, 3], 99))
