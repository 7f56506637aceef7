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
    monkeypatch.setattr(serve, "_build_async", lambda w, dt0: FakeMag(w.need))
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
    srv = server.RelaxServer(budget_bytes=1e12, attempts_per_round=4, build_async=False)
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


class SlowBuild:
    """A context build on the worker thread that, for the geometry `shape`,
    finishes only after the batch has run `steps` lock steps (set from
    FakeBatch.advance); other geometries build at once."""
    def __init__(self, steps, shape):
        import threading
        self.steps = steps
        self.shape = shape
        self.event = threading.Event()
        self.started = threading.Event()

    def __call__(self, w, dt0):
        if tuple(w.problem.shape) != self.shape:
            return FakeMag(w.need)
        self.started.set()
        assert self.event.wait(10.0)
        return FakeMag(w.need)


def test_new_geometry_builds_while_the_batch_steps(server, monkeypatch):
    """A request of a new geometry has its context (and kernel spectrum)
    built on the worker thread while the admitted members keep stepping; it
    joins after its build, and its build buffers are released then."""
    slow = SlowBuild(steps=5, shape=(96, 64, 1))
    monkeypatch.setattr(server, "_build_async", slow)

    class CountingBatch(FakeBatch):
        def advance(self, n):
            if slow.started.is_set():
                slow.steps -= 1
                if slow.steps <= 0:
                    slow.event.set()
            return super().advance(n)
    monkeypatch.setattr(server, "Batch", CountingBatch)
    monkeypatch.setattr(server, "_make_magnet", lambda w, dt0: FakeMag(w.need))
    a = server.Request(0, W((64, 64, 1), need=400), 0.0, 1e-3, 1e-10)
    b = server.Request(1, W((96, 64, 1), need=8), 0.002, 1e-3, 1e-10)
    srv = server.RelaxServer(budget_bytes=1e12, attempts_per_round=4, build_async=True)
    srv.submit(a)
    srv._admit(0.0)                 # a's build on the worker (fake: immediate)
    srv.pending[0][1].result(5.0)
    srv._collect(0.001)
    assert [r.id for r in srv.active] == [0]
    srv.submit(b)
    srv._admit(0.003)
    assert srv.pending and srv.pending[0][0] is b and not b.admitted
    shape_b = (96, 64, 1)
    assert srv.used == pytest.approx(server.state_bytes((64, 64, 1)) + server.spectrum_bytes((64, 64, 1)) +
                                     server.request_bytes(shape_b, False))
    assert slow.started.wait(5.0)                   # the worker thread is building b
    steps = 0
    while srv.pending:
        srv.batch.advance(srv.attempts)            # the member keeps stepping during b's build
        steps += 1
        srv.pending[0][1].result(5.0) if slow.event.is_set() else None
        srv._collect(0.01 * steps)
        assert steps < 50
    assert steps >= 5 and b.admitted is not None
    assert srv.used == pytest.approx(server.state_bytes((64, 64, 1)) + server.spectrum_bytes((64, 64, 1)) +
                                     server.state_bytes(shape_b) + server.spectrum_bytes(shape_b))
    srv.close()


def test_same_geometry_waits_for_the_pending_build(server):
    reqs = [server.Request(i, W((128, 64, 1), need=8 + 4 * i), 0.0, 1e-3, 1e-10) for i in range(3)]
    srv = server.RelaxServer(budget_bytes=1e12, attempts_per_round=4, build_async=True)
    done = srv.run(reqs, clock=Clock())
    assert [r.status for r in done] == [0, 0, 0]
    assert all(r.accepted >= reqs[0].accepted for r in reqs)
    assert sorted(r.admitted for r in reqs) == [r.admitted for r in reqs]
    assert srv.used == pytest.approx(0.0) and not srv.building and not srv.pending
    srv.close()


def test_refused_admission_waits_for_memory(server):
    """A request that does not fit beside the running ones stays queued
    (nothing of it is built) until a member leaves."""
    big, small = (256, 256, 1), (128, 128, 1)
    first = server.Request(0, W(big, need=40), 0.0, 1e-3, 1e-10)
    second = server.Request(1, W(small, need=8), 0.0, 1e-3, 1e-10)
    # the first is admitted into the empty server; once its build buffers are
    # freed the second still does not fit beside it
    budget = server.state_bytes(big) + server.spectrum_bytes(big) + 0.5 * server.request_bytes(small, False)
    srv = server.RelaxServer(budget_bytes=budget, attempts_per_round=4)
    done = {r.id: r for r in srv.run([first, second], clock=Clock())}
    assert done[1].accepted >= done[0].done          # refused while the first ran
    assert done[0].status == 0 and done[1].status == 0
    assert srv.batch.max_members == 1 and srv.used == pytest.approx(0.0)
    srv.close()


def test_deadline_ends_running_and_queued_requests(server):
    """Past its wall-clock deadline a running request leaves the batch and a
    queued one leaves the queue, both with MMP_E_TIMEOUT, and their memory is
    released; the others finish normally."""
    shape = (128, 128, 1)
    long_ = server.Request(0, W(shape, need=10 ** 6), 0.0, 1e-3, 1e-10, deadline=0.05)
    blocked = server.Request(1, W((256, 128, 1), need=8), 0.0, 1e-3, 1e-10, deadline=0.02)
    ok = server.Request(2, W(shape, need=8), 0.0, 1e-3, 1e-10)
    budget = server.request_bytes(shape, False) + server.request_bytes(shape, True) + 1.0
    srv = server.RelaxServer(budget_bytes=budget, attempts_per_round=4, build_async=False)
    done = {r.id: r for r in srv.run([long_, blocked, ok], clock=Clock())}
    assert done[0].status == server.MMP_E_TIMEOUT and done[0].done >= 0.05
    assert done[1].status == server.MMP_E_TIMEOUT and done[1].admitted is None and done[1].mag is None
    assert done[2].status == 0
    assert not srv.active and srv.used == pytest.approx(0.0)
    srv.close()


def test_failed_build_ends_the_request_with_its_status(server, monkeypatch):
    """A context build that fails (here the library's MMP_E_OOM from a
    refused allocation, injected on the host) ends its request with that
    status and returns its reserved memory; the server keeps serving."""
    from paper_2411_18194_gb300.binding import MmpError

    def failing(w, dt0):
        if w.problem.shape == (96, 96, 1):
            raise MmpError(-2, "allocation refused (injected)")
        return FakeMag(w.need)
    monkeypatch.setattr(server, "_build_async", failing)
    reqs = [server.Request(0, W((96, 96, 1), need=8), 0.0, 1e-3, 1e-10),
            server.Request(1, W((64, 64, 1), need=8), 0.001, 1e-3, 1e-10)]
    srv = server.RelaxServer(budget_bytes=1e12, attempts_per_round=4, build_async=True)
    done = {r.id: r for r in srv.run(reqs, clock=Clock())}
    assert done[0].status == -2 and done[0].admitted is None
    assert done[1].status == 0
    assert srv.used == pytest.approx(0.0) and not srv.spectra[((96, 96, 1), (4e-9, 4e-9, 2e-9))]
    srv.close()
