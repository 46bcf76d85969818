"""Continuous-batching scheduler logic on the host (no GPU): admission by
memory footprint, batching by shape, stream reuse, draining."""
import pytest

from paper_2601_15401_gb300.serve import Request, Scheduler, latency_stats


class FakeBackend:
    """Each batch 'runs' for a fixed number of polls; footprint = 10 per request."""

    def __init__(self, n_streams=2, polls=2):
        self.n_streams = n_streams
        self.polls = polls
        self.launched = []

    def footprint(self, shape, n):
        return 10 * n

    def launch(self, b):
        self.launched.append(b)
        return [self.polls]

    def poll(self, h):
        h[0] -= 1
        return h[0] <= 0


def req(i, k=3, level=10, t=0.0):
    return Request(i, 14, k, level, tuple(range(k)), arrival=t)


def test_batches_group_by_shape_and_respect_max_batch():
    be = FakeBackend(n_streams=4)
    s = Scheduler(be, cap_bytes=10 ** 9, max_batch=3)
    for i in range(7):
        s.submit(req(i, k=3))
    for i in range(7, 9):
        s.submit(req(i, k=4, t=0.5))
    s.step(0.0)
    sizes = sorted(len(b.reqs) for b in be.launched)
    assert sizes == [1, 2, 3, 3]
    for b in be.launched:
        assert len({r.shape for r in b.reqs}) == 1


def test_admission_by_footprint_waits_for_memory():
    be = FakeBackend(n_streams=4, polls=1)
    s = Scheduler(be, cap_bytes=25, max_batch=8)  # at most 2 requests in flight
    for i in range(5):
        s.submit(req(i))
    s.step(0.0)
    assert sum(len(b.reqs) for b in s.running) == 2 and s.in_use == 20
    s.step(1.0)  # the first batch completes, the next two are admitted
    assert len(s.completed) == 2 and s.in_use == 20
    while not s.idle():
        s.step(2.0)
    assert len(s.completed) == 5 and s.in_use == 0


def test_continuous_batching_admits_late_arrivals_while_running():
    be = FakeBackend(n_streams=2, polls=3)
    s = Scheduler(be, cap_bytes=10 ** 9, max_batch=4)
    s.submit(req(0))
    s.step(0.0)
    s.submit(req(1, k=5))   # arrives while batch 0 runs: takes the free stream
    s.step(0.1)
    assert len(s.running) == 2
    s.submit(req(2))
    s.step(0.2)             # no stream free: waits in the queue
    assert s.pending() == 1
    while not s.idle():
        s.step(1.0)
    assert {r.rid for r in s.completed} == {0, 1, 2}


def test_batch_shrinks_to_the_backend_workspace():
    class Small(FakeBackend):
        def fits(self, shape, n):
            return n <= 2
    be = Small(n_streams=1)
    s = Scheduler(be, cap_bytes=10 ** 9, max_batch=8)
    for i in range(5):
        s.submit(req(i))
    s.step(0.0)
    assert [len(b.reqs) for b in be.launched] == [2]


def test_queue_limit_rejects():
    s = Scheduler(FakeBackend(), cap_bytes=10 ** 9, max_queue=2)
    assert s.submit(req(0)) and s.submit(req(1))
    assert not s.submit(req(2)) and s.rejected == 1


def test_latency_stats():
    rs = [Request(i, 14, 2, 2, (0, 1), arrival=0.0) for i in range(100)]
    for i, r in enumerate(rs):
        r.done = (i + 1) / 1000.0
    st = latency_stats(rs)
    assert st["p50_ms"] == pytest.approx(50.0) and st["p99_ms"] == pytest.approx(99.0)


class StuckBackend(FakeBackend):
    """Injects a fault on the host: every batch of shape k = 7 never completes."""

    def launch(self, b):
        self.launched.append(b)
        return [10 ** 9 if b.shape[1] == 7 else self.polls]

    def abandon(self, b):
        self.abandoned = getattr(self, "abandoned", 0) + 1


def test_watchdog_fails_a_stuck_batch_and_the_rest_completes():
    be = StuckBackend(n_streams=2, polls=1)
    s = Scheduler(be, cap_bytes=10 ** 9, max_batch=4, timeout_s=1.0)
    s.submit(req(0, k=7))
    for i in range(1, 6):
        s.submit(req(i, k=3, t=0.1))
    now = 0.0
    while not s.idle() and now < 10:
        s.step(now)
        now += 0.5
    assert [r.rid for r in s.failed] == [0] and s.failed[0].error == "timeout"
    assert sorted(r.rid for r in s.completed) == [1, 2, 3, 4, 5]
    assert be.abandoned == 1 and s.healthy_streams() == 1


class GroupingBackend(FakeBackend):
    """Cross-shape batching: requests of one ring degree share a batch; the
    footprint and the workspace check see the actual requests."""

    @staticmethod
    def group_key(r):
        return (r.log_n,)

    def footprint_reqs(self, reqs):
        return sum(r.level for r in reqs)

    def fits(self, reqs):
        return sum(r.k for r in reqs) <= 20


def test_cross_shape_batches_group_by_ring_degree():
    be = GroupingBackend()
    s = Scheduler(be, cap_bytes=10 ** 9, max_batch=16)
    # mixed k and level at two ring degrees
    reqs = [Request(i, 14 + (i % 2), 2 + i % 5, 10 + i % 7, (0,), arrival=i * 1e-6) for i in range(12)]
    for r in reqs:
        s.submit(r)
    s.step(0.0)
    for b in s.running:
        assert len({r.log_n for r in b.reqs}) == 1
        assert sum(r.k for r in b.reqs) <= 20
    assert any(len({(r.k, r.level) for r in b.reqs}) > 1 for b in s.running)
    # drain
    for t in range(1, 50):
        s.step(float(t))
        if s.idle():
            break
    assert sorted(r.rid for r in s.completed) == list(range(12))


def test_cross_shape_admission_uses_request_footprints():
    be = GroupingBackend()
    s = Scheduler(be, cap_bytes=25, max_batch=16)  # levels 10..16: at most two requests in flight
    for i in range(5):
        s.submit(Request(i, 16, 3, 10 + i, (0,), arrival=i * 1e-6))
    s.step(0.0)
    assert sum(len(b.reqs) for b in s.running) == 2
    assert s.in_use <= 25
