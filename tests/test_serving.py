"""Scheduling logic of the render server against a host-only executor: budget
admission, slot limit, FIFO order, cancellation, rejection and failures
(a device-side timeout injected as the error a real status check raises).
No GPU is involved."""
import time

import pytest

from paper_2505_18764_gb300.serving import Server, ServeRequest


class FakeHandle:
    def __init__(self, slot, request, t_end):
        self.slot, self.request, self.t_end = slot, request, t_end


class FakeExecutor:
    def __init__(self, mem, duration=0.002, fail=(), retry_once=()):
        self.mem, self.duration, self.fail = mem, duration, set(fail)
        self.retry_once = set(retry_once)
        self.submitted, self.live, self.max_live = [], 0, 0

    def memory(self, r):
        return self.mem.get(r.rid, 10)

    def submit(self, r, slot):
        self.submitted.append(r.rid)
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return FakeHandle(slot, r, time.perf_counter() + self.duration)

    def poll(self, h):
        return time.perf_counter() >= h.t_end

    def finish(self, h):
        self.live -= 1
        if h.request.rid in self.retry_once:
            from paper_2505_18764_gb300.serving import Retry
            self.retry_once.discard(h.request.rid)
            raise Retry()
        if h.request.rid in self.fail:
            from paper_2505_18764_gb300._lib import GsError, GS_ERR_TIMEOUT
            raise GsError(GS_ERR_TIMEOUT, "gs_check_status", "a device-side look-back wait gave up")
        return {"rid": h.request.rid}


def _reqs(n, gap=0.0):
    return [ServeRequest(rid=i, scene=0, camera=None, arrival=i * gap) for i in range(n)]


def test_all_complete_and_latency_reported():
    ex = FakeExecutor({})
    stats = Server(ex, hbm_budget_bytes=1000, max_slots=4).run(_reqs(30, gap=0.0005))
    assert stats["done"] == 30 and stats["p50_ms"] > 0 and stats["p99_ms"] >= stats["p50_ms"]
    assert stats["views_per_s"] > 0


def test_budget_limits_concurrency():
    ex = FakeExecutor({i: 40 for i in range(20)})
    srv = Server(ex, hbm_budget_bytes=100, max_slots=8)
    stats = srv.run(_reqs(20))
    assert stats["done"] == 20
    assert srv.peak_bytes <= 100 and ex.max_live <= 2 and srv.peak_concurrency == 2


def test_slot_limit_and_fifo_order():
    ex = FakeExecutor({})
    srv = Server(ex, hbm_budget_bytes=10**9, max_slots=3)
    srv.run(_reqs(12, gap=0.0))
    assert ex.max_live <= 3
    assert ex.submitted == list(range(12))


def test_cancel_before_admission():
    ex = FakeExecutor({i: 60 for i in range(5)}, duration=0.01)
    srv = Server(ex, hbm_budget_bytes=100, max_slots=4)
    reqs = _reqs(5)
    srv.cancel(3)
    stats = srv.run(reqs)
    assert reqs[3].status == "cancelled" and 3 not in ex.submitted
    assert stats["done"] == 4 and stats["cancelled"] == 1


def test_oversized_request_is_rejected_not_stuck():
    ex = FakeExecutor({2: 500})
    reqs = _reqs(5)
    stats = Server(ex, hbm_budget_bytes=100, max_slots=2).run(reqs)
    assert reqs[2].status == "rejected" and stats["done"] == 4


def test_device_failure_marks_request_failed_and_continues():
    ex = FakeExecutor({}, fail={1, 4})
    reqs = _reqs(8)
    stats = Server(ex, hbm_budget_bytes=1000, max_slots=2).run(reqs)
    assert [r.status for r in reqs].count("failed") == 2 and stats["done"] == 6
    assert "look-back" in reqs[1].error


def test_retry_requeues_at_the_front_and_keeps_arrival():
    ex = FakeExecutor({}, retry_once={2})
    reqs = _reqs(6, gap=0.0)
    stats = Server(ex, hbm_budget_bytes=1000, max_slots=1).run(reqs)
    assert stats["done"] == 6 and reqs[2].retries == 1 and stats["retries"] == 1
    assert ex.submitted.count(2) == 2
    # the retried request runs again before the ones that arrived after it
    assert ex.submitted.index(3) > len(ex.submitted) - 1 - ex.submitted[::-1].index(2)


class PlanExecutor(FakeExecutor):
    """Offers a fast plan and a smaller, slower one (the memory-efficiency mode)."""

    def __init__(self, fast, small):
        super().__init__({})
        self.fast, self.small, self.ran = fast, small, {}

    def plans(self, r):
        return [(self.fast, "single"), (self.small, "chunked")]

    def submit(self, r, slot, plan="single"):
        self.ran[r.rid] = plan
        return super().submit(r, slot)


def test_admission_takes_the_smaller_plan_when_the_fast_one_does_not_fit():
    # budget below the fast plan: every request runs chunked, none is rejected
    ex = PlanExecutor(fast=120, small=30)
    srv = Server(ex, hbm_budget_bytes=100, max_slots=4)
    stats = srv.run(_reqs(12, gap=0.0))
    assert stats["done"] == 12 and stats["rejected"] == 0
    assert set(ex.ran.values()) == {"chunked"} and stats["plans"] == {"chunked": 12}
    assert srv.peak_bytes <= 100 and srv.peak_concurrency == 3


def test_admission_prefers_the_fast_plan_and_falls_back_under_pressure():
    # room for one fast request; while it runs, the others take the small plan
    ex = PlanExecutor(fast=60, small=20)
    srv = Server(ex, hbm_budget_bytes=100, max_slots=4)
    stats = srv.run(_reqs(8, gap=0.0))
    assert stats["done"] == 8 and ex.ran[0] == "single"
    assert "chunked" in set(ex.ran.values())
    assert srv.peak_bytes <= 100


def test_smallest_plan_over_budget_is_rejected():
    ex = PlanExecutor(fast=500, small=200)
    stats = Server(ex, hbm_budget_bytes=100, max_slots=2).run(_reqs(3))
    assert stats["rejected"] == 3 and stats["done"] == 0
