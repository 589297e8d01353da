"""Admission and budget logic of the serving loop, on the CPU with a fake device."""
import pytest

from paper_2501_07047_gb300.serve import Admission, Request, request_bytes, serve


class FakeExecutor:
    """Completes each request after a fixed number of polls; records concurrency."""

    def __init__(self, polls=3):
        self.polls = polls
        self.live = 0
        self.max_live = 0
        self.order = []

    def launch(self, req):
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        self.order.append(req.rid)
        return {"left": self.polls}

    def done(self, h):
        h["left"] -= 1
        if h["left"] <= 0:
            self.live -= 1
            return True
        return False

    def outputs(self, req, h):
        return ()


def test_request_bytes_worst_case_fits_many_in_40gb():
    worst = request_bytes(16, 36)
    assert 90e6 < worst < 120e6
    assert (40 << 30) // worst >= 350


def test_budget_never_exceeded_and_fifo():
    budget = 3 * request_bytes(13, 8) + 10
    adm = Admission(budget, max_slots=100)
    reqs = [Request(i, 13, 8, 0.0) for i in range(7)]
    for r in reqs:
        adm.submit(r)
    first = list(adm.admit())
    assert [r.rid for r in first] == [0, 1, 2]          # the fourth does not fit
    assert adm.in_use <= budget and adm.active == 3
    adm.release(first[1])
    nxt = list(adm.admit())
    assert [r.rid for r in nxt] == [3]                   # freed memory admits the next in order
    assert adm.high_water <= budget


def test_oversized_request_rejected():
    adm = Admission(request_bytes(14, 8), max_slots=4)
    big = Request(0, 16, 36, 0.0)
    adm.submit(big)
    assert big.status == "rejected" and not adm.queue


def test_slot_limit():
    adm = Admission(1 << 40, max_slots=2)
    for i in range(5):
        adm.submit(Request(i, 13, 8, 0.0))
    assert len(list(adm.admit())) == 2


def test_serve_loop_with_fake_device():
    ex = FakeExecutor(polls=4)
    reqs = [Request(i, 13 + (i % 3), 8 + i, arrival=0.0005 * i) for i in range(40)]
    budget = 5 * request_bytes(15, 48)
    st = serve(reqs, ex, budget_bytes=budget, max_slots=6)
    assert st["completed"] == 40 and st["rejected"] == 0
    assert ex.max_live <= 6 and st["memory_high_water_bytes"] <= budget
    assert ex.order == sorted(ex.order)                  # admitted in arrival order
    assert all(r.completed >= r.arrival for r in reqs)
