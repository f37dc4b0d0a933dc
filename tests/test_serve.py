"""Host-side admission logic of the serving loop (no device): budget and slot
limits, FIFO order with backfill, no starvation of the head, retirement."""
import pytest

from paper_2110_12448_gb300.serve import Request, Scheduler, percentile


def sched(budget=100, slots=3, backfill=True, max_bypass=2):
    return Scheduler(budget, slots, lambda r: r.workload, backfill=backfill, max_bypass=max_bypass)


def req(i, size):
    return Request(i, size, steps=10)


def test_admits_in_fifo_order_within_budget():
    s = sched()
    for i, b in enumerate([40, 30, 20, 50]):
        s.submit(req(i, b))
    got = [r.rid for r in s.admissible()]
    assert got == [0, 1, 2]          # 90 used; slot limit 3 reached
    assert s.used == 90
    s.retire(1)
    assert [r.rid for r in s.admissible()] == []  # 60 used + 50 > 100
    s.retire(0)
    assert [r.rid for r in s.admissible()] == [3]


def test_backfill_and_no_starvation():
    s = sched(budget=100, slots=10, max_bypass=2)
    s.submit(req(0, 60))
    assert [r.rid for r in s.admissible()] == [0]
    for i, b in [(1, 70), (2, 10), (3, 10), (4, 10)]:
        s.submit(req(i, b))
    # head (70) does not fit; small ones backfill, but at most max_bypass of them
    assert [r.rid for r in s.admissible()] == [2, 3]
    assert [r.rid for r in s.admissible()] == []
    s.retire(0)
    s.retire(2)
    s.retire(3)
    assert [r.rid for r in s.admissible()] == [1, 4]


def test_without_backfill_head_blocks():
    s = sched(budget=100, slots=10, backfill=False)
    s.submit(req(0, 60))
    s.admissible()
    s.submit(req(1, 70))
    s.submit(req(2, 10))
    assert s.admissible() == []


def test_oversized_request_rejected():
    s = sched(budget=100)
    with pytest.raises(ValueError):
        s.submit(req(0, 101))


def test_idle_and_percentiles():
    s = sched()
    assert s.idle
    s.submit(req(0, 10))
    assert not s.idle
    s.admissible()
    s.retire(0)
    assert s.idle
    assert percentile([1, 2, 3, 4], 50) == 2.5
    assert percentile(list(range(101)), 99) == 99.0
