"""Host logic of the serving form on the CPU: HBM-budget admission of handles
(serve.HandlePool), with fake handles in place of device workspaces."""
import pytest

from paper_1807_04638_gb300.serve import HandlePool, Reservation


class Fake:
    def __init__(self, name):
        self.name = name
        self.closed = False

    def close(self):
        self.closed = True


def test_admits_until_the_budget_and_waits_for_busy_handles():
    pool = HandlePool(100)
    a = pool.acquire("A", 40, lambda: Fake("a1"))
    b = pool.acquire("A", 40, lambda: Fake("a2"))
    assert a[1] == 40 and b[1] == 40 and pool.used == 80
    # 40 more would exceed 100 and nothing is parked: wait
    assert pool.acquire("B", 40, lambda: Fake("b")) is None
    assert pool.used == 80 and pool.peak_used == 80


def test_parked_handle_is_reused_for_the_same_key_only():
    pool = HandlePool(100)
    a = pool.acquire("A", 40, lambda: Fake("a"))
    pool.park("A", a)
    made = []
    again = pool.acquire("A", 40, lambda: made.append(1) or Fake("new"))
    assert again is a and not made and pool.used == 40


def test_parked_handles_of_other_keys_are_evicted_to_make_room():
    pool = HandlePool(100)
    a = pool.acquire("A", 60, lambda: Fake("a"))
    pool.park("A", a)
    b = pool.acquire("B", 60, lambda: Fake("b"))
    assert b is not None and a[0].closed
    assert pool.used == 60 and pool.peak_used == 60


def test_requests_that_can_never_fit_are_rejected():
    pool = HandlePool(100)
    with pytest.raises(ValueError):
        pool.acquire("A", 101, lambda: Fake("x"))
    with pytest.raises(ValueError):
        pool.acquire("A", 0, lambda: Fake("x"))   # invalid shape or parameters
    assert pool.used == 0


def test_failed_handles_are_dropped_and_parked_ones_closed_at_the_end():
    pool = HandlePool(100)
    a = pool.acquire("A", 30, lambda: Fake("a"))
    b = pool.acquire("B", 30, lambda: Fake("b"))
    assert pool.drop(a) is a[0] and not a[0].closed   # the caller closes it
    assert pool.used == 30
    pool.park("B", b)
    pool.close_parked()
    assert b[0].closed and pool.used == 0 and not pool.parked
    assert pool.peak_used == 60


def test_reservation_counts_bytes_before_the_handle_exists():
    """The server reserves bytes under its lock and creates the handle (and
    closes evicted ones) outside it: the reservation already counts against
    the budget, eviction is undone when room cannot be made, and a failed
    creation gives the bytes back."""
    pool = HandlePool(100)
    a = pool.acquire("A", 50, lambda: Fake("a"))
    pool.park("A", a)
    b = pool.acquire("B", 40, lambda: Fake("b"))          # in use
    r = pool.reserve("C", 60)                               # needs A's room
    assert isinstance(r, Reservation) and r.victims == [a[0]] and not a[0].closed
    assert pool.used == 100 and not pool.parked["A"]
    # nothing else can be admitted while the reservation holds its bytes
    assert pool.reserve("D", 10) is None
    pool.cancel(r)
    assert pool.used == 40
    # no room even after evicting every parked handle: the parked one stays
    pool.park("B", b)
    c = pool.acquire("C", 50, lambda: Fake("c"))
    assert pool.reserve("E", 60) is None
    assert pool.parked["B"] == [b] and pool.used == 90


def test_failed_creation_releases_the_reservation():
    pool = HandlePool(100)

    def boom():
        raise RuntimeError("device out of memory")

    with pytest.raises(RuntimeError):
        pool.acquire("A", 70, boom)
    assert pool.used == 0
