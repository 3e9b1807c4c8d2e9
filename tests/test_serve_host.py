"""Host-side scheduling rules of the serving loop (no GPU): batch size
classes, slots and run-time admission by a device-memory budget, the SM
share of a batch, and the overlap count of kernel spans."""
import pytest

from paper_1202_3777_gb300.serve import (admissible, batch_size_class, overlapping_pairs, slots_within_budget,
                                         sm_share)


def test_batch_size_class():
    assert batch_size_class(1) == 1
    assert [batch_size_class(n) for n in (2, 7, 8, 9, 16, 17, 63, 64)] == [8, 8, 8, 16, 16, 24, 64, 64]


@pytest.mark.parametrize("budget,table,case,maxb,expect", [
    (1000, 100, 10, 64, 64),      # room for 90 slots, capped at 64
    (1000, 100, 20, 64, 40),      # 45 slots, rounded down to a multiple of 8
    (1000, 100, 200, 64, 4),      # 4 slots (below 8: kept as is)
    (1000, 995, 10, 64, 0),       # the tables fit, no slot does
    (100, 200, 1, 64, 0),         # the tables alone exceed the budget
])
def test_slots_within_budget(budget, table, case, maxb, expect):
    assert slots_within_budget(budget, table, case, maxb) == expect


class _FakeEvent:
    def __init__(self, t_done):
        self.t_done = t_done

    def query(self):
        import time
        return time.perf_counter() >= self.t_done


def _fake_server(service_s, slots=8):
    """A Server whose batches are timers instead of propagations (the
    scheduling loop itself is under test)."""
    import time
    from paper_1202_3777_gb300 import serve

    class FakeServer(serve.Server):
        def __init__(self):
            self.trees = {"a": serve._Resident("a", None, 4, slots, None, 10)}
            self.completed = []
            self.launches = []

        def _launch(self, r):
            take = min(len(r.queue), r.slots)
            r.batch = [r.queue.popleft() for _ in range(take)]
            r.event = _FakeEvent(time.perf_counter() + service_s)
            self.launches.append((time.perf_counter(), take))

        def _finish(self, r):
            t = time.perf_counter()
            for q in r.batch:
                q.done, q.status = t, 0
                self.completed.append(q)
            r.batch, r.event = [], None

    return FakeServer()


def test_run_arrivals_serves_while_queries_arrive():
    """Batches start as soon as queries wait, not once every arrival is in:
    with arrivals spread over 0.3 s and 1 ms batches, no query waits long."""
    import numpy as np
    from paper_1202_3777_gb300.serve import Query, latency_summary
    srv = _fake_server(0.001)
    arr = [(0.01 * i, Query(i, "a", np.full(4, -1, np.int16))) for i in range(30)]
    done = srv.run_arrivals(arr)
    assert len(done) == 30 and all(q.status == 0 for q in done)
    lat = np.array([q.done - q.arrival for q in done])
    assert lat.max() < 0.1, lat.max()
    assert srv.launches[0][0] < arr[-1][0] + min(q.arrival for q in done)   # the first batch ran before the last arrival
    assert latency_summary(done, {"a": 10})["queries"] == 30


def test_run_arrivals_batches_a_burst_up_to_the_slots():
    import numpy as np
    from paper_1202_3777_gb300.serve import Query
    srv = _fake_server(0.002, slots=8)
    done = srv.run_arrivals([(0.0, Query(i, "a", np.full(4, -1, np.int16))) for i in range(20)])
    assert sorted(q.qid for q in done) == list(range(20))
    assert [n for _, n in srv.launches] == [8, 8, 4]


@pytest.mark.parametrize("waiting,slots,free,case,expect", [
    (5, 64, 10**9, 100, 5),        # everything waiting fits
    (100, 64, 10**9, 100, 64),     # capped by the slots
    (20, 64, 1600, 100, 16),       # 20 would reserve 24 slots: 16 fit the budget left
    (20, 64, 700, 100, 1),         # only a single case fits
    (3, 64, 50, 100, 0),           # nothing fits: the batch waits
])
def test_admissible(waiting, slots, free, case, expect):
    n = admissible(waiting, slots, free, case)
    assert n == expect
    assert n == 0 or batch_size_class(n) * case <= free


def test_sm_share_and_overlap_count():
    assert sm_share(152, False) == 0 and sm_share(152, True) == 76
    spans = [("a", 0, 10, 8), ("b", 5, 15, 8), ("a", 20, 30, 8), ("b", 31, 40, 1), ("a", 12, 14, 1)]
    assert overlapping_pairs(spans) == 2     # (a 0-10, b 5-15) and (b 5-15, a 12-14)


def _admission_server(budget_cases):
    """Two trees whose batches are timers; the budget leaves room for the
    per-case state of `budget_cases` cases in flight."""
    import time
    from paper_1202_3777_gb300 import serve

    class FakeServer(serve.Server):
        def __init__(self):
            self.trees = {n: serve._Resident(n, None, 4, 16, None, 10, case_bytes=100, table_bytes=1000)
                          for n in ("a", "b")}
            self.budget = 2000 + 100 * budget_cases
            self.table_bytes = 2000
            self.n_sm = 152
            self.completed, self.spans, self.issued = [], [], []
            self.deferred = 0

        def _issue(self, r, batch, n, cap):
            r.event = _FakeEvent(time.perf_counter() + 0.003)
            self.issued.append((r.name, n, cap, self.free_bytes))

        def _finish(self, r):
            for q in r.batch:
                q.done, q.status = time.perf_counter(), 0
                self.completed.append(q)
            r.batch, r.event, r.reserved = [], None, 0

    return FakeServer()


def test_memory_budget_defers_a_batch_until_another_finishes():
    """With room for 8 cases in flight, a full batch of one tree makes the
    other tree's batch wait; it starts once the first finishes, and the
    batches in flight never exceed the budget."""
    import numpy as np
    from paper_1202_3777_gb300.serve import Query
    srv = _admission_server(8)
    arr = [(0.0, Query(i, "a" if i < 8 else "b", np.full(4, -1, np.int16))) for i in range(16)]
    done = srv.run_arrivals(arr)
    assert len(done) == 16
    assert srv.deferred > 0
    assert all(free >= 0 for *_, free in srv.issued)
    assert [x[:2] for x in srv.issued] == [("a", 8), ("b", 8)]


def test_batches_share_the_sms_when_other_trees_wait():
    import numpy as np
    from paper_1202_3777_gb300.serve import Query
    srv = _admission_server(64)
    done = srv.run_arrivals([(0.0, Query(i, "ab"[i % 2], np.full(4, -1, np.int16))) for i in range(8)])
    assert len(done) == 8
    assert [x[2] for x in srv.issued][:2] == [76, 76]     # both trees had work: half of the SMs each
    lone = _admission_server(64)
    lone.run_arrivals([(0.0, Query(0, "a", np.full(4, -1, np.int16)))])
    assert lone.issued[0][2] == 0                          # alone: every SM
