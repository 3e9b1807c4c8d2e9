"""Host-side scheduling rules of the serving loop (no GPU): batch size
classes and admission of evidence-case slots by a device-memory budget."""
import pytest

from paper_1202_3777_gb300.serve import batch_size_class, slots_within_budget


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
