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
