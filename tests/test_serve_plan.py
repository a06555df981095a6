"""The served stream's slot plan (bench.py) fits its HBM budget: the slot
sizes come from the library's own workspace query, so a change to the
context's buffers that would push the plan over the budget fails here, on
the CPU, before a GPU run."""
import bench
from paper_2501_10622_gb300 import serve


def test_served_slots_fit_budget():
    need = serve.plan_bytes(bench.SERVED_SLOTS)
    assert 0 < need <= bench.SERVED_BUDGET, (need / 2 ** 30, bench.SERVED_BUDGET / 2 ** 30)


def test_plan_counts_every_slot():
    one = serve.plan_bytes({96: 1})
    assert serve.plan_bytes({96: 3}) == 3 * one
    assert serve.plan_bytes({96: 1, 192: 1}) > serve.plan_bytes({192: 1})
