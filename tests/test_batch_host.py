"""The batched form's job placement on the CPU: longest job first onto the
least-loaded slot."""
import numpy as np

from paper_2501_10622_gb300.batch import assign_slots


def _loads(sizes, slots, n):
    load = [0] * n
    for (ng, np_), s in zip(sizes, slots):
        load[s] += ng ** 3 + np_
    return load


def test_every_job_placed_and_loads_within_the_lpt_bound():
    rng = np.random.default_rng(4)
    sizes = [(int(rng.choice([32, 64, 96, 128, 192])), int(10 ** rng.uniform(4, 7))) for _ in range(64)]
    slots = assign_slots(sizes, 8)
    assert len(slots) == 64 and set(slots) <= set(range(8))
    load = _loads(sizes, slots, 8)
    cost = [ng ** 3 + p for ng, p in sizes]
    # greedy LPT: the heaviest slot exceeds the mean by at most one job
    assert max(load) <= sum(cost) / 8 + max(cost)
    assert sum(load) == sum(cost)


def test_longest_jobs_go_to_distinct_slots_first():
    sizes = [(16, 0), (192, 0), (64, 0), (128, 0)]
    slots = assign_slots(sizes, 4)
    assert len(set(slots)) == 4            # four jobs, four slots: one each
    assert slots[1] == 0 and slots[3] == 1  # the two longest take slots 0 and 1


def test_more_slots_than_jobs_and_ties():
    assert assign_slots([(32, 10), (32, 10)], 3) == [0, 1]
    assert assign_slots([], 2) == []
