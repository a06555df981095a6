"""The serving scheduler's host logic on the CPU: slots are fakes whose
completion event fires a set time after launch, so admission order, backfill,
slot choice and the statistics are checked without a GPU."""
import time

import pytest
import torch

from paper_2501_10622_gb300 import serve


class FakeEvent:
    def __init__(self):
        self.t = None

    def query(self):
        return self.t is not None and time.perf_counter() >= self.t

    def synchronize(self):
        while not self.query():
            time.sleep(1e-4)


class FakeSlot:
    def __init__(self, ng, np_max, seconds):
        self.ng, self.np_max, self.n_scales, self.bytes = ng, np_max, 1, 0
        self.job, self.event, self.seconds, self.log = None, FakeEvent(), seconds, []

    def fits(self, job):
        return job.ng <= self.ng and job.np <= self.np_max

    def launch(self, job):
        assert self.job is None, "a slot runs one job at a time"
        self.job = job
        self.event.t = time.perf_counter() + self.seconds
        self.log.append(job.jid)

    def finish(self):
        self.job.n_halo = [0]
        self.job, self.event.t = None, None


def _server(monkeypatch, slots):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    srv = serve.Server.__new__(serve.Server)
    srv.device = torch.device("cpu")
    srv.slots = sorted(slots, key=lambda s: s.ng)
    return srv


def _job(jid, ng, arrival):
    return serve.Job(jid, ng, ng * 0.78125, torch.empty((ng ** 3 // 64, 3)), arrival)


def test_backfill_admits_a_later_small_job_past_a_blocked_large_one(monkeypatch):
    small, large = FakeSlot(96, 96 ** 3, 0.005), FakeSlot(512, 512 ** 3, 0.060)
    srv = _server(monkeypatch, [large, small])
    jobs = [_job(0, 384, 0.000), _job(1, 384, 0.001), _job(2, 64, 0.002)]
    srv.run(jobs)
    j0, j1, j2 = jobs
    assert all(j.done >= j.admitted >= j.arrival for j in jobs)
    assert j2.admitted < j1.admitted          # the small job did not wait behind job 1
    assert j1.admitted >= j0.done - 1e-3      # job 1 waited for the only large slot
    assert large.log == [0, 1] and small.log == [2]


def test_smallest_fitting_free_slot_first(monkeypatch):
    small, large = FakeSlot(96, 96 ** 3, 0.002), FakeSlot(512, 512 ** 3, 0.002)
    srv = _server(monkeypatch, [large, small])
    jobs = [_job(0, 64, 0.0), _job(1, 64, 0.0)]
    srv.run(jobs)
    assert small.log[0] == 0 and large.log == [1]  # the second one takes the larger free slot


def test_back_to_back_runs_one_job_at_a_time(monkeypatch):
    slot = FakeSlot(512, 512 ** 3, 0.003)
    srv = _server(monkeypatch, [slot])
    jobs = [_job(i, 96, 0.0) for i in range(4)]
    srv.run_back_to_back(jobs)
    order = sorted(jobs, key=lambda j: j.admitted)
    for a, b in zip(order, order[1:]):
        assert b.admitted >= a.done


def test_a_job_larger_than_every_slot_is_refused(monkeypatch):
    srv = _server(monkeypatch, [FakeSlot(96, 96 ** 3, 0.001)])
    with pytest.raises(ValueError):
        srv.run([_job(0, 192, 0.0)])


def test_stats_quantiles():
    jobs = [_job(i, 8, 0.0) for i in range(100)]
    for i, j in enumerate(jobs):
        j.done = (i + 1) * 1e-3  # latencies 1 .. 100 ms
    s = serve.stats(jobs)
    assert s["p50_ms"] == pytest.approx(50.0) and s["p99_ms"] == pytest.approx(99.0)
    assert s["mean_ms"] == pytest.approx(50.5) and s["jobs"] == 100


def test_poisson_jobs_sizes_and_arrivals():
    jobs = serve.poisson_jobs(12, rate=100.0, lo_ng=8, hi_ng=24, per_cell=0.5, device="cpu")
    sizes = set(serve.smooth_sizes(8, 24))
    assert all(j.ng in sizes for j in jobs)
    assert all(b.arrival > a.arrival for a, b in zip(jobs, jobs[1:]))
    assert all(j.np == round(0.5 * j.ng ** 3) for j in jobs)
    for j in jobs:
        assert float(j.pos.min()) >= 0.0 and float(j.pos.max()) < j.box


def test_scaled_load_keeps_the_draws():
    jobs = [serve.Job(i, 32, 25.0, torch.zeros((5, 3)), 0.01 * i * i) for i in range(6)]
    fast = serve.scaled_load(jobs, 400.0, 200.0)
    assert [j.arrival for j in fast] == pytest.approx([0.005 * i * i for i in range(6)])
    assert [j.jid for j in fast] == [j.jid for j in jobs] and fast[3].pos is jobs[3].pos
    burst = serve.scaled_load(jobs, float("inf"), 200.0)
    assert all(j.arrival == 0.0 for j in burst)
