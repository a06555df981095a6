"""Continuous-batching halo-finding service on one GPU.

Jobs (a particle box on the device, its grid size and scales) arrive over
time.  The server keeps a fixed set of *slots* -- each a library context
(sized for one grid class) plus its own CUDA stream and output buffers,
created once at start-up so that no cudaMalloc happens while serving.  A job
is admitted as soon as it has arrived, a free slot of a class that fits it
exists, and the job's memory fits the HBM budget; admitted jobs run
concurrently on their slots' streams, so small jobs overlap with each other
and with large ones.  Admission is first-come-first-served with backfill: a
later job may take a free slot that the head of the queue cannot use.

`run_back_to_back` runs the same jobs one at a time, in arrival order, on one
stream -- the baseline the service is compared with.  Both report per-job
latency (completion - arrival, host clock), p50 / p99, and particles per
second over the makespan.  Results are per-job and deterministic: a job's
halo ids are identical alone, back to back, and in the mix.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import torch

from . import _lib
from . import synth

SIZE_CLASSES = (96, 192, 288, 384, 512)


@dataclass
class Job:
    jid: int
    ng: int
    box: float
    pos: torch.Tensor           # device float32 [np, 3]
    arrival: float              # seconds after the start of the run
    params: list = field(default_factory=list)
    # filled by the server
    admitted: float = math.nan
    done: float = math.nan
    n_halo: list = field(default_factory=list)
    checksum: int = 0

    @property
    def np(self) -> int:
        return int(self.pos.shape[0])


def smooth_sizes(lo=64, hi=512):
    return sorted({2 ** a * 3 ** b for a in range(1, 10) for b in range(0, 6) if lo <= 2 ** a * 3 ** b <= hi})


def poisson_jobs(n_jobs: int, rate: float = 200.0, lo_ng: int = 64, hi_ng: int = 512, per_cell: float = 8.0,
                 spacing: float = 0.78125, seed: int = 5, device="cuda", scales=(2.0,)):
    """A Poisson stream of jobs: exponential inter-arrival times at `rate` per
    second, grid sizes log-uniform in [lo_ng, hi_ng] rounded to 2^a 3^b,
    `per_cell` particles per cell, box = ng * spacing.  One clumped snapshot
    per distinct grid size is generated and shared by the jobs of that size."""
    g = torch.Generator().manual_seed(seed)
    t = 0.0
    jobs, snaps = [], {}
    for j in range(n_jobs):
        t += float(-math.log(1.0 - float(torch.rand(1, generator=g))) / rate)
        u = float(torch.rand(1, generator=g))
        ng = synth.smooth_ng(math.exp(math.log(lo_ng) + u * (math.log(hi_ng) - math.log(lo_ng))))
        ng = min(max(ng, lo_ng), hi_ng)
        box = ng * spacing
        if ng not in snaps:
            npart = int(round(per_cell * ng ** 3))
            snaps[ng] = synth.clumped_box(npart, box, None, seed=seed * 10000 + ng, device=device)
        params = [_lib.default_params(w) for w in scales]
        jobs.append(Job(j, ng, box, snaps[ng], t, params))
    return jobs


class Slot:
    """One context + stream + output buffers for jobs up to (ng, np)."""

    def __init__(self, device, ng, np_max, n_scales, cat_cap):
        self.ng, self.np_max, self.n_scales, self.cat_cap = ng, np_max, n_scales, cat_cap
        self.ctx = _lib.Context(device.index or 0, max_ng=ng, max_np=np_max, max_scales=n_scales)
        self.stream = torch.cuda.Stream(device)
        self.halo_id = torch.empty(n_scales * np_max, dtype=torch.int32, device=device)  # [ns][np] per job
        self.cat = torch.empty((n_scales, cat_cap, 64), dtype=torch.uint8, device=device)
        self.n_halo = torch.zeros(n_scales, dtype=torch.int64, device=device)
        self.event = torch.cuda.Event()
        self.job = None
        self.bytes = slot_bytes(ng, np_max, n_scales, cat_cap)

    def fits(self, job: Job) -> bool:
        return job.ng <= self.ng and job.np <= self.np_max and len(job.params) <= self.n_scales

    def launch(self, job: Job):
        ns = len(job.params)
        self.ctx.find(job.pos, job.box, job.ng, job.params, cat_cap=self.cat_cap, halo_id=self.job_ids(ns, job.np),
                      cat=self.cat[:ns], n_halo=self.n_halo[:ns], stream=self.stream)
        self.event.record(self.stream)
        self.job = job

    def job_ids(self, ns, np_):
        """The slot's id buffer as a contiguous [ns][np] array for one job."""
        return self.halo_id[: ns * np_].view(ns, np_)

    def finish(self):
        """Called once the slot's event has completed."""
        job = self.job
        ns = len(job.params)
        rc = self.ctx.sync(self.stream)
        if rc:
            raise _lib.CwthfError(rc, f"job {job.jid}")
        job.n_halo = [int(x) for x in self.n_halo[:ns].cpu()]
        hid = self.job_ids(ns, job.np)
        job.checksum = int((hid.to(torch.int64) * torch.arange(1, job.np + 1, device=hid.device)).sum().item())
        self.job = None


def slot_bytes(ng, np_max, n_scales, cat_cap):
    """Device bytes one slot holds: the context's workspace, the halo ids and
    the catalogue."""
    return _lib.workspace_bytes(ng, np_max, n_scales) + n_scales * np_max * 4 + n_scales * cat_cap * 64 + 64


def plan_bytes(slots_per_class, n_scales=1, per_cell=8.0, classes=SIZE_CLASSES, cat_cap=1 << 18):
    """Device bytes of a server's slots (the sizes Server allocates), without a GPU."""
    return sum(k * slot_bytes(ng, int(round(per_cell * ng ** 3)) + 1024, n_scales, cat_cap)
               for ng in classes for k in [slots_per_class.get(ng, 0)])


class Server:
    def __init__(self, device="cuda", budget_bytes=120 * 2 ** 30, slots_per_class=None, n_scales=1,
                 per_cell=8.0, classes=SIZE_CLASSES, cat_cap=1 << 18):
        self.device = torch.device(device)
        self.budget = budget_bytes
        if slots_per_class is None:
            slots_per_class = {96: 4, 192: 3, 288: 2, 384: 1, 512: 1}
        self.slots = []
        for ng in classes:
            for _ in range(slots_per_class.get(ng, 0)):
                self.slots.append(Slot(self.device, ng, int(round(per_cell * ng ** 3)) + 1024, n_scales, cat_cap))
        self.slots.sort(key=lambda s: s.bytes)
        self.used = sum(s.bytes for s in self.slots)
        if self.used > self.budget:
            raise ValueError(f"slots need {self.used / 2**30:.1f} GiB, above the {self.budget / 2**30:.1f} GiB budget")

    def close(self):
        for s in self.slots:
            s.ctx.close()
        self.slots = []

    def prepare(self, jobs):
        """Fill every slot's FFT and wavelet table slots for the (grid, box,
        scales) of the jobs it can take, so that serving does no table work."""
        seen = {(j.ng, j.box, tuple(p.w for p in j.params)) for j in jobs}
        for slot in self.slots:
            for ng, box, ws in sorted(seen):
                if ng <= slot.ng and len(ws) <= slot.n_scales:
                    slot.ctx.prepare(ng, box, ws, stream=slot.stream)
        torch.cuda.synchronize(self.device)

    def table_fills(self) -> int:
        return sum(s.ctx.table_fills() for s in self.slots if hasattr(s, "ctx"))

    def _pick(self, job):
        for s in self.slots:  # smallest fitting free slot first
            if s.job is None and s.fits(job):
                return s
        return None

    def run(self, jobs, poll_s=50e-6):
        """Serve `jobs` against their arrival times; returns statistics (with
        the number of table slots the run had to fill, 0 after prepare())."""
        if any(not any(s.fits(j) for s in self.slots) for j in jobs):
            raise ValueError("a job does not fit any slot class")
        fills0 = self.table_fills()
        queue, order = [], sorted(jobs, key=lambda j: j.arrival)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        nxt = 0
        running = []
        while nxt < len(order) or queue or running:
            now = time.perf_counter() - t0
            while nxt < len(order) and order[nxt].arrival <= now:
                queue.append(order[nxt])
                nxt += 1
            for job in list(queue):  # FCFS with backfill
                slot = self._pick(job)
                if slot is not None:
                    job.admitted = time.perf_counter() - t0
                    slot.launch(job)
                    running.append(slot)
                    queue.remove(job)
            for slot in list(running):
                if slot.event.query():
                    job = slot.job
                    job.done = time.perf_counter() - t0
                    slot.finish()
                    running.remove(slot)
            if not queue and not running and nxt < len(order):
                time.sleep(max(0.0, min(order[nxt].arrival - (time.perf_counter() - t0), 1e-3)))
            elif running:
                time.sleep(poll_s)
        return {**stats(jobs), "table_fills": self.table_fills() - fills0}

    def run_back_to_back(self, jobs):
        """The same jobs one at a time in arrival order on one stream (no overlap)."""
        order = sorted(jobs, key=lambda j: j.arrival)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        for job in order:
            now = time.perf_counter() - t0
            if job.arrival > now:
                time.sleep(job.arrival - now)
            slot = next(s for s in self.slots if s.fits(job))
            job.admitted = time.perf_counter() - t0
            slot.launch(job)
            slot.event.synchronize()
            job.done = time.perf_counter() - t0
            slot.finish()
        return stats(jobs)


def with_arrivals(jobs, arrivals):
    """The same jobs (same snapshots and parameters) with new arrival times."""
    return [Job(j.jid, j.ng, j.box, j.pos, float(a), j.params) for j, a in zip(jobs, arrivals)]


def scaled_load(jobs, rate, drawn_rate):
    """The jobs' Poisson arrivals, drawn at `drawn_rate` jobs per second,
    stretched or squeezed to `rate` (the same draws: same order, same
    relative gaps).  rate = inf: every job arrives at time 0."""
    if math.isinf(rate):
        return with_arrivals(jobs, [0.0] * len(jobs))
    return with_arrivals(jobs, [j.arrival * drawn_rate / rate for j in jobs])


def stats(jobs):
    lat = sorted(j.done - j.arrival for j in jobs)
    q = lambda p: lat[min(len(lat) - 1, max(0, int(math.ceil(p * len(lat))) - 1))]
    span = max(j.done for j in jobs) - min(j.arrival for j in jobs)
    npart = sum(j.np for j in jobs)
    offered_span = max(j.arrival for j in jobs) - min(j.arrival for j in jobs)
    return {"jobs": len(jobs), "p50_ms": q(0.50) * 1e3, "p99_ms": q(0.99) * 1e3, "mean_ms": sum(lat) / len(lat) * 1e3,
            "makespan_s": span, "mparticles_per_s": npart / span / 1e6,
            "offered_mparticles_per_s": npart / max(offered_span, 1e-9) / 1e6,
            "particles": npart}
