"""Batched halo finding: many uneven periodic subvolumes in one CUDA graph.

The jobs are spread over `n_slots` slots (a library context with its own
stream), longest job first onto the least-loaded slot.  One pass over all
jobs -- each job's whole cwthf_find (deposit, FFT, segmentation, assignment)
on its slot's stream, the slot streams forked from and joined back into one
capture stream -- is recorded once into a CUDA graph; a batch then costs a
single graph launch, and jobs on different slots overlap on the GPU.

No job runs eagerly before the capture: the library keeps its FFT and
wavelet tables in slots sized when the contexts are created; each slot's
tables for its jobs are filled once (cwthf_prepare) before the capture, so
the graph only reads them.  Results are deterministic: each job's halo ids
equal those of a single cwthf_find call.  With `fft_plans` (autotune.tune /
autotune.load) every slot uses the FFT radix orders and tile widths the
autotuner picked for each grid size.
"""
from __future__ import annotations

import torch

from . import _lib, autotune


class BatchJob:
    def __init__(self, pos, box, ng, params):
        self.pos, self.box, self.ng, self.params = pos, box, ng, params
        self.np = int(pos.shape[0])
        self.slot = None
        self.halo_id = None
        self.cat = None
        self.n_halo = None


def assign_slots(sizes, n_slots):
    """Longest-processing-time placement: jobs (ng, np), costed as cells +
    particles, longest first onto the least-loaded slot (the lowest index on
    ties).  Returns each job's slot, in the jobs' order."""
    load = [0] * n_slots
    slot = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda i: -(sizes[i][0] ** 3 + sizes[i][1])):
        s = min(range(n_slots), key=lambda k: load[k])
        slot[i] = s
        load[s] += sizes[i][0] ** 3 + sizes[i][1]
    return slot


class Batch:
    def __init__(self, jobs, n_slots=8, cat_cap=1 << 16, device="cuda", fft_plans=None):
        self.device = torch.device(device)
        self.jobs = list(jobs)
        ns = max(len(j.params) for j in self.jobs)
        max_ng = max(j.ng for j in self.jobs)
        max_np = max(j.np for j in self.jobs)
        self.n_slots = min(n_slots, len(self.jobs))
        self.ctx = [_lib.Context(self.device.index or 0, max_ng=max_ng, max_np=max_np, max_scales=ns)
                    for _ in range(self.n_slots)]
        if fft_plans:  # FFT plans picked by the autotuner (autotune.py)
            for c in self.ctx:
                autotune.apply(c, fft_plans)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.n_slots)]
        for j, s in zip(self.jobs, assign_slots([(j.ng, j.np) for j in self.jobs], self.n_slots)):
            j.slot = s
        for j in self.jobs:
            k = len(j.params)
            j.halo_id = torch.empty((k, j.np), dtype=torch.int32, device=self.device)
            j.cat = torch.empty((k, cat_cap, 64), dtype=torch.uint8, device=self.device)
            j.n_halo = torch.zeros(k, dtype=torch.int64, device=self.device)
        self.cat_cap = cat_cap
        self.graph = None
        self.main = torch.cuda.Stream(self.device)

    def _enqueue(self, main):
        """All jobs on their slots' streams, forked from / joined into `main`."""
        for s in self.streams:
            s.wait_stream(main)
        for j in self.jobs:
            s = self.streams[j.slot]
            with torch.cuda.stream(s):
                self.ctx[j.slot].find(j.pos, j.box, j.ng, j.params, cat_cap=self.cat_cap, halo_id=j.halo_id,
                                      cat=j.cat, n_halo=j.n_halo, stream=s)
        for s in self.streams:
            main.wait_stream(s)

    def run_eager(self):
        cur = torch.cuda.current_stream(self.device)
        self._enqueue(cur)
        torch.cuda.synchronize(self.device)
        self.check()

    def capture(self):
        for j in self.jobs:  # tables on the device before the capture; no job runs
            self.ctx[j.slot].prepare(j.ng, j.box, [p.w for p in j.params], stream=self.streams[j.slot])
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.main):
            self._enqueue(self.main)
        torch.cuda.synchronize(self.device)

    def replay(self):
        self.graph.replay()

    def check(self):
        for c in self.ctx:
            c.check()

    def close(self):
        self.graph = None
        for c in self.ctx:
            c.close()
        self.ctx = []
