"""Batched form: a batch of uneven subvolumes captured into one CUDA graph
gives each job exactly the result of a single cwthf_find call."""
import pytest
import torch

import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import batch, synth

pytestmark = pytest.mark.gpu


def test_graph_batch_equals_single_calls():
    subs = synth.batched_subvolumes(n_jobs=10, seed=7, grids=(32, 48, 64, 96), np_range=(1e4, 2e5))
    jobs = [batch.BatchJob(w.positions("cuda"), w.box, w.ng, [pkg.default_params(2.0)]) for w in subs]
    b = batch.Batch(jobs, n_slots=3)
    try:
        b.capture()
        for j in jobs:
            j.halo_id.fill_(-7)
            j.n_halo.fill_(-7)
        b.replay()
        b.replay()  # replaying twice gives the same results
        torch.cuda.synchronize()
        b.check()
        ctx = pkg.Context(0, max_ng=96, max_np=max(j.np for j in jobs), max_scales=1)
        for j in jobs:
            hid, cat, nh = ctx.find(j.pos, j.box, j.ng, j.params)
            ctx.check()
            assert int(nh[0]) == int(j.n_halo[0])
            assert torch.equal(hid[0], j.halo_id[0])
        ctx.close()
    finally:
        b.close()
