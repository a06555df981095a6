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


def test_fft_plan_overrides_keep_results_within_rounding():
    # a tuned plan changes only the fp32 rounding of the transform: a plan the
    # kernels cannot run is refused, an accepted one transforms within the
    # CWT bars of the oracle, and clearing it restores the built-in plan
    import numpy as np

    import oracle
    from tests.gpu_util import CWT_MAX_REL, CWT_REL_L2, cwt_errors
    ng, L = 96, 75.0
    pos = synth.clumped_box(60000, L, 20, seed=5).numpy()
    grid, _ = oracle.cic(pos, L, ng)
    ref = oracle.cwt(grid, L, 2.0)
    g = torch.as_tensor(grid).cuda()
    ctx = pkg.Context(0, max_ng=ng, max_np=1, max_scales=1)
    try:
        base = ctx.transform(g, L, 2.0).clone()
        assert not ctx.set_fft_plan(ng, 0, 8, (5, 19))  # product 95
        assert not ctx.set_fft_plan(ng, 0, 16, (96,))   # 96 is no radix
        for which, c, rad in ((0, 4, (12, 8)), (0, 16, (4, 24)), (1, 8, (6, 8)), (1, 2, (3, 16))):
            assert ctx.set_fft_plan(ng, which, c, rad), (which, c, rad)
            out = ctx.transform(g, L, 2.0)
            ctx.check()
            rel, mx = cwt_errors(out.cpu().numpy(), ref)
            assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (which, c, rad, rel, mx)
        ctx.set_fft_plan(ng, 0)
        ctx.set_fft_plan(ng, 1)
        assert torch.equal(ctx.transform(g, L, 2.0), base)
    finally:
        ctx.close()


def test_autotune_picks_runnable_plans_and_the_batch_applies_them(tmp_path):
    from paper_2501_10622_gb300 import autotune
    plans = autotune.tune(0, [32, 48], reps=2, path=tmp_path / "plans.json")
    assert set(plans) == {32, 48} and autotune.load(tmp_path / "plans.json") == plans
    subs = synth.batched_subvolumes(n_jobs=6, seed=9, grids=(32, 48), np_range=(1e4, 5e4))
    jobs = [batch.BatchJob(w.positions("cuda"), w.box, w.ng, [pkg.default_params(2.0)]) for w in subs]
    b = batch.Batch(jobs, n_slots=2, fft_plans=plans)
    try:
        b.capture()
        b.replay()
        torch.cuda.synchronize()
        b.check()
        assert all(int(j.n_halo[0]) >= 0 for j in jobs)
    finally:
        b.close()
