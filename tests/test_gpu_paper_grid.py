"""The paper's largest grid: Int(400 * 2.5 + 150) = 1150 = 2 5^2 23 (Bluestein
passes along every axis) and the radix size 1152, above 2^30 cells.  The
deposit bit for bit against the oracle's whole grid, Eq. 2 at sampled nodes,
and the segmentation's defining properties at sampled nodes (flagged chains
across tiles included)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import synth
from tests.gpu_util import CWT_MAX_REL, record
from tests.test_gpu_fullsize import _strict_parent

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ng", [1150, 1152])
def test_largest_paper_grid(ng):
    L, w, n = 50.0, 50.0, 1 << 22  # k_w = 2.5: w = 2.5 * 1000 / L
    ctx = pkg.Context(0, max_ng=ng, max_np=n, max_scales=1)
    try:
        pos = synth.clumped_box(n, L, 200, seed=ng, device="cuda")
        g = ctx.deposit(pos, L, ng)
        ctx.check()
        grid = g.cpu().numpy()
        ref, _ = oracle.cic(pos.cpu().numpy(), L, ng)
        assert np.array_equal(grid, ref)
        del ref
        c = ctx.transform(g, L, w)
        ctx.check()
        del g
        top = torch.topk(c.reshape(-1), 12).indices.cpu().numpy()
        nodes = np.concatenate([np.random.default_rng(ng).integers(0, ng ** 3, 12), top])
        cref = oracle.cwt_at(grid, L, w, nodes)
        got = c.reshape(-1)[torch.as_tensor(nodes, device="cuda")].double().cpu().numpy()
        err = float(np.max(np.abs(got - cref))) / float(c.abs().max())
        del grid
        lab = ctx.segment(c, 0.0)
        ctx.check()
        C = c.cpu().numpy()
        del c
        Lb = lab.cpu().numpy().reshape(-1)
        del lab
        torch.cuda.empty_cache()
        samp = np.random.default_rng(ng + 1).integers(0, ng ** 3, 300_000)
        par = _strict_parent(C, samp)
        is_max = par == samp
        val = C.reshape(-1)[samp]
        assert np.all(Lb[samp[is_max]] == np.where(val[is_max] > 0.0, samp[is_max], -1))
        assert np.all(Lb[samp[~is_max]] == Lb[par[~is_max]])
        seeds = np.unique(Lb[samp][Lb[samp] >= 0])
        assert len(seeds) > 0 and np.all(Lb[seeds] == seeds)
        assert np.all(_strict_parent(C, seeds) == seeds) and np.all(C.reshape(-1)[seeds] > 0.0)
        assert Lb.min() >= -1  # no pointer is left flagged
        record({"config": f"paper's largest grid {ng}^3 (2^22 clumped particles, L={L}, w={w:g})",
                "deposit": "bit-exact", "cwt_max_rel_spot": err, "segmentation_sampled_nodes": len(samp)})
        assert err <= CWT_MAX_REL, err
    finally:
        ctx.close()
        torch.cuda.empty_cache()
