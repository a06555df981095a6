"""Grid CWT on the GPU (fp32 FFT) against the fp64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_10622_gb300 import synth
from tests.gpu_util import CWT_MAX_REL, CWT_REL_L2, cwt_errors, dev, random_box

pytestmark = pytest.mark.gpu


def test_workload64(gctx, work64):
    wl, pos, ref = work64
    g = gctx.deposit(dev(pos), wl.box, wl.ng)
    c = gctx.transform(g, wl.box, 2.0)
    gctx.check()
    rel, mx = cwt_errors(c.cpu().numpy(), ref["cwt"])
    assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (rel, mx)


@pytest.mark.parametrize("ng", [8, 12, 16, 18, 24, 32, 36, 48, 54, 64, 72, 96, 128])
def test_sizes(gctx, ng):
    L = 0.78125 * ng
    pos = synth.clumped_box(8 * ng ** 3 // 10, L, max(2, ng // 4), seed=ng).numpy()
    grid, _ = oracle.cic(pos, L, ng)
    for w in (2.0, 3.3):
        ref = oracle.cwt(grid, L, w)
        c = gctx.transform(dev(grid), L, w)
        gctx.check()
        rel, mx = cwt_errors(c.cpu().numpy(), ref)
        assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (ng, w, rel, mx)


def test_point_mass_kernel_and_variable_unit(gctx):
    ng, L, w = 32, 20.0, 1.3
    pos = np.array([[5.0, 7.5, 10.0]], np.float32)
    grid, _ = oracle.cic(pos, L, ng)
    ref = oracle.cwt(grid, L, w, mass_unit=2.5)
    c = gctx.transform(dev(grid), L, w, mass_unit=2.5)
    gctx.check()
    rel, mx = cwt_errors(c.cpu().numpy(), ref)
    assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL


def test_workload256(gctx):
    wl = synth.WORKLOADS["clumped-256cube-L200"]
    pos = wl.positions("cuda")
    g = gctx.deposit(pos, wl.box, wl.ng)
    c = gctx.transform(g, wl.box, 2.0)
    gctx.check()
    grid = g.cpu().numpy()
    ref_grid, _ = oracle.cic(pos.cpu().numpy(), wl.box, wl.ng)
    assert np.array_equal(grid, ref_grid)
    ref = oracle.cwt(ref_grid, wl.box, 2.0)
    rel, mx = cwt_errors(c.cpu().numpy(), ref)
    print(f"256^3 CWT rel-L2 {rel:.3e} max-rel {mx:.3e}")
    assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL
