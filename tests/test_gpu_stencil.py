"""The paper's direct-space stencil CWT (Sec. 2.1, cube of radius R) on the
GPU against the oracle's literal cube sum, and against the FFT path once the
cube covers the wavelet's support."""
import numpy as np
import pytest

import oracle
import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import synth
from tests.gpu_util import CWT_MAX_REL, CWT_REL_L2, cwt_errors, dev, record

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ng,R", [(8, 0), (8, 3), (12, 2), (16, 5), (24, 6), (48, 7), (54, 11), (64, 6), (96, 5)])
def test_stencil_against_the_oracle(gctx, ng, R):
    L = 0.78125 * ng
    pos = synth.clumped_box(8 * ng ** 3 // 10, L, max(2, ng // 4), seed=ng + R).numpy()
    grid, _ = oracle.cic(pos, L, ng)
    for w in (2.0, 3.3):
        ref = oracle.cwt_stencil(grid, L, w, R)
        c = gctx.transform_stencil(dev(grid), L, w, R)
        gctx.check()
        rel, mx = cwt_errors(c.cpu().numpy(), ref)
        assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (ng, R, w, rel, mx)


def test_workload64_table1_stencil(gctx, work64):
    # the 64^3 workload at w = 2 (k_w = 0.1 at L = 50): Table 1's stencil of
    # Int(1.5 / 0.1 + 5) = 20 cells on the paper's 190^3 grid spans 5.3 Mpc/h,
    # 7 cells of this 64^3 grid
    wl, pos, _ = work64
    grid = gctx.deposit(dev(pos), wl.box, wl.ng)
    ref = oracle.cwt_stencil(grid.cpu().numpy(), wl.box, 2.0, 7)
    c = gctx.transform_stencil(grid, wl.box, 2.0, 7)
    gctx.check()
    rel, mx = cwt_errors(c.cpu().numpy(), ref)
    record({"config": "direct-space stencil, clumped 64^3, 64^3 grid, L=50, w=2, R=7", "cwt_rel_l2": rel,
            "cwt_max_rel": mx})
    assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (rel, mx)


def test_covering_stencil_equals_the_fft_path(gctx):
    ng, L, w = 32, 32.0, 2.5  # w * Delta * R = 37.5: the wavelet is zero in fp64 beyond the cube
    pos = synth.clumped_box(20000, L, 8, seed=3).numpy()
    grid = dev(oracle.cic(pos, L, ng)[0])
    a = gctx.transform_stencil(grid, L, w, 15).cpu().numpy().astype(np.float64)
    b = gctx.transform(grid, L, w).cpu().numpy().astype(np.float64)
    gctx.check()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 2 * CWT_REL_L2


def test_workload256_spot_values(gctx):
    wl = synth.WORKLOADS["clumped-256cube-L200"]
    pos = wl.positions()
    grid = gctx.deposit(dev(pos), wl.box, wl.ng)
    g = grid.cpu().numpy()
    for w, R in ((2.0, 7), (4.0, 5)):
        c = gctx.transform_stencil(grid, wl.box, w, R)
        gctx.check()
        ch = c.cpu().numpy().reshape(-1)
        rng = np.random.default_rng(int(w))
        nodes = np.unique(np.concatenate([[int(np.argmax(ch)), int(np.argmin(ch))],
                                          np.argpartition(g.reshape(-1), -8)[-8:], rng.integers(0, wl.ng ** 3, 24)]))
        ref = oracle.cwt_stencil_at(g, wl.box, w, R, nodes)
        err = np.abs(ch[nodes].astype(np.float64) - ref)
        assert np.max(err) <= CWT_MAX_REL * np.max(np.abs(ref)), (w, R, np.max(err) / np.max(np.abs(ref)))


def test_invalid_stencil_radius_rejected(gctx):
    grid = dev(np.zeros((16, 16, 16), np.int64))
    for R in (-1, 8, 65):  # 2R + 1 > ng, or beyond the maximum
        with pytest.raises(pkg.CwthfError):
            gctx.transform_stencil(grid, 10.0, 2.0, R)
