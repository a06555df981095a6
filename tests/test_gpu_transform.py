"""Grid CWT on the GPU (fp32 FFT) against the fp64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_10622_gb300 import synth
from tests.gpu_util import CWT_MAX_REL, CWT_REL_L2, cwt_errors, dev, random_box, record

pytestmark = pytest.mark.gpu


def test_workload64(gctx, work64):
    wl, pos, ref = work64
    g = gctx.deposit(dev(pos), wl.box, wl.ng)
    c = gctx.transform(g, wl.box, 2.0)
    gctx.check()
    rel, mx = cwt_errors(c.cpu().numpy(), ref["cwt"])
    assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (rel, mx)


@pytest.mark.parametrize("ng", [8, 10, 12, 14, 16, 18, 20, 24, 28, 30, 32, 36, 40, 48, 50, 54, 64, 70, 72, 96, 100,
                                128, 140])
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


# Bluestein passes (Sec. 2.1's grid rule gives sizes with prime factors above
# 7): y/z length with a large prime (22 = 2 11, 190 = 2 5 19), x length ng/2
# prime (94: 47, 38: 19), both, and lengths whose TMA box overhangs the axis
@pytest.mark.parametrize("ng", [22, 26, 34, 38, 46, 58, 62, 74, 94, 110, 146, 190])
def test_bluestein_sizes(gctx, ng):
    L = 0.78125 * ng
    pos = synth.clumped_box(8 * ng ** 3 // 10, L, max(2, ng // 4), seed=ng).numpy()
    grid, _ = oracle.cic(pos, L, ng)
    for w in (2.0, 3.3):
        ref = oracle.cwt(grid, L, w)
        c = gctx.transform(dev(grid), L, w)
        gctx.check()
        rel, mx = cwt_errors(c.cpu().numpy(), ref)
        record({"config": f"Bluestein CWT, clumped {ng}^3, w={w}", "rel_l2": rel, "max_rel": mx})
        assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (ng, w, rel, mx)


@pytest.mark.parametrize("ng", [490, 1022])
def test_bluestein_large_spot_values(ng):
    # 490 = 2 5 7^2 has radix stages but no tile width that fits a TMA box and
    # 512 threads, so its y/z passes run Bluestein; 1022 = 2 7 73 runs Bluestein
    # on every axis (inner lengths 2048 and 1024)
    import paper_2501_10622_gb300 as pkg
    L, w = 0.5 * ng, 2.0
    ctx = pkg.Context(0, max_ng=ng, max_np=1 << 22, max_scales=1)
    try:
        pos = synth.clumped_box(1 << 22, L, 400, seed=ng, device="cuda")
        g = ctx.deposit(pos, L, ng)
        c = ctx.transform(g, L, w)
        ctx.check()
        grid = g.cpu().numpy()
        # random nodes and the field's twelve largest values (the clumps)
        top = torch.topk(c.reshape(-1), 12).indices.cpu().numpy()
        nodes = np.concatenate([np.random.default_rng(ng).integers(0, ng ** 3, 12), top])
        ref = oracle.cwt_at(grid, L, w, nodes)
        got = c.reshape(-1)[torch.as_tensor(nodes, device="cuda")].double().cpu().numpy()
        scale = float(c.abs().max())
        err = float(np.max(np.abs(got - ref))) / scale
        record({"config": f"Bluestein CWT spot values, clumped 2^22 on {ng}^3, w={w}", "max_rel_spot": err})
        assert err <= CWT_MAX_REL, err
    finally:
        ctx.close()
        torch.cuda.empty_cache()


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


@pytest.mark.parametrize("ng", [16, 256])
def test_stuck_copy_reports_timeout(gctx, ng):
    # Fault injection without a fault: in the next y/z pass one CTA arms its
    # transfer barrier for the tile but issues no copy, so its bounded wait runs
    # out with nothing in flight.  The call must come back as CWTHF_E_TIMEOUT,
    # and the same context must then transform correctly (16^3 takes the
    # run-time FFT plan, 256^3 a compile-time one).
    import paper_2501_10622_gb300 as pkg
    L, w = 0.78125 * ng, 2.0
    pos = synth.clumped_box(ng ** 3 // 4, L, 4, seed=ng).numpy()
    grid, _ = oracle.cic(pos, L, ng)
    g = dev(grid)
    gctx.debug_set(pkg._lib.DEBUG_TMA_NO_COPY, 1)
    gctx.transform(g, L, w)
    assert gctx.sync() == pkg._lib.E_TIMEOUT
    assert gctx.debug_get(pkg._lib.DEBUG_TMA_NO_COPY) == 0  # one-shot
    c = gctx.transform(g, L, w)
    gctx.check()
    if ng <= 64:
        rel, mx = cwt_errors(c.cpu().numpy(), oracle.cwt(grid, L, w))
        assert rel <= CWT_REL_L2 and mx <= CWT_MAX_REL, (rel, mx)
    else:
        nodes = np.random.default_rng(1).integers(0, ng ** 3, 24)
        ref = oracle.cwt_at(grid, L, w, nodes)
        got = c.cpu().numpy().reshape(-1)[nodes].astype(np.float64)
        assert np.max(np.abs(got - ref)) <= CWT_MAX_REL * np.max(np.abs(c.cpu().numpy()))


def test_every_supported_size_transforms_a_point_mass():
    # every grid size the library accepts must run its FFT plan: a unit mass on
    # one node gives the wavelet's peak 6 w^1.5 there (Eq. 4)
    import paper_2501_10622_gb300 as pkg
    sizes = pkg.supported_sizes(8, 1024)
    ctx = pkg.Context(0, max_ng=max(sizes), max_np=1, max_scales=1)
    try:
        w = 1.0
        for ng in sizes:
            g = torch.zeros((ng, ng, ng), dtype=torch.int64, device="cuda")
            g[ng // 3, ng // 2, ng // 5] = 1 << 30
            c = ctx.transform(g, float(ng), w)
            ctx.check(what=f"ng={ng}")
            assert abs(float(c[ng // 3, ng // 2, ng // 5]) - 6.0) <= 1e-4 * 6.0, ng
            del g, c
    finally:
        ctx.close()
        torch.cuda.empty_cache()
