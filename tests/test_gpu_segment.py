"""Maxima and steepest-ascent labels on the GPU: bit-exact against the oracle
when both segment the same fp32 field."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10622_gb300 as pkg
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def _check(gctx, C, cwt_min=0.0):
    lab = gctx.segment(dev(C), cwt_min)
    gctx.check()
    ref = oracle.segment(C, cwt_min)
    np.testing.assert_array_equal(lab.cpu().numpy(), ref)


def test_workload64_oracle_field(gctx, work64):
    _, _, ref = work64
    _check(gctx, ref["cwt32"])
    _check(gctx, ref["cwt32"], cwt_min=50.0)


@pytest.mark.parametrize("ng", [8, 12, 18, 24, 36, 48, 54, 72, 96])
def test_random_fields_with_plateaus(gctx, ng):
    rng = np.random.default_rng(ng)
    C = rng.standard_normal((ng, ng, ng)).astype(np.float32)
    C[rng.random(C.shape) < 0.15] = 0.25  # ties resolved by the index order
    C[rng.random(C.shape) < 0.02] = -0.0
    _check(gctx, C)
    _check(gctx, np.round(C * 4) / 4)  # heavy plateaus
    _check(gctx, rng.integers(0, 3, C.shape).astype(np.float32))  # three levels: ties everywhere


def test_constant_field_single_seed(gctx):
    _check(gctx, np.ones((16, 16, 16), np.float32))
    _check(gctx, np.ones((16, 16, 16), np.float32), cwt_min=2.0)


def test_long_chains_cross_many_tiles(gctx):
    # one broad bump over a 96^3 box: chains run up to ~48 cells across tile borders
    n = 96
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    d2 = (np.minimum(x, n - x) ** 2 + np.minimum(y - 40, n - abs(y - 40)) ** 2 +
          np.minimum(abs(z - 70), n - abs(z - 70)) ** 2).astype(np.float64)
    C = np.exp(-d2 / (2 * 30.0 ** 2)).astype(np.float32)
    _check(gctx, C)
    # plus a ripple that creates many small basins
    C2 = (C + 0.02 * np.sin(x * 0.9) * np.cos(y * 0.7) * np.sin(z * 1.3)).astype(np.float32)
    _check(gctx, C2)


def test_nan_reported(gctx):
    C = np.zeros((16, 16, 16), np.float32)
    C[3, 4, 5] = np.nan
    gctx.segment(dev(C))
    assert gctx.sync() == pkg._lib.E_BAD_INPUT


def _zigzag_field(n=128, seed=21):
    """Three ascent chains that cross a chain-tile face at almost every step
    (tiles are 64 x 16 x 16 cells along x, y, z), each hundreds of hops long,
    over a random background: chain A snakes along x over three z-planes with
    y alternating 15/16, chain B runs along x with z alternating 31/32, chain
    C runs along y with x alternating 63/64.  The values rise along each chain
    and stay clear of the periodic wrap, so the strict-order parent of every
    chain cell is the next chain cell (or a cell further along)."""
    rng = np.random.default_rng(seed)
    C = rng.random((n, n, n)).astype(np.float32)
    a = []
    for p, z in enumerate((4, 6, 8)):
        xs = range(1, n - 1) if p % 2 == 0 else range(n - 2, 0, -1)
        a += [(x, z) for x in xs]
        if p < 2:
            a.append((a[-1][0], z + 1))
    for t, (x, z) in enumerate(a):
        C[z, 15 + (t & 1), x] = 100.0 + 0.5 * t
    for t, x in enumerate(range(1, n - 1)):
        C[31 + (t & 1), 40, x] = 300.0 + 0.5 * t
        C[80, x, 63 + (t & 1)] = 500.0 + 0.5 * t
    return C


def _zigzag_chain_ends(n=128):
    """(first cell, last cell) of the three chains of _zigzag_field."""
    idx = lambda z, y, x: (z * n + y) * n + x
    la = 3 * (n - 2) + 2
    t = n - 3
    return [(idx(4, 15, 1), idx(8, 15 + ((la - 1) & 1), n - 2)),
            (idx(31, 40, 1), idx(31 + (t & 1), 40, n - 2)),
            (idx(80, 1, 63), idx(80, n - 2, 63 + (t & 1)))]


def _sizes_match_oracle(gctx, ref):
    seeds, n_cells, n = gctx.segment_sizes(ref.size // 8 + 8)
    want_seeds, want_cells = np.unique(ref[ref >= 0], return_counts=True)
    assert n == len(want_seeds)
    np.testing.assert_array_equal(seeds.cpu().numpy(), want_seeds)
    np.testing.assert_array_equal(n_cells.cpu().numpy(), want_cells)


def test_zigzag_chains_take_the_fallback(gctx):
    # chains of ~380 tile hops outlive the resolve pass's 64-step walks, so the
    # pointer-doubling rounds and the recount run; labels and segment sizes must
    # still equal the oracle's
    C = _zigzag_field()
    lab = gctx.segment(dev(C))
    gctx.check()
    assert gctx.debug_get(pkg._lib.DEBUG_FALLBACK_RAN) == 1
    ref = oracle.segment(C)
    np.testing.assert_array_equal(lab.cpu().numpy(), ref)
    _sizes_match_oracle(gctx, ref)
    # each chain's first cell belongs to the seed at the chain's far end
    flat = ref.reshape(-1)
    for first, last in _zigzag_chain_ends():
        assert flat[first] == last and flat[last] == last


@pytest.mark.parametrize("limit", [1, 3])
def test_short_walks_finish_in_the_fallback(gctx, limit):
    # with the bounded walks cut to 1 or 3 steps, ordinary fields need the
    # doubling rounds too: bit-exact all the same
    rng = np.random.default_rng(limit)
    fields = [rng.standard_normal((72, 72, 72)).astype(np.float32), _zigzag_field(96, seed=limit)]
    try:
        gctx.debug_set(pkg._lib.DEBUG_CHASE_LIMIT, limit)
        for C in fields:
            lab = gctx.segment(dev(C))
            gctx.check()
            assert gctx.debug_get(pkg._lib.DEBUG_FALLBACK_RAN) == 1
            ref = oracle.segment(C)
            np.testing.assert_array_equal(lab.cpu().numpy(), ref)
            _sizes_match_oracle(gctx, ref)
    finally:
        gctx.debug_set(pkg._lib.DEBUG_CHASE_LIMIT, 64)


def test_round_limit_reports_not_converged(gctx):
    # no doubling rounds allowed and one-step walks: the long chains cannot
    # finish, which must come back as CWTHF_E_NOT_CONVERGED (no fault, no hang);
    # the context then works normally again
    C = _zigzag_field()
    try:
        gctx.debug_set(pkg._lib.DEBUG_JUMP_ROUNDS, 0)
        gctx.debug_set(pkg._lib.DEBUG_CHASE_LIMIT, 1)
        gctx.segment(dev(C))
        assert gctx.sync() == pkg._lib.E_NOT_CONVERGED
    finally:
        gctx.debug_set(pkg._lib.DEBUG_JUMP_ROUNDS, 31)
        gctx.debug_set(pkg._lib.DEBUG_CHASE_LIMIT, 64)
    lab = gctx.segment(dev(C))
    gctx.check()
    np.testing.assert_array_equal(lab.cpu().numpy(), oracle.segment(C))


def test_debug_settings_reject_out_of_range(gctx):
    for key, bad in [(pkg._lib.DEBUG_JUMP_ROUNDS, 32), (pkg._lib.DEBUG_JUMP_ROUNDS, -1),
                     (pkg._lib.DEBUG_CHASE_LIMIT, 0), (pkg._lib.DEBUG_CHASE_LIMIT, 65), (99, 1)]:
        with pytest.raises(pkg.CwthfError):
            gctx.debug_set(key, bad)
    assert gctx.debug_get(pkg._lib.DEBUG_JUMP_ROUNDS) == 31
    assert gctx.debug_get(pkg._lib.DEBUG_CHASE_LIMIT) == 64
