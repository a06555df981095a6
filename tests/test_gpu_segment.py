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
