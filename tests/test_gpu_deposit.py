"""CIC deposit on the GPU against the oracle: bit-exact int64 grids."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import synth
from tests.gpu_util import dev, random_box

pytestmark = pytest.mark.gpu


def test_workload64_bit_exact(gctx, work64):
    wl, pos, ref = work64
    mt = torch.zeros(1, dtype=torch.int64, device="cuda")
    g = gctx.deposit(dev(pos), wl.box, wl.ng, mtot=mt)
    gctx.check()
    np.testing.assert_array_equal(g.cpu().numpy(), ref["grid"])
    assert int(mt) == pos.shape[0]


@pytest.mark.parametrize("ng", [8, 12, 18, 24, 36, 48, 54, 96])
def test_ragged_sizes_bit_exact(gctx, ng):
    L = 0.7 * ng
    pos = random_box(20000 + 37 * ng, L, ng)
    g = gctx.deposit(dev(pos), L, ng)
    gctx.check()
    ref, _ = oracle.cic(pos, L, ng)
    np.testing.assert_array_equal(g.cpu().numpy(), ref)


def test_clustered_cells_and_variable_masses(gctx):
    ng, L = 32, 16.0
    rng = np.random.default_rng(3)
    # a very dense core: thousands of particles inside one cell, plus a background
    core = (np.array([8.3, 8.6, 8.1]) + rng.random((6000, 3)) * 0.3).astype(np.float32)
    pos = np.concatenate([core, random_box(4000, L, 4)])
    mass = (rng.random(pos.shape[0]) * 5).astype(np.float32)
    unit = 1.0 / 512
    g = gctx.deposit(dev(pos), L, ng, mass=dev(mass), mass_unit=unit)
    gctx.check()
    ref, mt = oracle.cic(pos, L, ng, mass=mass, mass_unit=unit)
    np.testing.assert_array_equal(g.cpu().numpy(), ref)


def test_deterministic_and_order_free(gctx, work64):
    wl, pos, ref = work64
    p = dev(pos)
    a = gctx.deposit(p, wl.box, wl.ng).clone()
    b = gctx.deposit(p[torch.randperm(p.shape[0], device="cuda")], wl.box, wl.ng)
    gctx.check()
    assert torch.equal(a, b)


@pytest.mark.parametrize("masses", [False, True])
def test_dense_tiles_split_into_parts(gctx, masses):
    # cores of tens of thousands of particles in a cell or two, one at a tile
    # corner (reaching into eight tiles), so their tiles hold many more than
    # 4096 records: the first part of each is stored by the tile pass, the
    # others are added by the part pass; the grid is bit-exact all the same
    ng, L = 48, 24.0
    rng = np.random.default_rng(7)
    corner = (np.array([15.8, 3.8, 3.8]) + rng.random((150000, 3)) * 0.35).astype(np.float32)  # x 31.6-32.3 cells
    inner = (np.array([5.2, 9.1, 17.3]) + rng.random((50000, 3)) * 0.9).astype(np.float32)
    pos = np.concatenate([corner, inner, random_box(20000, L, 5)])
    # masses of 1-3 quanta: the oracle's fp64 cell sums stay below 2^53
    mass = rng.integers(1, 4, pos.shape[0]).astype(np.float32) if masses else None
    unit = 1.0
    g = gctx.deposit(dev(pos), L, ng, mass=None if mass is None else dev(mass), mass_unit=unit)
    gctx.check()
    ref, _ = oracle.cic(pos, L, ng, mass=mass, mass_unit=unit)
    np.testing.assert_array_equal(g.cpu().numpy(), ref)


def test_empty_particle_set(gctx):
    g = gctx.deposit(torch.zeros((0, 3), dtype=torch.float32, device="cuda"), 10.0, 16)
    gctx.check()
    assert int(g.abs().sum()) == 0


def test_bad_inputs_reported(gctx):
    pos = random_box(1000, 10.0, 1)
    pos[17, 1] = np.nan
    gctx.deposit(dev(pos), 10.0, 16)
    assert gctx.sync() == pkg._lib.E_BAD_INPUT
    pos = random_box(1000, 10.0, 1)
    mass = np.ones(1000, np.float32)
    mass[5] = 3e9  # m_q >= 2^31 with mass_unit 1
    gctx.deposit(dev(pos), 10.0, 16, mass=dev(mass))
    assert gctx.sync() == pkg._lib.E_OVERFLOW
    mass = np.full(1000, 2.0 ** 31 - 256, np.float32)  # sum m_q >= 2^33
    gctx.deposit(dev(pos), 10.0, 16, mass=dev(mass))
    assert gctx.sync() == pkg._lib.E_OVERFLOW
    mass = np.ones(1000, np.float32)
    mass[3] = -1.0
    gctx.deposit(dev(pos), 10.0, 16, mass=dev(mass))
    assert gctx.sync() == pkg._lib.E_BAD_INPUT
    assert gctx.sync() == 0  # the status clears after being read


def test_host_side_argument_errors(gctx):
    p = dev(random_box(10, 10.0, 1))
    with pytest.raises(pkg.CwthfError) as e:  # odd: the real transform pairs the x samples
        gctx.deposit(p, 10.0, 101)
    assert e.value.code == pkg._lib.E_UNSUPPORTED_SIZE
    with pytest.raises(pkg.CwthfError) as e:
        gctx.deposit(p, -1.0, 16)
    assert e.value.code == pkg._lib.E_INVALID_ARG
    with pytest.raises(pkg.CwthfError):
        gctx.deposit(p, 10.0, 16, mass_unit=0.0)


def test_workload256_bit_exact(gctx):
    wl = synth.WORKLOADS["clumped-256cube-L200"]
    pos = wl.positions("cuda")
    g = gctx.deposit(pos, wl.box, wl.ng)
    gctx.check()
    ref, mt = oracle.cic(pos.cpu().numpy(), wl.box, wl.ng)
    assert mt == pos.shape[0]
    np.testing.assert_array_equal(g.cpu().numpy(), ref)
