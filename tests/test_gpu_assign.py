"""Particle assignment and catalogue on the GPU: exact against the oracle for
the same labels (every per-halo sum is an integer, centres use the same fp64
operations)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10622_gb300 as pkg
from tests.gpu_util import dev, random_box

pytestmark = pytest.mark.gpu


def _compare(gctx, pos, L, lab, C, mass=None, unit=1.0, dens_th=4.0, pth=15, cap=None):
    hid, cat, nh = gctx.assign(dev(pos), L, dev(lab), dev(C), mass=None if mass is None else dev(mass),
                               mass_unit=unit, dens_th=dens_th, particle_th=pth, cat_cap=cap)
    rc = gctx.sync()
    rhid, rcat = oracle.assign(pos, L, lab, C, mass=mass, mass_unit=unit, dens_th=dens_th, particle_th=pth)
    n = int(nh)
    assert n == len(rcat["seed"])
    np.testing.assert_array_equal(hid.cpu().numpy(), rhid)
    got = pkg.catalogue_to_numpy(cat, min(n, cat.shape[0]))
    m = len(got)
    np.testing.assert_array_equal(got["seed"], rcat["seed"][:m])
    np.testing.assert_array_equal(got["n_part"], rcat["n_part"][:m])
    np.testing.assert_array_equal(got["n_cells"], rcat["n_cells"][:m])
    np.testing.assert_array_equal(got["mass"], rcat["mass"][:m])
    np.testing.assert_array_equal(got["centre"], rcat["centre"][:m])
    np.testing.assert_array_equal(got["peak"], rcat["peak"][:m])
    return rc, n


def test_workload64(gctx, work64):
    wl, pos, ref = work64
    rc, n = _compare(gctx, pos.numpy(), wl.box, ref["label"], ref["cwt32"])
    assert rc == 0 and n == len(ref["cat"]["seed"]) > 10


@pytest.mark.parametrize("dens_th,pth", [(0.0, 0), (0.0, 15), (4.0, 1), (40.0, 15)])
def test_thresholds(gctx, work64, dens_th, pth):
    wl, pos, ref = work64
    rc, _ = _compare(gctx, pos.numpy(), wl.box, ref["label"], ref["cwt32"], dens_th=dens_th, pth=pth)
    assert rc == 0


def test_variable_masses_and_boundary_wrap(gctx):
    rng = np.random.default_rng(5)
    ng, L = 24, 12.0
    pos = random_box(30000, L, 9)
    mass = (rng.random(30000) * 3 + 0.01).astype(np.float32)
    C = (rng.standard_normal((ng, ng, ng)) + 0.3).astype(np.float32)
    lab = oracle.segment(C)
    rc, _ = _compare(gctx, pos, L, lab, C, mass=mass, unit=1.0 / 300, dens_th=0.5, pth=3)
    assert rc == 0


def test_capacity_reported(gctx, work64):
    wl, pos, ref = work64
    rc, n = _compare(gctx, pos.numpy(), wl.box, ref["label"], ref["cwt32"], dens_th=0.0, pth=0, cap=7)
    assert rc == pkg._lib.E_CAPACITY and n > 7


def test_workload256_on_the_gpu_field(gctx):
    # at the 256^3 workload the oracle segments the GPU's own fp32 CWT field:
    # labels bit for bit, then the assignment and catalogue element by element
    from paper_2501_10622_gb300 import synth
    wl = synth.WORKLOADS["clumped-256cube-L200"]
    pos = wl.positions().numpy()
    c = gctx.transform(gctx.deposit(dev(pos), wl.box, wl.ng), wl.box, 2.0)
    lab = gctx.segment(c)
    gctx.check()
    C = c.cpu().numpy()
    ref_lab = oracle.segment(C)
    np.testing.assert_array_equal(lab.cpu().numpy(), ref_lab)
    seeds, n_cells, ns = gctx.segment_sizes(1 << 22)
    want_seeds, want_cells = np.unique(ref_lab[ref_lab >= 0], return_counts=True)
    assert ns == len(want_seeds)
    np.testing.assert_array_equal(seeds.cpu().numpy(), want_seeds)
    np.testing.assert_array_equal(n_cells.cpu().numpy(), want_cells)
    rc, n = _compare(gctx, pos, wl.box, ref_lab, C, cap=1 << 20)
    assert rc == 0 and n > 1000
