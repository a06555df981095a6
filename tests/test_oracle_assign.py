"""Pins of the oracle's particle assignment, per-halo sums and thresholds
(Sec. 2 steps 6-7, Sec. 2.3-2.4, Table 1): hand-built label grids with
hand-computed catalogues, mass bookkeeping, a brute-force recount and
periodic centres."""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _labels_two_halos(n=4):
    """Cells x < 2 belong to seed A = cell (0,0,0); x >= 2 to seed B = cell (3,0,0)."""
    lab = np.empty((n, n, n), np.int32)
    lab[:, :, :2] = 0
    lab[:, :, 2:] = 3
    return lab


def test_hand_built_catalogue_and_thresholds():
    n, L = 4, 4.0  # cell = 1
    lab = _labels_two_halos(n)
    # 20 particles at node (0,0,0) (+1/4 cell in x on half of them), 10 at node (3,0,0)
    pos = np.array([[0.0, 0.0, 0.0]] * 10 + [[0.25, 0.0, 0.0]] * 10 + [[3.0, 0.0, 0.0]] * 10, np.float32)
    hid, cat = oracle.assign(pos, L, lab, dens_th=0.0, particle_th=15)
    # B has 10 < 15 particles and is dropped; A keeps all 20
    assert cat["seed"].tolist() == [0]
    assert cat["n_part"].tolist() == [20] and cat["n_cells"].tolist() == [32]
    assert cat["mass"].tolist() == [20.0]
    # centre of mass: 10 at x=0 and 10 at x=0.25 -> 0.125
    np.testing.assert_allclose(cat["centre"][0], [0.125, 0.0, 0.0], rtol=0, atol=1e-15)
    assert hid.tolist() == [0] * 20 + [-1] * 10
    # density: A holds 20 of 30 units of mass in 32 of 64 cells -> 20/32 / (30/64) = 4/3 mean
    hid, cat = oracle.assign(pos, L, lab, dens_th=4.0 / 3.0, particle_th=1)
    assert cat["seed"].tolist() == [0]           # exactly at the threshold is kept (>=)
    hid, cat = oracle.assign(pos, L, lab, dens_th=1.3334, particle_th=1)
    assert cat["seed"].tolist() == []


def test_nearest_node_rounds_half_up():
    n, L = 4, 4.0
    lab = _labels_two_halos(n)
    pos = np.array([[1.5, 0.0, 0.0], [1.4990234375, 0.0, 0.0]], np.float32)  # 1.5 -> node 2 (B), just below -> node 1 (A)
    hid, _ = oracle.assign(pos, L, lab, dens_th=0.0, particle_th=0)
    assert hid.tolist() == [3, 0]


def test_table1_defaults_in_wrapper():
    g = json.load(open(os.path.join(GOLD, "table1_defaults.json")))
    import inspect
    sig = inspect.signature(oracle.assign)
    assert sig.parameters["dens_th"].default == g["dens_th"]
    assert sig.parameters["particle_th"].default == g["particle_th"]


def test_centre_across_periodic_boundary():
    n, L = 8, 8.0
    lab = np.zeros((n, n, n), np.int32)  # everything belongs to seed 0 = node (0,0,0)
    pos = np.array([[7.75, 0.0, 0.0], [0.5, 0.0, 0.0]], np.float32)
    _, cat = oracle.assign(pos, L, lab, dens_th=0.0, particle_th=0)
    # offsets -0.25 and +0.5 about node 0 -> mean +0.125 (not the naive (7.75+0.5)/2)
    np.testing.assert_allclose(cat["centre"][0], [0.125, 0.0, 0.0], atol=1e-15)
    pos = np.array([[7.5, 0.0, 0.0], [7.75, 0.0, 0.0]], np.float32)
    _, cat = oracle.assign(pos, L, lab, dens_th=0.0, particle_th=0)
    np.testing.assert_allclose(cat["centre"][0], [7.625, 0.0, 0.0], atol=1e-15)  # wrapped into [0, L)


def test_mass_bookkeeping_and_bruteforce_recount():
    rng = np.random.default_rng(2)
    n, L = 12, 12.0
    pos = (rng.random((4000, 3)) * L).astype(np.float32)
    mass = (0.5 + rng.random(4000)).astype(np.float32)
    unit = 1.0 / 256
    C = rng.standard_normal((n, n, n)).astype(np.float32) + 0.2
    lab = oracle.segment(C, 0.0)
    hid, cat = oracle.assign(pos, L, lab, C, mass=mass, mass_unit=unit, dens_th=0.0, particle_th=0)
    mq = np.rint(mass.astype(np.float64) / unit).astype(np.int64)
    # every seed is kept with thresholds off; halo masses + unassigned mass = total
    seeds = np.flatnonzero(lab.ravel() == np.arange(lab.size))
    np.testing.assert_array_equal(cat["seed"], seeds)
    assert cat["mass"].sum() + mq[hid < 0].sum() * unit == pytest.approx(mq.sum() * unit, rel=1e-15)
    # brute-force recount of particles and cells per seed
    node = (np.floor(pos.astype(np.float64) * (n / L) * 1024).astype(np.int64) + 512) >> 10
    node %= n
    cell_lab = lab[node[:, 2], node[:, 1], node[:, 0]]
    np.testing.assert_array_equal(hid, cell_lab)
    for k, s in enumerate(cat["seed"]):
        assert cat["n_part"][k] == np.count_nonzero(cell_lab == s)
        assert cat["n_cells"][k] == np.count_nonzero(lab == s)
        assert cat["peak"][k] == C.ravel()[s]


def test_capacity_error_reports_count():
    n, L = 4, 4.0
    lab = _labels_two_halos(n)
    pos = np.array([[0.0, 0, 0], [3.0, 0, 0]], np.float32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.assign(pos, L, lab, dens_th=0.0, particle_th=0, cap=1)
    assert e.value.code == oracle.E_CAPACITY
