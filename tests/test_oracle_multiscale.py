"""Pins of the oracle's multi-scale loop (Sec. 2, Fig. 1; App. B; Sec. 2.4)."""
import numpy as np
import pytest

import oracle
from paper_2501_10622_gb300 import synth


def _quadratic(ng, centre, c=50.0, a=0.8):
    z, y, x = np.meshgrid(*(np.arange(ng),) * 3, indexing="ij")
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return (c - a * r2).astype(np.float32), c, a


@pytest.mark.parametrize("off", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.45), (-0.49, 0.1, -0.33)])
def test_b1_recovers_the_peak_of_a_sampled_quadratic(off):
    # Eq. B1 fits the quadratic through a maximum node and its two neighbours
    # per axis: for a field that is exactly quadratic the corrected value is
    # the true peak c, wherever the peak sits within the node's cell
    ng = 16
    centre = (8 + off[0], 7 + off[1], 9 + off[2])
    C, c, a = _quadratic(ng, centre)
    seed = (9 * ng + 7) * ng + 8
    assert oracle.parent(C).reshape(-1)[seed] == seed
    assert abs(oracle.corrected_peak(C, seed) - c) <= 2e-5 * c


@pytest.mark.parametrize("ng,ng_next", [(16, 24), (16, 32), (24, 27)])
def test_grid_size_term_against_the_analytic_quadratic(ng, ng_next):
    # App. B: with the factor 3/5 removed, the larger grid's peak is raised by
    # (5/2) (c - f(Delta/2)) (1 - (Delta_next/Delta)^2) for a quadratic f:
    # c - f(Delta/2) = a / 4 in this grid's cell units
    C, c, a = _quadratic(ng, (8.0, 7.0, 9.0))
    seed = (9 * ng + 7) * ng + 8
    r = ng / ng_next
    want = c + 2.5 * (a / 4.0) * (1.0 - r * r)
    assert abs(oracle.corrected_peak(C, seed, ng_next) - want) <= 2e-5 * c


def test_cross_scale_enclosing_nodes():
    ng, ngn = 8, 12
    C = np.zeros((ng, ng, ng), np.float32)
    C[3, 2, 5] = 10.0  # seed at x=5, y=2, z=3 -> position (7.5, 3, 4.5) in next-grid cells
    seed = (3 * ng + 2) * ng + 5
    Cn = np.zeros((ngn, ngn, ngn), np.float32)
    assert oracle.cross_scale(C, seed, Cn)
    assert oracle.cross_scale(C, seed, None)  # the last scale: against a zero field
    # a higher value at one of the 8 enclosing nodes (x 7-8, y 3-4, z 4-5) defeats it ...
    big = oracle.corrected_peak(C, seed, ngn) + 1.0
    for x, y, z in [(7, 3, 4), (8, 4, 5), (8, 3, 5)]:
        Cn2 = Cn.copy()
        Cn2[z, y, x] = big
        assert not oracle.cross_scale(C, seed, Cn2)
    # ... one just outside them does not
    for x, y, z in [(6, 3, 4), (9, 3, 4), (7, 5, 4), (7, 3, 6)]:
        Cn2 = Cn.copy()
        Cn2[z, y, x] = big
        assert oracle.cross_scale(C, seed, Cn2)
    # a maximum below zero fails against the zero field of the last scale
    assert not oracle.cross_scale(-C, seed, None)


def test_one_scale_reduces_to_the_single_scale_oracle():
    # with one scale, the cross-scale check is against a zero field, which every
    # seed above cwt_min = 0 passes: the loop is the single-scale path, with
    # halo ids renumbered in seed order
    wl = synth.WORKLOADS["clumped-64cube-L50"]
    pos = wl.positions().numpy()
    ref = oracle.find(pos, wl.box, wl.ng, 2.0)
    hid, cat = oracle.multiscale_on_fields(pos, wl.box, [ref["cwt32"]])
    np.testing.assert_array_equal(cat["seed"], ref["cat"]["seed"])
    np.testing.assert_array_equal(cat["n_part"], ref["cat"]["n_part"])
    np.testing.assert_array_equal(cat["n_cells"], ref["cat"]["n_cells"])
    np.testing.assert_array_equal(cat["centre"], ref["cat"]["centre"])
    back = np.where(hid >= 0, cat["seed"][np.maximum(hid, 0)], -1)
    np.testing.assert_array_equal(back, ref["halo_id"])


def test_ids_are_kept_and_every_halo_is_consistent():
    # three scales on the 48^3 box: a particle keeps the first id it gets, every
    # catalogue count matches the ids, and the halos of a later scale are
    # built from particles no earlier halo took
    L = 37.5
    pos = synth.clumped_box(48 ** 3, L, 84, seed=11).numpy()
    ws, ngs = [2.0, 3.0, 4.0], [32, 48, 64]
    out = oracle.find_multiscale(pos, L, ws, ngs)
    hid, cat = out["halo_id"], out["cat"]
    assert len(cat["seed"]) > 0 and set(cat["scale"].tolist()) <= {0, 1, 2}
    ids, counts = np.unique(hid[hid >= 0], return_counts=True)
    np.testing.assert_array_equal(ids, np.arange(len(cat["seed"]))[cat["n_part"] > 0])
    np.testing.assert_array_equal(counts, cat["n_part"][cat["n_part"] > 0])
    assert np.all(np.diff(cat["scale"]) >= 0)  # ids follow the processing order
    # the first scale alone (its own cross-scale check against scale 1) gives
    # exactly the first scale's halos: later scales never take their particles
    h1, c1 = oracle.multiscale_on_fields(pos, L, out["fields"][:2])
    first = cat["scale"] == 0
    np.testing.assert_array_equal(c1["seed"][c1["scale"] == 0], cat["seed"][first])
    n1 = int(first.sum())
    in1 = (h1 >= 0) & (h1 < n1)
    np.testing.assert_array_equal(in1, (hid >= 0) & (hid < n1))
    np.testing.assert_array_equal(h1[in1], hid[in1])


def _box_with_velocities(n=24000, L=40.0, seed=2):
    from paper_2501_10622_gb300 import synth
    pos, vel = synth.clumped_box(n, L, 40, seed=seed, velocities=True)
    return pos.numpy(), vel.numpy(), synth.particle_mass(n, L)


def test_self_boundness_in_the_loop_zero_velocities_change_nothing():
    # no relative motion: every member is bound (0 > v_esc^2 never holds), so
    # the loop with the check equals the loop without it
    pos, vel, mp = _box_with_velocities()
    ws, ngs = [1.5, 2.5], [24, 36]
    a = oracle.find_multiscale(pos, 40.0, ws, ngs, mass_unit=mp)
    b = oracle.find_multiscale(pos, 40.0, ws, ngs, mass_unit=mp, vel=np.zeros_like(vel))
    np.testing.assert_array_equal(a["halo_id"], b["halo_id"])
    for col in ("seed", "n_part", "mass", "centre", "scale"):
        np.testing.assert_array_equal(a["cat"][col], b["cat"][col])
    assert len(a["cat"]["seed"]) > 0


def test_self_boundness_in_the_loop_no_gravity_discards_everything():
    # G = 0: every member moving relative to its group's mean velocity is
    # unbound, so every group loses more than 40 % and is discarded
    pos, vel, mp = _box_with_velocities()
    r = oracle.find_multiscale(pos, 40.0, [1.5, 2.5], [24, 36], mass_unit=mp, vel=vel, G=0.0)
    assert len(r["cat"]["seed"]) == 0 and (r["halo_id"] < 0).all()


def test_self_boundness_in_the_loop_halos_are_bound_and_consistent():
    pos, vel, mp = _box_with_velocities()
    L = 40.0
    r = oracle.find_multiscale(pos, L, [1.5, 2.5, 3.5], [24, 36, 48], mass_unit=mp, vel=vel)
    hid, cat = r["halo_id"], r["cat"]
    n = len(cat["seed"])
    assert n > 0 and r["cat"]["margin"] > 1e-9
    # the catalogue describes exactly the particles holding each id
    np.testing.assert_array_equal(np.bincount(hid[hid >= 0], minlength=n), cat["n_part"])
    np.testing.assert_allclose(cat["mass"], cat["n_part"] * mp, rtol=1e-12)
    # every final halo is bound: one more check of its members excludes no one
    out, nk, it, _ = oracle.unbind(pos, vel, hid, L, G=oracle.G_MPC_KMS_MSUN, mass_unit=mp, n_groups=n)
    np.testing.assert_array_equal(nk, cat["n_part"])
    assert (it == 1).all()
    # and the check changed the outcome against the loop without it
    plain = oracle.find_multiscale(pos, L, [1.5, 2.5, 3.5], [24, 36, 48], mass_unit=mp)
    assert not np.array_equal(plain["halo_id"], hid)
