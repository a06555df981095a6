"""Pins of the oracle's self-boundness check (Sec. 2.3) against closed forms:
two bodies, a central mass with massless test particles (escape speed
sqrt(2 G M / r)), the 40 % rule at its boundary, recentring between rounds,
the round limit, the periodic wrap and the order of the particles."""
import math

import numpy as np
import pytest

import oracle

L = 100.0


def _run(pos, vel, mass, group=None, G=1.0, **kw):
    pos = np.asarray(pos, np.float32)
    vel = np.asarray(vel, np.float32)
    mass = None if mass is None else np.asarray(mass, np.float32)
    if group is None:
        group = np.zeros(len(pos), np.int32)
    return oracle.unbind(pos, vel, np.asarray(group, np.int32), L, G=G, mass=mass, **kw)


def test_two_bodies_escape_speed():
    # masses 3 and 1 at distance 4: the centre of mass splits it 1 : 3, so
    # r_A = 1, r_B = 3 and each feels the other's shell at max(r_A, r_B) = 3:
    # v_esc,A^2 = 2 G m_B / 3, v_esc,B^2 = 2 G m_A / 3 (G = 1), speeds
    # measured from the mass-weighted mean velocity
    pos = [[50, 50, 50], [54, 50, 50]]
    mass = [3.0, 1.0]
    for vb, removed in ((0.999 * math.sqrt(2.0 * 3.0 / 3.0), False), (1.001 * math.sqrt(2.0 * 3.0 / 3.0), True)):
        # B moves at vb, A at -vb / 3: the mean velocity is 0, and A stays below
        # its own escape speed sqrt(2/3) for vb < sqrt(6)
        vel = [[-vb / 3.0, 0, 0], [vb, 0, 0]]
        out, n, it, _ = _run(pos, vel, mass)
        if removed:  # B leaves (1 of 2 = 50 % > 40 %): the group is discarded
            assert list(out) == [-1, -1] and n[0] == 0 and it[0] == 2
        else:
            assert list(out) == [0, 0] and n[0] == 2 and it[0] == 1


def test_central_mass_and_test_particles():
    # a unit mass at rest and massless particles at radii r with speeds
    # (1 +- 1e-3) sqrt(2 G M / r): exactly the fast ones leave; the centre and
    # the mean velocity are the central mass's (the others weigh nothing)
    G, M = 2.5, 1.0
    rng = np.random.default_rng(4)
    n = 40
    r = rng.uniform(0.5, 5.0, n)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    fast = rng.random(n) < 0.3
    speed = np.sqrt(2.0 * G * M / r) * np.where(fast, 1.001, 0.999)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    c = np.array([30.0, 40.0, 50.0])
    pos = np.vstack([c, c + r[:, None] * d])
    vel = np.vstack([np.zeros(3), speed[:, None] * u])
    mass = np.concatenate([[M], np.zeros(n)])
    out, nk, it, margin = _run(pos, vel, mass, G=G)
    # float32 positions shift r by ~1e-6 relative: far inside the 1e-3 margin
    assert margin > 5e-4
    assert out[0] == 0 and np.array_equal(out[1:] == 0, ~fast)
    assert nk[0] == 1 + n - fast.sum() and it[0] == 2


@pytest.mark.parametrize("n_fast,kept", [(2, True), (3, False)])
def test_forty_percent_rule(n_fast, kept):
    # five particles (a unit mass and four massless ones at radius 1, G = 1,
    # v_esc = sqrt 2): 2 of 5 leaving is 40 % (kept), 3 of 5 is 60 % (discarded)
    pos = [[50, 50, 50], [51, 50, 50], [49, 50, 50], [50, 51, 50], [50, 49, 50]]
    vel = [[0, 0, 0]] + [[0, 0, 1.5 if k < n_fast else 1.2] for k in range(4)]
    out, n, _, _ = _run(pos, vel, [1, 0, 0, 0, 0])
    if kept:
        assert list(out) == [0, -1, -1, 0, 0] and n[0] == 3
    else:
        assert list(out) == [-1] * 5 and n[0] == 0


def test_recentring_between_rounds():
    # G = 1.  M (mass 10, at rest, x = 0), H (mass 1, x = 1, speed 16) and a
    # massless T (x = -2, speed 16/11 + 3 along x).  Round 1: centre 1/11,
    # mean velocity 16/11; H (relative speed 160/11, above sqrt(2*10/(10/11)) =
    # sqrt 22) leaves, M (16/11, below sqrt 2.2) and T (3, below
    # sqrt(2 * 11 / (23/11)) = 3.24) stay.  Round 2: centre M, mean velocity 0,
    # T (speed 4.45 above sqrt(2 * 10 / 2) = 3.16) leaves.  Round 3: nothing.
    # 2 of 3 left: discarded.  With one round only, T stays (1 of 3 left).
    vb1 = 16.0 / 11.0
    pos = [[50, 50, 50], [51, 50, 50], [48, 50, 50]]
    vel = [[0, 0, 0], [16.0, 0, 0], [vb1 + 3.0, 0, 0]]
    mass = [10.0, 1.0, 0.0]
    out, n, it, margin = _run(pos, vel, mass)
    assert list(out) == [-1, -1, -1] and n[0] == 0 and it[0] == 3 and margin > 0.02
    out, n, it, _ = _run(pos, vel, mass, max_iter=1)
    assert list(out) == [0, -1, 0] and n[0] == 2 and it[0] == 1


def _halo(rng, n, c, sigma, mpart):
    pos = c + rng.normal(scale=1.0, size=(n, 3))
    vel = rng.normal(scale=sigma, size=(n, 3))
    return pos, vel, np.full(n, mpart)  # mpart: whole mass quanta (mass_unit 1)


def test_wrap_order_and_groups_are_independent():
    rng = np.random.default_rng(7)
    G = 1.0
    p1, v1, m1 = _halo(rng, 200, np.array([1.0, 50.0, 99.5]), 6.0, 1.0)  # straddles x = 0 and z = L
    p2, v2, m2 = _halo(rng, 150, np.array([30.0, 30.0, 30.0]), 5.0, 1.0)
    pos = np.vstack([p1, p2]) % L
    vel = np.vstack([v1, v2])
    mass = np.concatenate([m1, m2])
    group = np.concatenate([np.zeros(200, np.int32), np.ones(150, np.int32)])
    out, n, it, _ = _run(pos, vel, mass, group, G=G)
    assert n[0] > 0 and n[0] < 200  # some leave, the group stays
    # the same group moved to the middle of the box: same members kept
    shifted = (pos + np.array([49.0, 0.0, -49.5])) % L
    out_s, n_s, _, _ = _run(shifted, vel, mass, group, G=G)
    assert np.array_equal(out, out_s) and np.array_equal(n, n_s)
    # each group alone gives the same result as both together
    for g in (0, 1):
        sel = group == g
        o, nn, _, _ = _run(pos[sel], vel[sel], mass[sel], np.zeros(sel.sum(), np.int32), G=G)
        assert np.array_equal(np.where(o >= 0, g, -1), out[sel]) and nn[0] == n[g]
    # particle order does not matter (the first member only anchors the wrap)
    perm = rng.permutation(len(pos))
    out_p, n_p, _, _ = _run(pos[perm], vel[perm], mass[perm], group[perm], G=G)
    assert np.array_equal(out_p, out[perm]) and np.array_equal(n_p, n)


def test_ungrouped_particles_and_arguments():
    pos = np.array([[1, 1, 1], [2, 2, 2]], np.float32)
    vel = np.zeros((2, 3), np.float32)
    out, n, _, _ = oracle.unbind(pos, vel, np.array([-1, 0], np.int32), L, G=1.0)
    assert list(out) == [-1, 0] and list(n) == [1]
    with pytest.raises(oracle.OracleError):
        oracle.unbind(pos, vel, np.array([0, 0], np.int32), L, G=1.0, max_iter=0)
