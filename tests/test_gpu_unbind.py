"""The self-boundness check (Sec. 2.3) on the GPU against the oracle: the
closed-form cases, groups from a clumped box with virial velocities (small
groups sort in shared memory, larger ones in global memory, groups above a
size threshold take the whole-grid path), repeatability, and the error
paths."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import synth
from tests.gpu_util import dev, record

pytestmark = pytest.mark.gpu

# a decision this close to its threshold (relative) may fall either way
NEAR_TIE = 1e-9


@pytest.fixture(scope="module")
def uctx():
    c = pkg.Context(0, max_ng=64, max_np=1 << 20, max_scales=1, unbind=True)
    yield c
    c.close()


def _both(ctx, pos, vel, group, L, G, mass=None, mass_unit=1.0, n_groups=None, max_iter=100):
    pos = np.asarray(pos, np.float32)
    vel = np.asarray(vel, np.float32)
    group = np.asarray(group, np.int32)
    mass = None if mass is None else np.asarray(mass, np.float32)
    if n_groups is None:
        n_groups = int(group.max()) + 1
    ref = oracle.unbind(pos, vel, group, L, G=G, mass=mass, mass_unit=mass_unit, n_groups=n_groups,
                        max_iter=max_iter)
    out, nk, it = ctx.unbind(dev(pos), dev(vel), dev(group), L, G=G, mass=None if mass is None else dev(mass),
                             mass_unit=mass_unit, n_groups=n_groups, max_iter=max_iter)
    ctx.check()
    return (out.cpu().numpy(), nk.cpu().numpy(), it.cpu().numpy()), ref


def _same(got, ref):
    out, nk, it = got
    rout, rnk, rit, margin = ref
    if margin > NEAR_TIE:
        np.testing.assert_array_equal(out, rout)
        np.testing.assert_array_equal(nk, rnk)
        np.testing.assert_array_equal(it, rit)
    return margin


def test_closed_form_cases(uctx):
    L = 100.0
    # central mass with massless test particles at (1 +- 1e-3) v_esc
    rng = np.random.default_rng(4)
    n, G, M = 40, 2.5, 1.0
    r = rng.uniform(0.5, 5.0, n)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    fast = rng.random(n) < 0.3
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    c = np.array([30.0, 40.0, 50.0])
    pos = np.vstack([c, c + r[:, None] * d])
    vel = np.vstack([np.zeros(3), (np.sqrt(2.0 * G * M / r) * np.where(fast, 1.001, 0.999))[:, None] * u])
    mass = np.concatenate([[M], np.zeros(n)])
    got, ref = _both(uctx, pos, vel, np.zeros(n + 1), L, G, mass)
    assert _same(got, ref) > 5e-4
    assert np.array_equal(got[0][1:] == 0, ~fast)
    # recentring between rounds, and the round limit
    pos = [[50, 50, 50], [51, 50, 50], [48, 50, 50]]
    vel = [[0, 0, 0], [16.0, 0, 0], [16.0 / 11.0 + 3.0, 0, 0]]
    got, ref = _both(uctx, pos, vel, [0, 0, 0], L, 1.0, [10.0, 1.0, 0.0])
    _same(got, ref)
    assert list(got[0]) == [-1, -1, -1] and got[2][0] == 3
    got, ref = _both(uctx, pos, vel, [0, 0, 0], L, 1.0, [10.0, 1.0, 0.0], max_iter=1)
    _same(got, ref)
    assert list(got[0]) == [0, -1, 0]
    # the 40 % rule at its boundary, two groups in one call
    pos = [[50, 50, 50], [51, 50, 50], [49, 50, 50], [50, 51, 50], [50, 49, 50]] * 2
    vel = [[0, 0, 0]] + [[0, 0, 1.5 if k < 2 else 1.2] for k in range(4)]
    vel = vel + [[0, 0, 0]] + [[0, 0, 1.5 if k < 3 else 1.2] for k in range(4)]
    got, ref = _both(uctx, pos, vel, [0] * 5 + [1] * 5, L, 1.0, [1, 0, 0, 0, 0] * 2)
    _same(got, ref)
    assert list(got[0]) == [0, -1, -1, 0, 0] + [-1] * 5 and list(got[1]) == [3, 0]


def _box_groups(ng, n, L, seed, max_members=None):
    """Groups of a clumped box with virial velocities: the particles' cells
    (a coarse grid of cells of side L / ng), one group per occupied cell of the
    densest cells."""
    pos, vel = synth.clumped_box(n, L, max(2, n // 2000), seed=seed, velocities=True)
    pos, vel = pos.numpy(), vel.numpy()
    cell = np.floor(pos / (L / ng)).astype(np.int64) % ng
    key = (cell[:, 2] * ng + cell[:, 1]) * ng + cell[:, 0]
    uniq, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    keep = cnt >= 15
    if max_members is not None:
        keep &= cnt <= max_members
    gid = np.full(len(uniq), -1, np.int64)
    gid[keep] = np.arange(keep.sum())
    return pos, vel, gid[inv].astype(np.int32), int(keep.sum())


def test_clumped_box_groups_match_the_oracle(uctx):
    L = 50.0
    pos, vel, group, ng = _box_groups(16, 1 << 16, L, seed=3, max_members=1500)
    mp = synth.particle_mass(1 << 16, L)
    got, ref = _both(uctx, pos, vel, group, L, synth.G_MPC_KMS_MSUN, mass_unit=mp, n_groups=ng)
    margin = _same(got, ref)
    out, nk, it = got
    kept = int((nk > 0).sum())
    record({"config": f"self-boundness check, clumped 2^16 (L={L}), {ng} groups of 15-1500",
            "groups_kept": kept, "members_kept": int(nk.sum()), "members_in": int((group >= 0).sum()),
            "max_rounds": int(it.max()), "oracle_margin": margin})
    assert 0 < kept < ng and it.max() >= 2  # some groups lose members, some are discarded


def test_large_groups_sort_in_global_memory(uctx):
    # groups above 2048 members take the global-memory sort
    L = 20.0
    pos, vel = synth.clumped_box(30000, L, 3, seed=9, uniform_frac=0.1, velocities=True)
    pos, vel = pos.numpy(), vel.numpy()
    # three groups: the halves of the box along x, and one small one
    group = np.where(pos[:, 0] < L / 2, 0, 1).astype(np.int32)
    group[:300] = 2
    mp = synth.particle_mass(30000, L)
    got, ref = _both(uctx, pos, vel, group, L, synth.G_MPC_KMS_MSUN, mass_unit=mp, n_groups=3)
    _same(got, ref)
    assert (np.bincount(group, minlength=3)[:2] > 2048).all()


@pytest.mark.parametrize("grid_min", [1000, 1])
def test_whole_grid_path_matches_the_oracle(uctx, grid_min):
    # groups above grid_min members are processed by the whole grid, one at a
    # time (grid_min = 1: every group); the same decisions as the oracle, and
    # the same result on a second call
    L = 50.0
    pos, vel, group, ng = _box_groups(16, 1 << 16, L, seed=3)
    sizes = np.bincount(group[group >= 0], minlength=ng)
    assert (sizes > 1000).sum() >= 5 and sizes.max() > 16000
    mp = synth.particle_mass(1 << 16, L)
    uctx.debug_set(pkg._lib.DEBUG_UNBIND_GRID_MIN, grid_min)
    try:
        assert uctx.debug_get(pkg._lib.DEBUG_UNBIND_GRID_MIN) == grid_min
        got, ref = _both(uctx, pos, vel, group, L, synth.G_MPC_KMS_MSUN, mass_unit=mp, n_groups=ng)
        margin = _same(got, ref)
        again = uctx.unbind(dev(pos), dev(vel), dev(group), L, mass_unit=mp, n_groups=ng)
        uctx.check()
        for x, y in zip(again, got):
            np.testing.assert_array_equal(x.cpu().numpy(), y)
    finally:
        uctx.debug_set(pkg._lib.DEBUG_UNBIND_GRID_MIN, 1 << 16)
    out, nk, it = got
    record({"config": f"self-boundness check, whole-grid path for groups above {grid_min}, clumped 2^16 (L={L}), "
                      f"{ng} groups up to {int(sizes.max())}",
            "groups_kept": int((nk > 0).sum()), "members_kept": int(nk.sum()), "max_rounds": int(it.max()),
            "oracle_margin": margin})
    assert 0 < (nk > 0).sum() < ng


def test_repeatable_and_masses(uctx):
    L = 50.0
    pos, vel, group, ng = _box_groups(16, 1 << 15, L, seed=5, max_members=1000)
    rng = np.random.default_rng(1)
    mass = rng.uniform(0.5, 2.0, len(pos)).astype(np.float32)
    args = (dev(pos), dev(vel), dev(group), L)
    a = uctx.unbind(*args, G=1e-3, mass=dev(mass), mass_unit=0.125, n_groups=ng)
    b = uctx.unbind(*args, G=1e-3, mass=dev(mass), mass_unit=0.125, n_groups=ng)
    uctx.check()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    got, ref = _both(uctx, pos, vel, group, L, 1e-3, mass, 0.125, n_groups=ng)
    _same(got, ref)


def test_errors(uctx, gctx):
    pos = dev(np.zeros((4, 3), np.float32))
    grp = dev(np.zeros(4, np.int32))
    with pytest.raises(pkg.CwthfError):  # a context without the check's scratch
        gctx.unbind(pos, pos, grp, 10.0)
    with pytest.raises(pkg.CwthfError):
        uctx.unbind(pos, pos, grp, 10.0, max_iter=0)
    with pytest.raises(pkg.CwthfError):
        uctx.unbind(pos, pos, grp, -1.0)
    with pytest.raises(pkg.CwthfError):
        uctx.unbind(pos, pos, grp, 10.0, n_groups=64 ** 3)
    for v in (0, 1 << 31):
        with pytest.raises(pkg.CwthfError):
            uctx.debug_set(pkg._lib.DEBUG_UNBIND_GRID_MIN, v)
    bad = dev(np.array([1.0, -1.0, 1.0, 1.0], np.float32))
    uctx.unbind(pos, pos, grp, 10.0, mass=bad, n_groups=1)
    assert uctx.sync() == pkg._lib.E_BAD_INPUT
