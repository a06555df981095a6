"""The near-tie classifier on the CPU: fields perturbed from the oracle's own
fp64 field stand in for the GPU's.  Rounding-size noise must leave only
explained disagreements (and some must exist, so the check is not vacuous);
a real change to the field must leave unexplained ones."""
import numpy as np
import pytest

import oracle
from tests import near_tie


def _node(pos, L, ng):
    q = oracle.quantise(pos, L, ng)
    n = (q + 512) >> 10
    n[n == ng] = 0
    return (n[:, 2] * ng + n[:, 1]) * ng + n[:, 0]


def _run(pos, L, C64, C32_gpu, ref):
    lab_g = oracle.segment(C32_gpu)
    hid_g, cat_g = oracle.assign(pos, L, lab_g, C32_gpu)
    r = near_tie.classify_find(C64, ref["cwt32"], C32_gpu, ref["label"], lab_g, _node(pos, L, C64.shape[0]),
                               ref["halo_id"], hid_g)
    bad = near_tie.classify_catalogues(ref["cat"]["seed"], cat_g["seed"], ref["label"], lab_g,
                                       dict(zip(r["cells"].tolist(), r["cell_class"].tolist())),
                                       r["touched_seeds"])
    return r, bad


def test_rounding_noise_is_all_near_ties(work64):
    wl, pos, ref = work64
    pos = pos.numpy()
    C64 = ref["cwt"]
    amp = 3e-7 * np.max(np.abs(C64))  # fp32-rounding-sized error (about the GPU's)
    rng = np.random.default_rng(0)
    C32 = (C64 + amp * rng.standard_normal(C64.shape)).astype(np.float32)
    r, bad = _run(pos, wl.box, C64, C32, ref)
    assert len(r["cells"]) > 0  # labels differ (in the voids, where no kept halo lives)
    assert r["counts"]["unexplained"] == 0, r["counts"]
    assert r["cell_counts"]["unexplained"] == 0, r["cell_counts"]
    assert bad == []


def _boundary_flips(ref, k):
    """The k cells whose steepest-ascent choice beats a neighbour of another
    kept halo by the smallest fp64 margin: (cell, its parent, that neighbour,
    margin).  Rounding noise in the voids moves no particle, so the tests raise
    these neighbours instead, to make particles change halo."""
    C64, n = ref["cwt"], ref["cwt"].shape[0]
    lab, c64 = ref["label"].reshape(-1), C64.reshape(-1)
    P = oracle.parent(ref["cwt32"]).reshape(-1)
    kept = np.isin(lab, ref["cat"]["seed"])
    z, y, x = np.unravel_index(np.arange(n ** 3), (n, n, n))
    other, val = np.full(n ** 3, -1), np.full(n ** 3, -np.inf)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                j = (((z + dz) % n) * n + (y + dy) % n) * n + (x + dx) % n
                v = np.where((lab[j] != lab[P]) & kept[j] & kept[P], c64[j], -np.inf)
                t = v > val
                val, other = np.where(t, v, val), np.where(t, j, other)
    cells = np.flatnonzero((other >= 0) & (P != np.arange(n ** 3)))
    margin = c64[P[cells]] - val[cells]
    pick = cells[np.argsort(margin)[:k]]
    return pick, P[pick], other[pick], c64[P[pick]] - val[pick]


def test_flipped_boundary_choices_are_path_ties_and_threshold_flips(work64):
    # raise the rival neighbour of 12 basin-boundary cells just above the cell's
    # own choice: particles change halo.  With the tolerance set to cover the
    # largest raise, every change must be explained; with the default 1e-5 (far
    # below these margins) the same changes must not be
    wl, pos, ref = work64
    pos = pos.numpy()
    C64 = ref["cwt"]
    cells, par, rival, margin = _boundary_flips(ref, 12)
    C32 = ref["cwt32"].copy().reshape(-1)
    for r, p_ in zip(rival, par):
        C32[r] = np.nextafter(np.float32(max(C32[p_], C32[r])), np.float32(np.inf))
    C32 = C32.reshape(C64.shape)
    rel = 2.0 * (float(np.max(margin)) + 1e-3) / float(np.max(np.abs(C64)))
    lab_g = oracle.segment(C32)
    hid_g, cat_g = oracle.assign(pos, wl.box, lab_g, C32)
    node = _node(pos, wl.box, wl.ng)
    r = near_tie.classify_find(C64, ref["cwt32"], C32, ref["label"], lab_g, node, ref["halo_id"], hid_g, rel=rel)
    assert len(r["particles"]) > 0
    assert r["counts"]["unexplained"] == 0, r["counts"]
    assert r["counts"]["(i) near tie on the ascent path"] > 0
    r2 = near_tie.classify_find(C64, ref["cwt32"], C32, ref["label"], lab_g, node, ref["halo_id"], hid_g)
    assert r2["counts"]["unexplained"] > 0


def test_a_moved_peak_is_not_a_near_tie(work64):
    wl, pos, ref = work64
    pos = pos.numpy()
    C64 = ref["cwt"]
    C32 = ref["cwt32"].copy()
    # lower the field by 20 % of its maximum around the biggest halo's seed: its
    # basin changes, far beyond any rounding error
    s = int(ref["cat"]["seed"][np.argmax(ref["cat"]["n_part"])])
    z, y, x = np.unravel_index(s, C64.shape)
    C32[z - 1:z + 2, y - 1:y + 2, x - 1:x + 2] -= np.float32(0.2 * np.max(np.abs(C64)))
    r, bad = _run(pos, wl.box, C64, C32, ref)
    assert r["counts"]["unexplained"] > 0


def test_seed_tie_on_hand_cells():
    # one 8^3 field with two maxima: classify_cells must report a seed tie when a
    # maximum stays a maximum but crosses cwt_min by less than tol, and an
    # unexplained change when it moves by more
    z, y, x = np.meshgrid(*(np.arange(8),) * 3, indexing="ij")
    C64 = -1.0 - 0.01 * ((z - 2) ** 2 + (y - 2) ** 2 + (x - 2) ** 2)  # one slope up to (2, 2, 2)
    C64[2, 2, 2] = 10.0
    C64[6, 6, 6] = 1e-6  # a second maximum, within 1e-5 * 10 of cwt_min = 0
    ref32 = C64.astype(np.float32)
    gpu32 = ref32.copy()
    gpu32[6, 6, 6] = -1e-6  # no longer a seed on the "GPU" side
    lab_r, lab_g = oracle.segment(ref32), oracle.segment(gpu32)
    cells = np.flatnonzero(lab_r.reshape(-1) != lab_g.reshape(-1))
    assert cells.size > 0
    cls = near_tie.classify_cells(C64, ref32, gpu32, cells)
    assert set(cls.tolist()) == {near_tie.SEED_TIE}
    # a maximum whose fp64 value is far above cwt_min but that the other field
    # puts below it: no tie
    C64[6, 6, 6] = 0.3
    ref32 = C64.astype(np.float32)
    lab_r = oracle.segment(ref32)
    gpu32[6, 6, 6] = -0.5
    lab_g = oracle.segment(gpu32)
    cells = np.flatnonzero(lab_r.reshape(-1) != lab_g.reshape(-1))
    cls = near_tie.classify_cells(C64, ref32, gpu32, cells)
    assert cells.size > 0 and set(cls.tolist()) == {near_tie.UNEXPLAINED}
