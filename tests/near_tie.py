"""Near-tie classification of end-to-end disagreements (test infrastructure).

The GPU computes the CWT in fp32, the oracle in fp64; both segment their own
field, rounded to fp32, with the same strict order.  Where two fields differ
by rounding, a particle can change halo only through a decision that the
rounding can flip.  Every disagreement must be explained by one of:

  (i)   near tie on the ascent path: the two fields' ascent paths from the
        particle's node agree up to a cell where they pick different parents
        (or one of them stops at a maximum), and the two candidates' fp64
        values differ by at most tol = 1e-5 * max|C_fp64|;
  (ii)  near tie at the seed threshold: both paths reach the same maximum and
        its fp64 value lies within tol of cwt_min (seed on one side only);
  (iii) threshold flip: the node carries the same label on both sides, the
        halo is kept on one side only, and the halo's members differ between
        the sides (every differing cell being (i) or (ii)), so its filter
        quantities (Sec. 2.4, Table 1) move across a threshold.  A halo whose
        members are identical on both sides must get the same decision.

Only host code: the parents of both fields come from the oracle's own
26-neighbour scan (``oracle.parent``); nothing here runs on the GPU.
"""
from __future__ import annotations

import numpy as np

import oracle

NEAR_TIE_REL = 1e-5

UNEXPLAINED, PATH_TIE, SEED_TIE, THRESHOLD_FLIP = 0, 1, 2, 3
CLASS_NAMES = {UNEXPLAINED: "unexplained", PATH_TIE: "(i) near tie on the ascent path",
               SEED_TIE: "(ii) seed value near cwt_min", THRESHOLD_FLIP: "(iii) halo threshold flip"}


def classify_cells(C64, C32_ref, C32_gpu, cells, cwt_min=0.0, rel=NEAR_TIE_REL, max_steps=1 << 16):
    """Class (PATH_TIE, SEED_TIE or UNEXPLAINED) of each cell in `cells`
    (linear indices whose labels differ between the two fp32 fields)."""
    cells = np.asarray(cells, dtype=np.int64)
    out = np.full(cells.shape, UNEXPLAINED, dtype=np.int8)
    if cells.size == 0:
        return out
    c64 = np.asarray(C64, dtype=np.float64).reshape(-1)
    tol = rel * np.max(np.abs(c64))
    p_ref = oracle.parent(C32_ref).reshape(-1).astype(np.int64)
    p_gpu = oracle.parent(C32_gpu).reshape(-1).astype(np.int64)
    cur = cells.copy()
    active = np.ones(cells.shape, dtype=bool)
    for _ in range(max_steps):
        if not active.any():
            break
        a = np.flatnonzero(active)
        c = cur[a]
        pr, pg = p_ref[c], p_gpu[c]
        div = pr != pg
        if div.any():
            gap = np.abs(c64[pr[div]] - c64[pg[div]])
            out[a[div]] = np.where(gap <= tol, PATH_TIE, UNEXPLAINED)
            active[a[div]] = False
        top = ~div & (pr == c)  # a common maximum: only its seed status can differ
        if top.any():
            near = np.abs(c64[c[top]] - cwt_min) <= tol
            out[a[top]] = np.where(near, SEED_TIE, UNEXPLAINED)
            active[a[top]] = False
        step = ~div & ~top
        cur[a[step]] = pr[step]
    return out


def classify_find(C64, C32_ref, C32_gpu, lab_ref, lab_gpu, node, hid_ref, hid_gpu, cwt_min=0.0,
                  rel=NEAR_TIE_REL):
    """Classifies every particle whose halo id differs between the oracle's
    and the GPU's find.  node: each particle's nearest grid node (linear).
    Returns a dict with the per-particle classes, the per-cell classes and
    summary counts."""
    lab_ref = np.asarray(lab_ref).reshape(-1)
    lab_gpu = np.asarray(lab_gpu).reshape(-1)
    diff_cells = np.flatnonzero(lab_ref != lab_gpu)
    cell_cls = classify_cells(C64, C32_ref, C32_gpu, diff_cells, cwt_min, rel)
    cls_of_cell = dict(zip(diff_cells.tolist(), cell_cls.tolist()))
    # seeds whose membership differs: every label on either side of a differing cell
    touched = set(lab_ref[diff_cells].tolist()) | set(lab_gpu[diff_cells].tolist())
    touched.discard(-1)
    parts = np.flatnonzero(np.asarray(hid_ref) != np.asarray(hid_gpu))
    pcls = np.full(parts.shape, UNEXPLAINED, dtype=np.int8)
    for k, i in enumerate(parts.tolist()):
        c = int(node[i])
        if lab_ref[c] != lab_gpu[c]:
            pcls[k] = cls_of_cell[c]
        elif lab_ref[c] >= 0 and int(lab_ref[c]) in touched:
            pcls[k] = THRESHOLD_FLIP
    return dict(particles=parts, particle_class=pcls, cells=diff_cells, cell_class=cell_cls,
                counts={CLASS_NAMES[k]: int(np.sum(pcls == k)) for k in CLASS_NAMES},
                cell_counts={CLASS_NAMES[k]: int(np.sum(cell_cls == k)) for k in CLASS_NAMES},
                touched_seeds=touched)


def classify_catalogues(seeds_ref, seeds_gpu, lab_ref, lab_gpu, cell_class_of, touched):
    """Each seed kept on one side only must be explained: its own cell's label
    differs (a near tie at the seed, cell_class_of[seed] != 0) or its members
    differ (threshold flip).  Returns the list of unexplained seeds."""
    lab_ref = np.asarray(lab_ref).reshape(-1)
    lab_gpu = np.asarray(lab_gpu).reshape(-1)
    bad = []
    for s in np.setxor1d(seeds_ref, seeds_gpu).tolist():
        if lab_ref[s] != lab_gpu[s]:
            if cell_class_of.get(int(s), UNEXPLAINED) == UNEXPLAINED:
                bad.append(int(s))
        elif int(s) not in touched:
            bad.append(int(s))
    return bad
