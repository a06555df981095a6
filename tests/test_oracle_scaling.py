"""The oracle against the paper's stated linear scaling (Appendix A: run time
grows linearly with the data; Sec. 2.1: the grid CWT's cost is set by the
grid, the particle stages' by the particle count).  Timed on this host:

* grid stages (CWT, segmentation) from a 96^3 to a 192^3 grid: 8x the cells,
  so 8x the time (the CWT by FFT: 8 * log(192^3)/log(96^3)), within a factor 2;
* particle stages (CIC deposit, assignment) on one 96^3 grid: the time beyond
  the fixed cost of the grid (a call with no particles) grows in proportion to
  the particles, 4x from 2^21 to 2^23, within a factor 2.

Each size is timed as the best of several rounds that alternate the sizes.

Particles are presented in cell order at every size, so that the host's cache
hierarchy does not change the cost per particle between sizes; the arithmetic
the oracle performs is the same in any order."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_2501_10622_gb300 import synth


def _cell_ordered(n, L, ng, clumps, seed):
    pos = synth.clumped_box(n, L, clumps, seed=seed).numpy()
    c = np.floor(pos / (L / ng)).astype(np.int64) % ng
    return pos[np.argsort((c[:, 2] * ng + c[:, 1]) * ng + c[:, 0], kind="stable")]


def _best_interleaved(fns, reps):
    """Best time of each function over `reps` rounds that run them in turn, so
    that a burst of load on the host falls on every size alike."""
    t = [math.inf] * len(fns)
    for _ in range(reps):
        for k, fn in enumerate(fns):
            t0 = time.perf_counter()
            fn()
            t[k] = min(t[k], time.perf_counter() - t0)
    return t


def test_grid_stages_scale_with_the_cells():
    fields = {}
    for ng in (96, 192):
        L = ng * 0.78125
        pos = _cell_ordered(ng ** 3 // 8, L, ng, ng ** 3 // 1300, seed=ng)
        grid, _ = oracle.cic(pos, L, ng)
        fields[ng] = (grid, L, oracle.cwt(grid, L, 2.0).astype(np.float32))
    tc = _best_interleaved([lambda g=fields[n]: oracle.cwt(g[0], g[1], 2.0) for n in (96, 192)], 3)
    ts = _best_interleaved([lambda g=fields[n]: oracle.segment(g[2]) for n in (96, 192)], 3)
    cells = 8.0
    want_cwt = cells * math.log(192 ** 3) / math.log(96 ** 3)
    r_cwt = tc[1] / tc[0]
    r_seg = ts[1] / ts[0]
    print(f"grid stages 96^3 -> 192^3: CWT x{r_cwt:.2f} (N^3 log N: x{want_cwt:.2f}), segmentation x{r_seg:.2f} (x8)")
    assert want_cwt / 2 <= r_cwt <= want_cwt * 2, r_cwt
    assert cells / 2 <= r_seg <= cells * 2, r_seg


def test_particle_stages_scale_with_the_particles():
    ng, L = 96, 75.0
    sizes = (0, 1 << 21, 1 << 23)
    pos = {n: _cell_ordered(n, L, ng, 675, seed=3) for n in sizes[1:]}
    pos[0] = np.zeros((0, 3), np.float32)
    grid, _ = oracle.cic(pos[sizes[-1]], L, ng)
    C32 = oracle.cwt(grid, L, 2.0).astype(np.float32)
    lab = oracle.segment(C32)
    t_cic = _best_interleaved([lambda n=n: oracle.cic(pos[n], L, ng) for n in sizes], 5)
    t_asg = _best_interleaved([lambda n=n: oracle.assign(pos[n], L, lab, C32) for n in sizes], 5)
    for name, t in (("CIC deposit", t_cic), ("assignment", t_asg)):
        d1 = t[1] - t[0]  # time of 2^21 particles beyond the fixed cost of the grid
        d2 = t[2] - t[0]  # time of 2^23 particles
        r = d2 / d1
        print(f"{name}: {d1 * 1e3:.1f} ms per 2^21 particles, {d2 * 1e3:.1f} ms per 2^23 (ratio {r:.2f}, linear: 4)")
        assert d1 > 0 and 4 / 2 <= r <= 4 * 2, (name, t)
