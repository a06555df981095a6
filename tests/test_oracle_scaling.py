"""The oracle against the paper's stated linear scaling (Appendix A: run time
grows linearly with the data; Sec. 2.1: the grid CWT's cost is set by the
grid, the particle stages' by the particle count).  Timed on this host:

* grid stages (CWT, segmentation) from a 96^3 to a 192^3 grid: 8x the cells,
  so 8x the time (the CWT by FFT: 8 * log(192^3)/log(96^3)), within a factor 2;
* particle stages (CIC deposit, assignment) on one 96^3 grid: the time added by
  particles grows in proportion to the particles added (from 2^20 to 2^22 and
  from 2^22 to 2^23 particles), within a factor 2.

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


def _best(fn, reps):
    t = math.inf
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        t = min(t, time.perf_counter() - t0)
    return t


def test_grid_stages_scale_with_the_cells():
    times = {}
    for ng, reps in ((96, 3), (192, 1)):
        L = ng * 0.78125
        pos = _cell_ordered(ng ** 3 // 8, L, ng, ng ** 3 // 1300, seed=ng)
        grid, _ = oracle.cic(pos, L, ng)
        C = None

        def cwt():
            nonlocal C
            C = oracle.cwt(grid, L, 2.0)
        tc = _best(cwt, reps)
        C32 = C.astype(np.float32)
        ts = _best(lambda: oracle.segment(C32), reps)
        times[ng] = (tc, ts)
    cells = 8.0
    want_cwt = cells * math.log(192 ** 3) / math.log(96 ** 3)
    r_cwt = times[192][0] / times[96][0]
    r_seg = times[192][1] / times[96][1]
    print(f"grid stages 96^3 -> 192^3: CWT x{r_cwt:.2f} (N^3 log N: x{want_cwt:.2f}), segmentation x{r_seg:.2f} (x8)")
    assert want_cwt / 2 <= r_cwt <= want_cwt * 2, r_cwt
    assert cells / 2 <= r_seg <= cells * 2, r_seg


def test_particle_stages_scale_with_the_particles():
    ng, L = 96, 75.0
    lab = C32 = None
    t = {}
    for n in (1 << 20, 1 << 22, 1 << 23):
        pos = _cell_ordered(n, L, ng, 675, seed=3)
        if lab is None:
            grid, _ = oracle.cic(pos, L, ng)
            C32 = oracle.cwt(grid, L, 2.0).astype(np.float32)
            lab = oracle.segment(C32)
        t[n] = (_best(lambda: oracle.cic(pos, L, ng), 7), _best(lambda: oracle.assign(pos, L, lab, C32), 7))
    a, b, c = 1 << 20, 1 << 22, 1 << 23
    for k, name in enumerate(("CIC deposit", "assignment")):
        d1 = t[b][k] - t[a][k]  # time of 3 * 2^20 more particles
        d2 = t[c][k] - t[b][k]  # time of 4 * 2^20 more particles
        r = d2 / d1
        print(f"{name}: {d1 * 1e3:.1f} ms per 3*2^20 particles, {d2 * 1e3:.1f} ms per 4*2^20 (ratio {r:.2f}, "
              f"linear: 1.33)")
        assert d1 > 0 and (4 / 3) / 2 <= r <= (4 / 3) * 2, (name, d1, d2)
