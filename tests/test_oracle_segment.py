"""Pins of the oracle's maxima and steepest-ascent segmentation (Sec. 2 step 4-5,
Sec. 2.3): an independent vectorised 26-neighbour recount, hand-built fields with
known answers, and invariants that any correct labelling satisfies."""
import itertools

import numpy as np
import pytest

import oracle

OFFS = [d for d in itertools.product((-1, 0, 1), repeat=3)]


def maxima_by_rolls(C):
    """Independent recount: a cell is a maximum iff it beats each of its 26
    periodic neighbours under (value, smaller index wins)."""
    n = C.shape[0]
    idx = np.arange(C.size).reshape(C.shape)
    is_max = np.ones(C.shape, bool)
    for d in OFFS:
        if d == (0, 0, 0):
            continue
        Cn = np.roll(C, shift=(-d[0], -d[1], -d[2]), axis=(0, 1, 2))
        In = np.roll(idx, shift=(-d[0], -d[1], -d[2]), axis=(0, 1, 2))
        is_max &= (C > Cn) | ((C == Cn) & (idx < In))
    return is_max


@pytest.mark.parametrize("n,seed", [(6, 0), (8, 1), (12, 2), (16, 3)])
def test_maxima_match_independent_recount(n, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((n, n, n)).astype(np.float32)
    C[rng.random(C.shape) < 0.2] = 0.5  # plateaus exercise the tie order
    P = oracle.parent(C)
    np.testing.assert_array_equal(P.ravel() == np.arange(C.size), maxima_by_rolls(C).ravel())


def test_constant_field_single_maximum_at_index_zero():
    C = np.ones((8, 8, 8), np.float32)
    lab = oracle.segment(C, 0.0)
    assert np.all(lab == 0)
    assert np.all(oracle.segment(C, 1.0) == -1)  # the only maximum is not above cwt_min


@pytest.mark.parametrize("n,seed", [(8, 4), (12, 5), (16, 6)])
def test_label_invariants(n, seed):
    rng = np.random.default_rng(seed)
    C = (rng.standard_normal((n, n, n)) + 0.3).astype(np.float32)
    P = oracle.parent(C).ravel()
    lab = oracle.segment(C, 0.0).ravel()
    Cf = C.ravel()
    seeds = np.flatnonzero(lab == np.arange(lab.size))
    # every seed is a maximum above cwt_min; every non-negative label is a seed
    assert np.all(P[seeds] == seeds) and np.all(Cf[seeds] > 0)
    assert np.all(np.isin(lab[lab >= 0], seeds))
    # labels are constant along parent chains; values never decrease along them
    np.testing.assert_array_equal(lab, lab[P])
    assert np.all(Cf[P] >= Cf)
    # maxima at or below cwt_min label their whole basin -1
    maxima = np.flatnonzero(P == np.arange(P.size))
    assert np.all(lab[maxima[Cf[maxima] <= 0]] == -1)


def test_two_bumps_two_seeds_boundary_at_valley():
    n = 24
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")

    def bump(cx, cy, cz, amp):
        d2 = np.minimum(abs(x - cx), n - abs(x - cx)) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        return amp * np.exp(-d2 / 8.0)

    C = (bump(6, 12, 12, 1.0) + bump(16, 12, 12, 0.8)).astype(np.float32)
    lab = oracle.segment(C, 0.0)
    a, b = (12 * n + 12) * n + 6, (12 * n + 12) * n + 16
    seeds = sorted(set(lab.ravel().tolist()) - {-1})
    assert seeds == [a, b]
    row = lab[12, 12, :]
    # along the line joining the peaks the label switches once, at the valley
    valley = 6 + int(np.argmin(C[12, 12, 6:17]))
    assert np.all(row[6:valley] == a) and np.all(row[valley + 1:17] == b)


def test_roll_equivariance_of_partition():
    rng = np.random.default_rng(9)
    n = 12
    C = (rng.standard_normal((n, n, n)) + 0.2).astype(np.float32)  # tie-free with probability 1
    s = (3, 1, 7)
    la = oracle.segment(C, 0.0)
    lb = oracle.segment(np.roll(C, s, axis=(0, 1, 2)), 0.0)
    la_r = np.roll(la, s, axis=(0, 1, 2))
    # same partition: a bijection between label values
    pairs = set(zip(la_r.ravel().tolist(), lb.ravel().tolist()))
    assert len(pairs) == len(set(la_r.ravel().tolist())) == len(set(lb.ravel().tolist()))
    assert (-1, -1) in pairs or -1 not in la_r


def test_nan_rejected():
    C = np.zeros((4, 4, 4), np.float32)
    C[1, 2, 3] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.segment(C, 0.0)
