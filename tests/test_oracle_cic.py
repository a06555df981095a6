"""Pins of the oracle's CIC deposit (Sec. 2.1, Eq. 1) against hand-worked values,
exact invariants and special cases -- not against the oracle itself."""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ONE30 = 1 << 30


def test_hand_worked_particle():
    g = json.load(open(os.path.join(GOLD, "cic_hand.json")))
    pos = np.array([g["particle"]], np.float32)
    grid, mt = oracle.cic(pos, g["L"], g["ng"])
    assert mt == 1
    expect = np.zeros_like(grid)
    for c in g["cells"]:
        x, y, z = c["xyz"]
        expect[z, y, x] = c["value"]
    np.testing.assert_array_equal(grid, expect)


def test_particle_on_node_fills_one_cell():
    pos = np.array([[5.0, 0.0, 63.0]], np.float32)
    grid, _ = oracle.cic(pos, 64.0, 64)
    assert grid[63, 0, 5] == ONE30
    assert np.count_nonzero(grid) == 1


def test_cell_centre_gives_eight_equal_shares():
    pos = np.array([[2.5, 3.5, 4.5]], np.float32)
    grid, _ = oracle.cic(pos, 8.0, 8)
    nz = grid[grid != 0]
    assert nz.size == 8 and np.all(nz == ONE30 // 8)
    assert grid[4:6, 3:5, 2:4].sum() == ONE30


def test_periodic_wrap_to_node_zero():
    # x = L - dx/4 -> node N-1 gets 1/4, node 0 gets 3/4 (wrapped)
    pos = np.array([[7.75, 0.0, 0.0]], np.float32)
    grid, _ = oracle.cic(pos, 8.0, 8)
    assert grid[0, 0, 7] == ONE30 // 4
    assert grid[0, 0, 0] == 3 * (ONE30 // 4)


def test_positions_outside_box_wrap():
    a, _ = oracle.cic(np.array([[1.25, 2.5, 3.75]], np.float32), 8.0, 8)
    b, _ = oracle.cic(np.array([[1.25 - 8.0, 2.5 + 8.0, 3.75 - 8.0]], np.float32), 8.0, 8)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("ng", [8, 12, 16])
def test_mass_conservation_exact(ng):
    rng = np.random.default_rng(ng)
    pos = (rng.random((5000, 3)) * 10.0).astype(np.float32)
    grid, mt = oracle.cic(pos, 10.0, ng)
    assert mt == 5000
    assert int(grid.sum()) == 5000 * ONE30
    assert grid.min() >= 0


def test_variable_mass_quantisation_and_conservation():
    rng = np.random.default_rng(7)
    pos = (rng.random((3000, 3)) * 5.0).astype(np.float32)
    mass = (rng.random(3000) * 3.0).astype(np.float32)
    unit = 1.0 / 1024
    grid, mt = oracle.cic(pos, 5.0, 12, mass=mass, mass_unit=unit)
    mq = np.rint(mass.astype(np.float64) / unit).astype(np.int64)  # round half to even
    assert mt == int(mq.sum())
    assert int(grid.sum()) == int(mq.sum()) * ONE30


def test_integer_cell_shift_rolls_grid():
    # cell = 1, positions on the 2^-10 lattice: an integer shift is exact in float32
    rng = np.random.default_rng(3)
    q = rng.integers(0, 16 * 1024, size=(2000, 3))
    pos = (q / 1024.0).astype(np.float32)
    g0, _ = oracle.cic(pos, 16.0, 16)
    shift = np.array([3, 5, 11])
    g1, _ = oracle.cic(((q + shift * 1024) % (16 * 1024) / 1024.0).astype(np.float32), 16.0, 16)
    np.testing.assert_array_equal(g1, np.roll(g0, shift=(11, 5, 3), axis=(0, 1, 2)))


def test_order_independent():
    rng = np.random.default_rng(11)
    pos = (rng.random((4000, 3)) * 3.0).astype(np.float32)
    a, _ = oracle.cic(pos, 3.0, 8)
    b, _ = oracle.cic(pos[rng.permutation(4000)], 3.0, 8)
    np.testing.assert_array_equal(a, b)


def test_quantise_matches_definition_on_exact_lattice():
    # on positions that are exact multiples of 2^-10 cells, floor(x*N/L*2^10) is the lattice index
    q = np.array([[0, 1, 1023], [1024, 65535, 7]], np.int64)
    pos = (q / 1024.0 * (50.0 / 64)).astype(np.float64)
    got = oracle.quantise(pos.astype(np.float32), 50.0, 64)
    # float32 rounding of pos may move a value by at most one lattice step downwards
    assert np.all(np.abs(got - q) <= 1)
    exact = oracle.quantise((q / 1024.0).astype(np.float32), 64.0, 64)
    np.testing.assert_array_equal(exact, q)


def _scale29(ng, L):
    """N 2^10 / L in fp64, rounded half-to-even to 29 significant bits."""
    import math
    m, e = math.frexp((ng / L) * 1024.0)
    return round(m * 2 ** 29) * 2.0 ** (e - 29)


def test_quantise_is_floor_of_exact_product():
    # with a 29-bit scale and 24-bit floats the product is exact: the code is
    # the floor of the rational x*s, wrapped into [0, N 2^10)
    from fractions import Fraction
    rng = np.random.default_rng(11)
    for ng, L in ((64, 50.0), (1024, 500.0), (96, 77.7), (8, 3.0)):
        s = Fraction(_scale29(ng, L))
        assert s.denominator & (s.denominator - 1) == 0 and (s.numerator.bit_length() <= 29)
        x = np.concatenate([rng.random(3000) * L, rng.random(300) * L * 3 - L, [0.0, L, np.nextafter(L, 0)]])
        x = x.astype(np.float32)
        got = oracle.quantise(np.stack([x, x, x], 1), L, ng)[:, 0]
        mod = ng * 1024
        want = np.array([(int(Fraction(float(v)) * s // 1)) % mod for v in x], np.int64)
        np.testing.assert_array_equal(got, want)


def test_rejects_bad_input():
    with pytest.raises(oracle.OracleError) as e:
        oracle.cic(np.array([[np.nan, 0, 0]], np.float32), 8.0, 8)
    assert e.value.code == oracle.E_ARG
    big = np.full(5, 2.0 ** 31 - 1, np.float32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.cic(np.zeros((5, 3), np.float32), 8.0, 8, mass=big, mass_unit=1.0)
    assert e.value.code in (oracle.E_ARG, oracle.E_OVERFLOW)
    with pytest.raises(oracle.OracleError) as e:
        oracle.cic(np.zeros((5, 3), np.float32), 8.0, 8, mass=np.full(5, -1.0, np.float32))
    assert e.value.code == oracle.E_ARG
