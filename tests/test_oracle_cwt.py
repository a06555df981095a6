"""Pins of the oracle's grid CWT (Sec. 2.1, Eq. 2-4): its DFT against numpy and
brute force, the FFT convolution against the literal Eq. 2 double sum, the
sampled wavelet's spectrum against the analytic Fourier transform of Eq. 4,
and invariants (shift equivariance, linearity, uniform input)."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_10622_gb300 import synth


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 18, 24, 27, 32, 48, 64, 96, 128])
def test_dft1d_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle.dft1d(x, -1)
    ref = np.fft.fft(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    inv = oracle.dft1d(x, +1)
    assert np.max(np.abs(inv - np.fft.ifft(x) * n)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [6, 12, 20])
def test_dft1d_matches_brute_force_sum(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    brute = np.array([np.sum(x * np.exp(-2j * np.pi * kk * k / n)) for kk in k])
    assert np.max(np.abs(oracle.dft1d(x) - brute)) < 1e-11


@pytest.mark.parametrize("n", [4, 6, 8, 12])
def test_dft3d_matches_numpy_and_parseval(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    X = oracle.dft3d(x)
    assert np.max(np.abs(X - np.fft.fftn(x))) < 1e-10
    assert abs(np.sum(np.abs(X) ** 2) / n ** 3 - np.sum(np.abs(x) ** 2)) < 1e-9 * np.sum(np.abs(x) ** 2)


def test_wavelet_special_values():
    w = 1.7
    assert oracle.wavelet(w, 0.0) == pytest.approx(6.0 * w ** 1.5, rel=1e-15)
    # zero crossing at w r = sqrt(6)
    assert abs(oracle.wavelet(w, 6.0 / w ** 2)) < 1e-14
    assert oracle.wavelet(w, 7.0 / w ** 2) < 0 < oracle.wavelet(w, 5.0 / w ** 2)
    # the 3D wavelet has zero integral: 4 pi int r^2 Psi dr = 0 (trapezoid on a fine mesh)
    r = np.linspace(0.0, 12.0 / w, 200001)
    f = np.array([oracle.wavelet(w, rr * rr) for rr in r[::50]])
    rr = r[::50]
    integral = np.trapezoid(4 * np.pi * rr ** 2 * f, rr)
    scale = np.trapezoid(4 * np.pi * rr ** 2 * np.abs(f), rr)
    assert abs(integral) < 1e-6 * scale


@pytest.mark.parametrize("n,w", [(4, 1.3), (6, 0.9), (8, 2.0), (12, 1.5)])
def test_fft_cwt_equals_direct_eq2_sum(n, w):
    rng = np.random.default_rng(n)
    L = n * 0.8
    pos = (rng.random((60, 3)) * L).astype(np.float32)
    grid, _ = oracle.cic(pos, L, n)
    a = oracle.cwt(grid, L, w)
    b = oracle.cwt_direct(grid, L, w)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_point_mass_on_node_gives_shifted_kernel():
    n, L, w = 16, 16.0, 1.1
    g = (3, 7, 12)  # x, y, z node
    pos = np.array([[g[0], g[1], g[2]]], np.float32)
    grid, _ = oracle.cic(pos, L, n)
    C = oracle.cwt(grid, L, w)
    assert C[g[2], g[1], g[0]] == pytest.approx(6.0 * w ** 1.5, rel=1e-12)
    # every value is Eq. 4 at the minimum-image separation from the node
    idx = np.arange(n)
    d = lambda a, c: np.where(np.abs(a - c) <= n // 2, a - c, a - c - np.sign(a - c) * n)
    dz, dy, dx = np.meshgrid(d(idx, g[2]), d(idx, g[1]), d(idx, g[0]), indexing="ij")
    r2 = (dx * 1.0) ** 2 + (dy * 1.0) ** 2 + (dz * 1.0) ** 2
    closed = w ** 1.5 * (6 - w * w * r2) * np.exp(-w * w * r2 / 4)
    assert np.max(np.abs(C - closed)) < 1e-12 * 6 * w ** 1.5


def test_sampled_wavelet_spectrum_matches_analytic_transform():
    # Psi = -(4/w^2) w^{3/2} Laplacian(exp(-w^2 r^2/4)), so its 3D Fourier transform is
    # 32 pi^{3/2} w^{-7/2} k^2 exp(-k^2/w^2).  For w*dx << 1 the DFT of the sampled
    # kernel times dx^3 converges to it (Poisson summation; aliasing ~exp(-(2pi/dx)^2/w^2)).
    n, L, w = 48, 36.0, 0.6
    dx = L / n
    K = oracle.kernel(n, L, w)
    Kh = np.real(oracle.dft3d(K.astype(np.complex128))) * dx ** 3
    peak = 32 * math.pi ** 1.5 * w ** -3.5 * (w * w) * math.exp(-1.0)  # max over k at k = w
    for m in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 1, 2), (4, 4, 0), (5, 0, 3)]:
        k2 = sum((2 * math.pi * mi / L) ** 2 for mi in m)
        analytic = 32 * math.pi ** 1.5 * w ** -3.5 * k2 * math.exp(-k2 / w ** 2)
        assert abs(Kh[m[2], m[1], m[0]] - analytic) < 1e-6 * peak


def test_uniform_grid_gives_constant_mean_times_kernel_sum():
    n, L, w = 12, 9.0, 1.4
    grid = np.full((n, n, n), 5 * (1 << 30), np.int64)
    C = oracle.cwt(grid, L, w)
    ksum = oracle.kernel(n, L, w).sum()
    assert np.max(np.abs(C - 5.0 * ksum)) < 1e-10 * (1 + abs(5.0 * ksum))


def test_shift_equivariance_and_linearity():
    rng = np.random.default_rng(5)
    n, L, w = 12, 10.0, 1.2
    ga, _ = oracle.cic((rng.random((300, 3)) * L).astype(np.float32), L, n)
    gb, _ = oracle.cic((rng.random((200, 3)) * L).astype(np.float32), L, n)
    Ca, Cb = oracle.cwt(ga, L, w), oracle.cwt(gb, L, w)
    s = (2, 7, 5)
    Cr = oracle.cwt(np.roll(ga, s, axis=(0, 1, 2)), L, w)
    assert np.max(np.abs(Cr - np.roll(Ca, s, axis=(0, 1, 2)))) < 1e-12 * np.max(np.abs(Ca))
    Cab = oracle.cwt(ga + gb, L, w)
    assert np.max(np.abs(Cab - Ca - Cb)) < 1e-12 * np.max(np.abs(Cab))


def test_isolated_clump_peaks_at_its_centre():
    # a symmetric clump centred on a node: the CWT maximum is that node, and the
    # only positive maximum (the direct sum has no FFT round-off in the far field)
    n, L, w = 12, 12.0, 0.9
    c = np.array([6.0, 5.0, 4.0])
    offs = np.array([[dx, dy, dz] for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)], float) * 0.5
    pos = (c + offs).astype(np.float32)
    grid, _ = oracle.cic(pos, L, n)
    C = oracle.cwt_direct(grid, L, w)
    z, y, x = np.unravel_index(np.argmax(C), C.shape)
    assert (x, y, z) == (6, 5, 4)
    lab = oracle.segment(C.astype(np.float32), 0.0)
    seeds = np.flatnonzero(lab.ravel() == np.arange(lab.size))
    assert seeds.tolist() == [(4 * n + 5) * n + 6]


@pytest.mark.parametrize("n,L,w", [(12, 9.0, 1.0), (16, 40.0, 3.0), (10, 50.0, 4.0), (9, 7.0, 2.0)])
def test_cwt_at_nodes_equals_direct_eq2_sum(n, L, w):
    # the support-limited sum at chosen nodes is the literal Eq. 2 sum (only the
    # order of the additions differs); large w*dx exercises the truncated support
    rng = np.random.default_rng(n)
    grid = (rng.random((n, n, n)) < 0.3) * rng.integers(1, 1 << 31, (n, n, n))
    full = oracle.cwt_direct(grid, L, w)
    nodes = np.concatenate([[0, n ** 3 - 1], rng.integers(0, n ** 3, 40)])
    got = oracle.cwt_at(grid, L, w, nodes)
    np.testing.assert_allclose(got, full.ravel()[nodes], rtol=1e-12, atol=1e-12 * np.abs(full).max())


def test_cwt_at_far_nodes_see_only_the_support():
    # a single particle mass on a 96^3 grid: nodes far beyond the fp64 support get exactly 0
    n, L, w = 96, 96.0, 4.0
    grid = np.zeros((n, n, n), np.int64)
    grid[10, 20, 30] = 1 << 30
    near = (10 * n + 20) * n + 31
    far = (58 * n + 68) * n + 78
    v = oracle.cwt_at(grid, L, w, [near, far])
    assert v[0] == pytest.approx(oracle.wavelet(w, 1.0))
    assert v[1] == 0.0


# ---- the paper's direct-space stencil evaluation (Sec. 2.1, Table 1) --------

def test_stencil_point_mass_is_the_truncated_wavelet():
    # a unit mass on one node: C is the sampled wavelet on the cube around it
    # and exactly zero outside (closed form, Eq. 4)
    ng, L, w, R = 16, 16.0, 1.3, 3  # one cell per unit length: the mass sits exactly on node (5, 9, 2)
    pos = np.array([[5 * L / ng, 9 * L / ng, 2 * L / ng]], np.float32)
    assert np.count_nonzero(oracle.cic(pos, L, ng)[0]) == 1
    grid, _ = oracle.cic(pos, L, ng)
    C = oracle.cwt_stencil(grid, L, w, R)
    dx = L / ng
    for z in range(ng):
        for y in range(ng):
            for x in range(ng):
                d = [((x - 5 + 8) % 16) - 8, ((y - 9 + 8) % 16) - 8, ((z - 2 + 8) % 16) - 8]
                if max(abs(v) for v in d) <= R:
                    r2 = dx * dx * sum(v * v for v in d)
                    want = w ** 1.5 * (6 - w * w * r2) * np.exp(-w * w * r2 / 4)
                    assert abs(C[z, y, x] - want) <= 1e-12 * 6 * w ** 1.5
                else:
                    assert C[z, y, x] == 0.0


def test_stencil_covering_the_support_equals_the_fft_cwt():
    # once the cube holds every offset where the wavelet is not negligible in
    # fp64 (here w * Delta * R = 9.6: Psi < 1e-9 of its peak beyond), the stencil
    # sum and the whole-box convolution agree
    ng, L, w = 24, 24.0, 2.4
    pos = synth.clumped_box(3000, L, 4, seed=2).numpy()
    grid, _ = oracle.cic(pos, L, ng)
    R = 11  # 2R + 1 = 23 <= 24
    Cs = oracle.cwt_stencil(grid, L, w, R)
    Cf = oracle.cwt(grid, L, w)
    assert np.max(np.abs(Cs - Cf)) <= 1e-9 * np.max(np.abs(Cf))


def test_stencil_is_linear_and_roll_equivariant():
    ng, L, w, R = 20, 15.0, 1.3, 4
    rng = np.random.default_rng(4)
    a = rng.integers(0, 1 << 30, (ng, ng, ng)).astype(np.int64)
    b = rng.integers(0, 1 << 30, (ng, ng, ng)).astype(np.int64)
    Ca, Cb = oracle.cwt_stencil(a, L, w, R), oracle.cwt_stencil(b, L, w, R)
    np.testing.assert_allclose(oracle.cwt_stencil(a + b, L, w, R), Ca + Cb, rtol=0, atol=1e-9 * np.abs(Ca).max())
    sh = (3, -5, 7)
    np.testing.assert_allclose(oracle.cwt_stencil(np.roll(a, sh, (0, 1, 2)), L, w, R), np.roll(Ca, sh, (0, 1, 2)),
                               rtol=0, atol=1e-12 * np.abs(Ca).max())


def test_stencil_truncation_error_is_the_dropped_tail():
    # the difference between the whole-box CWT and the stencil CWT of a point
    # mass is the wavelet outside the cube; Table 1's stencil Int(1.5/k_w + 5)
    # drops at most a few 1e-3 of the peak at the paper's grid sizes
    for kw in (0.1, 0.5, 1.0, 2.5):
        L = 50.0
        ng = int(400 * kw + 150)
        w = kw * 1000.0 / L
        R = oracle.gdw_resolution(kw)
        dx = L / ng
        # largest |Psi| on the cube's surface and beyond, relative to the peak 6 w^1.5
        r = dx * (R + 1)
        tail = max(abs((6 - w * w * rr * rr) * np.exp(-w * w * rr * rr / 4)) for rr in np.linspace(r, 3 * r, 400))
        assert tail / 6.0 < 5e-3, (kw, R, tail / 6.0)


def test_stencil_at_nodes_equals_the_whole_stencil_grid():
    ng, L, w, R = 20, 16.0, 1.9, 4
    pos = synth.clumped_box(2500, L, 5, seed=9).numpy()
    grid, _ = oracle.cic(pos, L, ng)
    C = oracle.cwt_stencil(grid, L, w, R).reshape(-1)
    nodes = np.random.default_rng(0).integers(0, ng ** 3, 40)
    np.testing.assert_allclose(oracle.cwt_stencil_at(grid, L, w, R, nodes), C[nodes], rtol=0,
                               atol=1e-12 * np.abs(C).max())
