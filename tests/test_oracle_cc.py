"""Pins of the oracle's equiangular Clenshaw-Curtis grid (App. C.1, "Equiangular ...
Clenshaw-Curtis") against closed forms, exactness, a high-precision moment solve and
the heat operator's identities on that grid."""
import numpy as np
import pytest

from oracle.grid import Grid, clenshaw_curtis, gauss_legendre
from oracle import sht, dense


def test_cc_textbook_closed_forms():
    # 3 nodes: Simpson's rule [1, 4, 1]/3; 5 nodes: [1, 8, 12, 8, 1]/15
    x, w = clenshaw_curtis(3)
    np.testing.assert_allclose(x, [1, 0, -1], atol=0)
    np.testing.assert_allclose(w, np.array([1, 4, 1]) / 3, rtol=0, atol=1e-15)
    x, w = clenshaw_curtis(5)
    np.testing.assert_allclose(x, [1, np.sqrt(0.5), 0, -np.sqrt(0.5), -1], atol=1e-16)
    np.testing.assert_allclose(w, np.array([1, 8, 12, 8, 1]) / 15, rtol=0, atol=1e-15)
    # 2 nodes: the trapezoid rule
    x, w = clenshaw_curtis(2)
    np.testing.assert_allclose(w, [1, 1], atol=1e-15)


@pytest.mark.parametrize("n", [4, 7, 16, 33, 128, 513])
def test_cc_exactness_symmetry_positivity(n):
    x, w = clenshaw_curtis(n)
    N = n - 1
    assert np.all(np.diff(x) < 0) and x[0] == 1.0 and x[-1] == -1.0
    np.testing.assert_array_equal(x, -x[::-1])
    np.testing.assert_array_equal(w, w[::-1])
    assert np.all(w > 0)
    assert abs(w.sum() - 2.0) < 1e-13
    # exact for degree <= N; odd degrees vanish by symmetry
    for k in range(0, N + 1, max(1, N // 40)):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13, k
    # not exact at the next even degree beyond N (so it is not Gauss-Legendre); the
    # error on a monomial decays fast with n, so small n only
    k = N + 1 if (N + 1) % 2 == 0 else N + 2
    if n <= 16:
        assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-8


@pytest.mark.parametrize("n", [6, 11, 20])
def test_cc_matches_moment_solve(n):
    # weights from the moment equations sum_j w_j x_j^k = int x^k, k = 0..N, solved in
    # 40-digit arithmetic at the same nodes (independent of the Chebyshev form)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, w = clenshaw_curtis(n)
    N = n - 1
    xs = [mp.cos(mp.pi * j / N) for j in range(n)]
    V = mp.matrix(n, n)
    b = mp.matrix(n, 1)
    for k in range(n):
        for j in range(n):
            V[k, j] = xs[j] ** k
        b[k] = mp.mpf(2) / (k + 1) if k % 2 == 0 else 0
    ws = mp.lu_solve(V, b)
    for j in range(n):
        assert abs(float(w[j] - ws[j])) < 1e-14
        assert abs(float(x[j] - xs[j])) < 2e-16


def test_cc_area_weights_and_defaults():
    g = Grid(9, quadrature="cc")
    assert abs(g.a.sum() - 4 * np.pi) < 1e-13
    assert g.nlon == 18 and g.lmax == 8
    assert g.theta[0] == 0.0 and abs(g.theta[-1] - np.pi) < 1e-15
    # the GL grid of the same size has different nodes
    assert not np.allclose(g.x, gauss_legendre(9)[0])


@pytest.mark.parametrize("nlat,t", [(5, 0.1), (9, 0.01), (16, 0.02), (25, 0.003)])
def test_cc_sht_equals_dense_heat_matrix(nlat, t):
    # the addition theorem holds for any node set and weights: SHT path == H diag(a)
    g = Grid(nlat, quadrature="cc")
    f = np.random.default_rng(nlat).normal(size=(2, g.nlat, g.nlon))
    ref = dense.dense_apply(dense.kernel_matrix(g, t), f)
    np.testing.assert_allclose(sht.heat_apply(g, f, t), ref, atol=1e-12 * np.abs(ref).max())


def test_cc_heat_constant_mass_symmetry():
    g = Grid(24, quadrature="cc")
    rng = np.random.default_rng(7)
    v, w = rng.uniform(size=(2, g.nlat, g.nlon))
    t = 0.01
    np.testing.assert_allclose(sht.heat_apply(g, np.ones((g.nlat, g.nlon)), t), 1.0, atol=1e-13)
    kv, kw = sht.heat_apply(g, v, t), sht.heat_apply(g, w, t)
    a = g.a
    assert abs(np.sum(a * kv) - np.sum(a * v)) < 1e-13 * np.sum(a * v)
    assert abs(np.sum(a * w * kv) - np.sum(a * v * kw)) < 1e-13 * abs(np.sum(a * w * kv))


@pytest.mark.parametrize("nlat", [9, 17, 32])
def test_cc_round_trip_exact_below_half_band(nlat):
    # P_lm P_l'm is a polynomial of degree l + l' in x (times (1-x^2)^m, itself of degree
    # 2m), so the analysis is exact when 2 lmax <= N = nlat - 1 ...
    lmax = (nlat - 1) // 2
    g = Grid(nlat, lmax=lmax, quadrature="cc")
    rng = np.random.default_rng(nlat)
    c = rng.normal(size=(2, lmax + 1, lmax + 1)) + 1j * rng.normal(size=(2, lmax + 1, lmax + 1))
    c = np.tril(c)
    c[..., :, 0] = c[..., :, 0].real
    c2 = sht.analysis(g, sht.synthesis(g, c))
    assert np.abs(c2 - c).max() < 1e-12 * np.abs(c).max()
    # ... and not at the full band lmax = nlat - 1
    g2 = Grid(nlat, quadrature="cc")
    c = rng.normal(size=(1, g2.lmax + 1, g2.lmax + 1))
    c = np.tril(c)
    c2 = sht.analysis(g2, sht.synthesis(g2, c))
    assert np.abs(c2 - c).max() > 1e-6
