"""Pins of the oracle's grid and Legendre tables against mathematics and library routines."""
import numpy as np
import pytest
import scipy.special as sps

from oracle.grid import Grid, gauss_legendre
from oracle.legendre import pbar, legendre_series


@pytest.mark.parametrize("n", [1, 2, 5, 32, 64, 180, 256])
def test_gl_matches_library(n):
    # numpy's leggauss (library routine) returns ascending nodes
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.all(np.diff(x) < 0)
    np.testing.assert_allclose(x, xr[::-1], rtol=0, atol=2e-15)
    # numpy's weights carry ~1e-11 relative error at n = 256 (checked against mpmath below)
    np.testing.assert_allclose(w, wr[::-1], rtol=3e-11, atol=0)


@pytest.mark.parametrize("n", [64, 256])
def test_gl_matches_high_precision(n):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, w = gauss_legendre(n)
    for j in range(0, n, max(1, n // 12)):
        xj = mp.mpf(x[j])
        for _ in range(4):   # polish the root in 40-digit arithmetic
            p = mp.legendre(n, xj)
            dp = n * (mp.legendre(n - 1, xj) - xj * p) / (1 - xj * xj)
            xj -= p / dp
        dp = n * (mp.legendre(n - 1, xj) - xj * mp.legendre(n, xj)) / (1 - xj * xj)
        wj = 2 / ((1 - xj * xj) * dp * dp)
        assert abs(float(x[j] - xj)) < 2e-16
        assert abs(float((w[j] - wj) / wj)) < 2e-12


@pytest.mark.parametrize("n", [3, 16, 33, 720])
def test_gl_exactness(n):
    # exact for polynomials of degree <= 2n-1: int_{-1}^{1} x^k = 2/(k+1) (k even), 0 (odd)
    x, w = gauss_legendre(n)
    assert abs(w.sum() - 2.0) < 1e-13
    for k in range(0, 2 * n, max(1, (2 * n) // 40)):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13, k
    # and not exact at degree 2n (the error term shrinks like 4^-n, so small n only)
    if n <= 16:
        k = 2 * n
        assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-12


def test_area_weights_total_4pi():
    for n in (8, 31, 180):
        g = Grid(n)
        assert abs(g.a.sum() - 4 * np.pi) < 1e-12
        assert g.nlon == 2 * n and g.lmax == n - 1


@pytest.mark.parametrize("lmax", [0, 1, 7, 20])
def test_pbar_matches_scipy_sph_harm(lmax):
    # Y_lm(theta, 0) = Pbar_lm(cos theta) (orthonormal, Condon-Shortley), library routine
    theta = np.linspace(0.05, np.pi - 0.05, 13)
    P = pbar(lmax, np.cos(theta))
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            ref = sps.sph_harm_y(l, m, theta, 0.0).real
            np.testing.assert_allclose(P[m][l - m], ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("nlat", [8, 32, 96])
def test_pbar_discrete_orthonormality(nlat):
    # 2 pi sum_j w_j Pbar_lm Pbar_l'm = delta_ll' (GL exact for degree <= 2 nlat - 1)
    g = Grid(nlat)
    P = g.pbar()
    for m in range(g.lmax + 1):
        G = 2 * np.pi * (P[m] * g.w) @ P[m].T
        assert np.abs(G - np.eye(G.shape[0])).max() < 1e-13, m


def test_pbar_orthonormality_720_sampled():
    # the full-size table, including the sectoral values that underflow in FP64
    g = Grid(720)
    P = g.pbar()
    for m in (0, 1, 100, 359, 600, 718, 719):
        G = 2 * np.pi * (P[m] * g.w) @ P[m].T
        assert np.abs(G - np.eye(G.shape[0])).max() < 1e-12, m


def test_legendre_series_matches_numpy():
    z = np.linspace(-1, 1, 41)
    ser = legendre_series(30, z)
    for l in range(31):
        c = np.zeros(l + 1)
        c[l] = 1.0
        np.testing.assert_allclose(ser[l], np.polynomial.legendre.legval(z, c), atol=1e-13)
