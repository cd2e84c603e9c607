"""Pins of the oracle's heat-vs-matrix convolution comparison (App. "Convolution on S^2")."""
import numpy as np
import pytest

from oracle.grid import Grid
from oracle import convolution as cv
from paper_2605_18389_gb300 import inputs


def test_geodesic_special_cases():
    x = np.array([0.0, 0.0, 1.0])
    assert cv.geodesic(x, x) == 0.0
    assert abs(cv.geodesic(x, -x) - np.pi) < 1e-15
    assert abs(cv.geodesic(x, np.array([1.0, 0.0, 0.0])) - np.pi / 2) < 1e-15
    # small angles: exact where arccos(cos d) loses half the digits
    d = 1e-7
    y = np.array([np.sin(d), 0.0, np.cos(d)])
    assert abs(cv.geodesic(x, y) - d) < 1e-20


@pytest.mark.parametrize("eps", [1e-3, 3e-3, 1e-2])
def test_normaliser_small_eps_series(eps):
    # sin th = th - th^3/6 + ...: C = 2 pi (eps/2 - eps^2/12 + eps^3/120 + ...) up to e^{-pi^2/eps}
    series = 2 * np.pi * (eps / 2 - eps ** 2 / 12 + eps ** 3 / 120)
    assert abs(cv.gibbs_normaliser(eps) - series) < 2 * np.pi * eps ** 4


def test_normaliser_large_eps_limit():
    # exp(-th^2/eps) -> 1: C -> 4 pi; first correction -(2 pi / eps) int th^2 sin th = -(2 pi / eps)(pi^2 - 4)
    eps = 1e4
    c = cv.gibbs_normaliser(eps)
    assert abs(c - (4 * np.pi - 2 * np.pi * (np.pi ** 2 - 4) / eps)) < 1e-6


@pytest.mark.parametrize("eps", [0.05, 0.5])
def test_row_sums_match_normaliser_on_fine_grid(eps):
    g = Grid(48, quadrature="cc")
    one = np.ones((1, g.nlat, g.nlon))
    k1 = cv.gibbs_apply(g, one, eps)
    assert np.abs(k1 / cv.gibbs_normaliser(eps) - 1.0).max() < 1e-6


def test_matrix_convolution_is_a_weighted_symmetric():
    g = Grid(12, quadrature="cc")
    rng = np.random.default_rng(1)
    f, h = rng.uniform(size=(2, g.nlat, g.nlon))
    kf, kh = cv.gibbs_apply(g, f, 0.1), cv.gibbs_apply(g, h, 0.1)
    assert abs(np.sum(g.a * h * kf) - np.sum(g.a * f * kh)) < 1e-13 * np.sum(g.a * h * kf)


def test_rescaled_heat_kernel_matches_gibbs_near_diagonal():
    # C(eps) H_{eps/4}(x, y) ~ exp(-d^2/eps) sqrt(d / sin d) (1 + O(eps)) for small d
    g = Grid(64)
    eps = 0.01
    X = g.xyz.reshape(-1, 3)
    i = g.nlat // 3 * g.nlon
    d = cv.geodesic(X[i][None, :], X)
    from oracle.legendre import legendre_series   # one row of the heat matrix by the addition theorem
    z = np.clip(X @ X[i], -1.0, 1.0)
    Hrow = sum((2 * l + 1) / (4 * np.pi) * np.exp(-eps / 4 * l * (l + 1.0)) * Pl
               for l, Pl in enumerate(legendre_series(g.lmax, z)))
    near = (d > 0) & (d < 0.15)
    ratio = cv.gibbs_normaliser(eps) * Hrow[near] / (np.exp(-d[near] ** 2 / eps) * np.sqrt(d[near] / np.sin(d[near])))
    assert np.all(np.abs(ratio - 1.0) < 0.02)


def test_mae_decreases_with_resolution():
    # the paper's qualitative result: finer grids, smaller discrepancy (at eps = 0.01 the
    # discretisation dominates; at eps >= 0.1 the Varadhan approximation error does, and
    # the curve flattens)
    eps = 0.01
    maes = []
    for L in (8, 16, 32):
        g = Grid(L, quadrature="cc")
        f = inputs.field("vmf_k10", 42, g.x, g.nlon, g.a_ring)[None]
        maes.append(float(cv.conv_mae(g, f, eps)[0]))
    assert maes[0] > maes[1] > maes[2]
