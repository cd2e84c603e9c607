"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each."""
import numpy as np
import pytest

from oracle.grid import Grid
from oracle import sht, sinkhorn as sk, dense
from paper_2605_18389_gb300 import inputs


def _eigen_residual(g, t=0.02):
    import scipy.special as sps
    th, ph = np.meshgrid(g.theta, g.phi, indexing="ij")
    worst = 0.0
    for l, m in [(3, 1), (7, 4), (9, 0)]:
        y = sps.sph_harm_y(l, m, th, ph).real
        worst = max(worst, np.abs(sht.heat_apply(g, y, t) - np.exp(-t * l * (l + 1)) * y).max())
    return worst


def test_pins_pass_unmutated():
    g = Grid(12)
    assert _eigen_residual(g) < 1e-13


def test_wrong_eigenvalue_caught(monkeypatch):
    g = Grid(12)
    monkeypatch.setattr(sht, "heat_multipliers",
                        lambda t, lmax: np.exp(-t * np.arange(lmax + 1) * np.arange(lmax + 1)))
    assert _eigen_residual(g) > 1e-3


def test_wrong_quadrature_weight_caught(monkeypatch):
    g = Grid(12)
    g.a_ring = g.w.copy()          # forgot the 2 pi / nlon longitude factor
    one = sht.heat_apply(g, np.ones((g.nlat, g.nlon)), 0.01)
    assert np.abs(one - 1).max() > 1e-2


def test_dropped_factor_two_in_synthesis_caught(monkeypatch):
    g = Grid(10)
    orig = sht.ring_idft

    def bad(grid, gm):
        e = np.exp(2j * np.pi * (np.outer(np.arange(grid.nlon), np.arange(grid.lmax + 1))
                                 % grid.nlon) / grid.nlon).T
        return (gm @ e).real
    monkeypatch.setattr(sht, "ring_idft", bad)
    f = np.random.default_rng(0).normal(size=(g.nlat, g.nlon))
    K = dense.kernel_matrix(g, 0.05)
    assert np.abs(sht.heat_apply(g, f, 0.05) - dense.dense_apply(K, f)).max() > 1e-3
    monkeypatch.setattr(sht, "ring_idft", orig)


def test_wrong_recurrence_index_caught(monkeypatch):
    from oracle import legendre
    orig = legendre.pbar

    def bad(lmax, x):
        P = orig(lmax, x)
        for m in range(len(P)):        # off-by-one in l for the seeds' neighbours
            if P[m].shape[0] > 2:
                P[m][2:] = P[m][1:-1].copy()
        return P
    g = Grid(12)
    monkeypatch.setattr(legendre, "pbar", bad)
    g._pbar = None
    P = g.pbar()
    G = 2 * np.pi * (P[3] * g.w) @ P[3].T
    assert np.abs(G - np.eye(G.shape[0])).max() > 1e-2


def test_wrong_gauge_direction_caught(monkeypatch):
    g = Grid(12)
    p, q = inputs.pairs("paper_uniform", 1, 1, g.x, g.nlon, g.a_ring)
    orig_sum = np.sum

    # emulate u *= s, v /= s by feeding 1/s to the gauge
    class Flip:
        calls = 0

    def fake_sum(x, *a, **k):
        r = orig_sum(x, *a, **k)
        if k.get("axis") == (1, 2) and getattr(x, "ndim", 0) == 3 and Flip.calls == 0:
            Flip.calls = 1
            return 1.0 / r
        return r
    monkeypatch.setattr(sk.np, "sum", fake_sum)
    r = sk.sinkhorn(g, p, q, eps=0.1, T=1, C=0)
    monkeypatch.setattr(sk.np, "sum", orig_sum)
    assert abs(r["u"].sum() - 1.0) > 1e-3


def test_cc_endpoint_halving_dropped_caught():
    # Clenshaw-Curtis without halving the end terms of the cosine sums: the pins'
    # exactness check (int x^2 = 2/3 on 9 nodes) must fail
    from oracle.grid import clenshaw_curtis
    x, _ = clenshaw_curtis(9)
    N = 8
    j = np.arange(N + 1)
    w = np.zeros(N + 1)
    for k in range(0, N + 1, 2):
        w += (2.0 / N) * np.cos(np.pi * k * j / N) * (2.0 / (1.0 - k * k)) * (0.5 if k in (0, N) else 1.0)
    assert abs(np.sum(w * x ** 2) - 2.0 / 3.0) > 1e-3


def test_normaliser_without_jacobian_caught(monkeypatch):
    # C(eps) integrated without the sin(theta) surface element: the small-eps series pin
    # (C = pi eps - pi eps^2 / 6 + ...) must fail
    from scipy import integrate
    eps = 1e-2
    bad = 2 * np.pi * integrate.quad(lambda th: np.exp(-th * th / eps), 0.0, np.pi)[0]
    series = 2 * np.pi * (eps / 2 - eps ** 2 / 12 + eps ** 3 / 120)
    assert abs(bad - series) > 1e-3


def test_gibbs_without_area_weights_caught():
    # matrix convolution that forgets a_j: its row sums no longer approach C(eps)
    from oracle import convolution as cv
    g = Grid(24, quadrature="cc")
    X = g.xyz.reshape(-1, 3)
    d = cv.geodesic(X[:1, None, :], X[None, :, :])[0]
    bad_rowsum = np.exp(-d * d / 0.5).sum()
    assert abs(bad_rowsum / cv.gibbs_normaliser(0.5) - 1.0) > 1e-2


def test_healpix_longitude_offset_dropped_caught():
    # rings without their half-pixel longitude offset: the base-resolution pin fails
    from oracle.healpix import HealpixGrid
    g = HealpixGrid(1)
    bad = 2 * np.pi * (np.arange(g.npix) - g.off[g.ring_of]) / g.npx[g.ring_of]
    ph = np.sort(bad.reshape(3, 4) % (2 * np.pi), axis=1)
    assert np.abs(ph[0] - (np.pi / 4 + np.pi / 2 * np.arange(4))).max() > 0.5
