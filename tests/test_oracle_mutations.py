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


def _fails(pin, *args):
    """True when the pin test function fails (raises AssertionError) on the mutated oracle."""
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


def test_cc_endpoint_halving_dropped_caught(monkeypatch):
    # Clenshaw-Curtis weights without halving the end terms of the cosine sums, planted in
    # the oracle; the exactness pin of tests/test_oracle_cc.py must fail
    from oracle import grid as ogrid
    from tests import test_oracle_cc as pins
    good = ogrid.clenshaw_curtis

    def bad(nlat):
        x, _ = good(nlat)
        N = nlat - 1
        j = np.arange(N + 1)
        w = np.zeros(N + 1)
        for k in range(0, N + 1, 2):
            w += (2.0 / N) * np.cos(np.pi * k * j / N) * (2.0 / (1.0 - k * k)) * (0.5 if k in (0, N) else 1.0)
        return x, w
    monkeypatch.setattr(ogrid, "clenshaw_curtis", bad)
    monkeypatch.setattr(pins, "clenshaw_curtis", bad)
    assert _fails(pins.test_cc_exactness_symmetry_positivity, 7)
    assert _fails(pins.test_cc_textbook_closed_forms)


def test_normaliser_without_jacobian_caught(monkeypatch):
    # C(eps) integrated without the sin(theta) surface element, planted in the oracle; the
    # small-eps series pin and the large-eps limit pin must fail
    from scipy import integrate
    from oracle import convolution as cv
    from tests import test_oracle_convolution as pins

    def bad(eps):
        return 2 * np.pi * integrate.quad(lambda th: np.exp(-th * th / eps), 0.0, np.pi, limit=200)[0]
    monkeypatch.setattr(cv, "gibbs_normaliser", bad)
    assert _fails(pins.test_normaliser_small_eps_series, 1e-2)
    assert _fails(pins.test_normaliser_large_eps_limit)


def test_gibbs_without_area_weights_caught(monkeypatch):
    # matrix convolution that forgets a_j, planted in the oracle; the row-sum pin must fail
    from oracle import convolution as cv
    from tests import test_oracle_convolution as pins

    def bad(grid, f, eps, rows=1024):
        X = grid.xyz.reshape(-1, 3)
        F = np.asarray(f, dtype=np.float64).reshape(-1, X.shape[0])
        d = cv.geodesic(X[:, None, :], X[None, :, :])
        return (F @ np.exp(-d * d / eps).T).reshape(f.shape)
    monkeypatch.setattr(cv, "gibbs_apply", bad)
    assert _fails(pins.test_row_sums_match_normaliser_on_fine_grid, 0.5)


def test_healpix_longitude_offset_dropped_caught(monkeypatch):
    # rings without their half-pixel longitude offset, planted in the oracle; the
    # base-resolution geometry pin must fail
    from oracle import healpix as ohp
    from tests import test_oracle_healpix as pins
    good = ohp.ring_geometry

    def bad(nside):
        z, npx, phi0 = good(nside)
        return z, npx, np.zeros_like(phi0)
    monkeypatch.setattr(ohp, "ring_geometry", bad)
    monkeypatch.setattr(pins, "ring_geometry", bad)
    assert _fails(pins.test_base_resolution_geometry)


def test_unweighted_l1_marginal_error_caught(monkeypatch):
    # the L1 check without the area weights, planted in the oracle; the hand-computed pin
    # of tests/test_oracle_sinkhorn.py must fail
    from tests import test_oracle_sinkhorn as pins

    def bad(grid, u, kv, p, norm="l2"):
        ax = tuple(range(1, p.ndim))
        r = u * kv - p
        if norm == "l2":
            return np.sqrt(np.sum(r * r, axis=ax)) / np.sqrt(np.sum(p * p, axis=ax))
        return np.sum(np.abs(r), axis=ax) / np.sum(p, axis=ax)
    monkeypatch.setattr(sk, "marginal_error", bad)
    assert _fails(pins.test_l1_marginal_error_hand_computed)
    assert _fails(pins.test_l1_marginal_error_on_a_grid_equals_the_weighted_sum)


def test_mutation_helpers_pass_unmutated():
    # the same pins pass on the oracle as committed (so a failure above is the mutation's)
    from tests import test_oracle_cc, test_oracle_convolution, test_oracle_healpix, test_oracle_sinkhorn
    assert not _fails(test_oracle_cc.test_cc_exactness_symmetry_positivity, 7)
    assert not _fails(test_oracle_cc.test_cc_textbook_closed_forms)
    assert not _fails(test_oracle_convolution.test_normaliser_small_eps_series, 1e-2)
    assert not _fails(test_oracle_convolution.test_normaliser_large_eps_limit)
    assert not _fails(test_oracle_convolution.test_row_sums_match_normaliser_on_fine_grid, 0.5)
    assert not _fails(test_oracle_healpix.test_base_resolution_geometry)
    assert not _fails(test_oracle_sinkhorn.test_l1_marginal_error_hand_computed)
    assert not _fails(test_oracle_sinkhorn.test_l1_marginal_error_on_a_grid_equals_the_weighted_sum)
