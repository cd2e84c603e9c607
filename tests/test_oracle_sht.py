"""Pins of the oracle's DFT, SHT and heat operator (Sec. 3.2, App. B, App. C.1)."""
import numpy as np
import pytest
import scipy.special as sps

from oracle.grid import Grid
from oracle import sht, dense
from oracle.legendre import legendre_series


def test_dft_pure_modes():
    g = Grid(6, nlon=15, lmax=5)   # odd nlon, several radices
    for m0 in range(g.lmax + 1):
        f = np.cos(m0 * g.phi)[None, :] * np.ones((g.nlat, 1))
        F = sht.ring_dft(g, f)
        exp = np.zeros(g.lmax + 1)
        exp[m0] = g.nlon if m0 == 0 else g.nlon / 2.0
        np.testing.assert_allclose(F[0].real, exp, atol=1e-12)
        np.testing.assert_allclose(F[0].imag, 0, atol=1e-12)
        f = np.sin(m0 * g.phi)[None, :] * np.ones((g.nlat, 1))
        F = sht.ring_dft(g, f)
        exp = np.zeros(g.lmax + 1)
        if m0:
            exp[m0] = -g.nlon / 2.0
        np.testing.assert_allclose(F[0].imag, exp, atol=1e-12)


def test_dft_matches_numpy_fft():
    g = Grid(12)
    f = np.random.default_rng(1).normal(size=(3, g.nlat, g.nlon))
    np.testing.assert_allclose(sht.ring_dft(g, f), np.fft.rfft(f, axis=-1)[..., : g.lmax + 1],
                               atol=1e-12)


def _random_coeffs(g, rng, B=2):
    c = rng.normal(size=(B, g.lmax + 1, g.lmax + 1)) + 1j * rng.normal(size=(B, g.lmax + 1, g.lmax + 1))
    c = np.tril(c)                 # l >= m
    c[..., :, 0] = c[..., :, 0].real   # real field: c_l0 real
    return c


@pytest.mark.parametrize("nlat", [4, 17, 64])
def test_sht_round_trip(nlat):
    g = Grid(nlat)
    c = _random_coeffs(g, np.random.default_rng(nlat))
    f = sht.synthesis(g, c)
    c2 = sht.analysis(g, f)
    assert np.abs(c2 - c).max() < 1e-12 * max(1.0, np.abs(c).max())


def _real_ylm_scipy(g, l, m):
    th, ph = np.meshgrid(g.theta, g.phi, indexing="ij")
    return sps.sph_harm_y(l, m, th, ph).real


@pytest.mark.parametrize("l,m", [(0, 0), (1, 0), (1, 1), (5, 3), (12, 7), (15, 15)])
def test_heat_eigenfunctions(l, m):
    # K_t Y_lm = exp(-t l(l+1)) Y_lm (Sec. 3.2), Y from scipy (independent of the table)
    g = Grid(16)
    t = 0.013
    y = _real_ylm_scipy(g, l, m)
    ky = sht.heat_apply(g, y, t)
    np.testing.assert_allclose(ky, np.exp(-t * l * (l + 1)) * y, atol=1e-13)


def test_heat_preserves_constant_mass_and_is_symmetric():
    g = Grid(32)
    rng = np.random.default_rng(3)
    v, w = rng.uniform(size=(2, g.nlat, g.nlon))
    t = 0.01
    np.testing.assert_allclose(sht.heat_apply(g, np.ones((g.nlat, g.nlon)), t), 1.0, atol=1e-13)
    kv = sht.heat_apply(g, v, t)
    kw = sht.heat_apply(g, w, t)
    a = g.a
    assert abs(np.sum(a * kv) - np.sum(a * v)) < 1e-13 * np.sum(a * v)
    assert abs(np.sum(a * w * kv) - np.sum(a * v * kw)) < 1e-13 * abs(np.sum(a * w * kv))


@pytest.mark.parametrize("nlat,t", [(4, 0.1), (8, 0.01), (16, 0.02), (24, 0.003)])
def test_sht_equals_dense_heat_matrix(nlat, t):
    # addition theorem: SHT path == H diag(a) for ANY grid vector
    g = Grid(nlat)
    f = np.random.default_rng(nlat).normal(size=(2, g.nlat, g.nlon))
    K = dense.kernel_matrix(g, t)
    ref = dense.dense_apply(K, f)
    np.testing.assert_allclose(sht.heat_apply(g, f, t), ref, atol=1e-12 * np.abs(ref).max())


def test_varadhan_trend():
    # -4t log H_t(x,y) -> d(x,y)^2 as t -> 0 (Sec. 2, Varadhan); lmax 719 keeps the
    # truncation (~e^{-t lmax^2}) far below e^{-d^2/4t}, and d^2/4t <= 15 keeps H
    # well above the FP64 rounding floor of the series (~1e-12).
    lmax = 719
    d = np.linspace(0.05, 0.24, 11)
    errs = []
    for t in (1e-2, 3e-3, 1e-3):
        H = sum((2 * l + 1) / (4 * np.pi) * np.exp(-t * l * (l + 1)) * Pl
                for l, Pl in enumerate(legendre_series(lmax, np.cos(d))))
        assert np.all(H > 0)
        errs.append(np.max(np.abs(-4 * t * np.log(H) - d * d)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.03


def test_heat_kernel_negative_lobes_exist():
    # App. C.4: the truncated kernel can be negative when t^{-1/2} >~ L
    from oracle.grid import Grid as G
    g = G(32)
    H = dense.heat_matrix(g, 1e-2)
    assert (H < 0).mean() > 0.1
