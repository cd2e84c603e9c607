"""Pins of the oracle's HEALPix grid and SHT (App. C.1 "HEALPix")."""
import numpy as np
import pytest
import scipy.special as sps

from oracle.healpix import HealpixGrid, ring_geometry
from oracle import dense, sinkhorn as sk


def test_base_resolution_geometry():
    # Nside = 1: the 12 base pixels, 4 per ring at z = 2/3, 0, -2/3; longitudes
    # pi/4 + k pi/2 on the two outer rings and k pi/2 on the equator
    z, npx, phi0 = ring_geometry(1)
    np.testing.assert_allclose(z, [2 / 3, 0, -2 / 3], atol=1e-15)
    np.testing.assert_array_equal(npx, [4, 4, 4])
    g = HealpixGrid(1)
    ph = np.sort(g.phi.reshape(3, 4) % (2 * np.pi), axis=1)
    np.testing.assert_allclose(ph[0], np.pi / 4 + np.pi / 2 * np.arange(4), atol=1e-15)
    np.testing.assert_allclose(ph[1], np.pi / 2 * np.arange(4), atol=1e-15)
    np.testing.assert_allclose(ph[2], ph[0], atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 64])
def test_ring_structure(nside):
    z, npx, phi0 = ring_geometry(nside)
    assert len(z) == 4 * nside - 1
    assert npx.sum() == 12 * nside * nside
    assert np.all(np.diff(z) < 0)
    np.testing.assert_array_equal(z, -z[::-1])
    np.testing.assert_array_equal(npx, npx[::-1])
    np.testing.assert_array_equal(phi0, phi0[::-1])
    # polar cap ring i has 4 i pixels; the belt 4 nside
    np.testing.assert_array_equal(npx[: nside - 1], 4 * np.arange(1, nside))
    assert np.all(npx[nside - 1: 3 * nside] == 4 * nside)
    # polar cap: the area above ring i's centre latitude is ... pixel centres sit at
    # z = 1 - i^2/(3 nside^2): the cap of the first i rings holds 2 i (i + 1) pixels
    # = fraction 2 i (i+1) / (12 nside^2) of the sphere, between the centre colatitudes
    # of rings i and i + 1
    for i in range(1, nside - 1):
        frac = 2 * i * (i + 1) / (12 * nside * nside)
        zb = 1 - 2 * frac                   # z of the cap boundary holding that area
        assert z[i] < zb < z[i - 1]


def test_low_degree_quadrature_is_approximate():
    # no sampling theorem: sum_p a Y_lm(p) is small but not zero for l >= 1, and shrinks
    # with nside
    errs = []
    for nside in (4, 8, 16):
        g = HealpixGrid(nside)
        th = np.arccos(g.z[g.ring_of])
        e = max(abs(np.sum(g.area * sps.sph_harm_y(l, 0, th, g.phi).real)) for l in (2, 4, 6))
        errs.append(e)
    assert errs[0] > errs[1] > errs[2] > 0


@pytest.mark.parametrize("nside,t", [(1, 0.3), (2, 0.05), (4, 0.02)])
def test_sht_heat_equals_dense_matrix(nside, t):
    # the addition theorem holds on any node set: SHT path == H diag(a) for any vector
    g = HealpixGrid(nside)
    f = np.random.default_rng(nside).normal(size=(2, 1, g.npix))
    ref = dense.dense_apply(dense.kernel_matrix(g, t), f)
    np.testing.assert_allclose(g.heat_apply(f, t), ref, atol=1e-12 * np.abs(ref).max())


def test_heat_symmetric_in_area_inner_product():
    # without a sampling theorem K_t Y_lm = e^{-t l(l+1)} Y_lm holds only up to quadrature
    # aliasing; what stays exact is the symmetry of K = H diag(a) in the a-weighted
    # inner product
    g = HealpixGrid(4)
    rng = np.random.default_rng(2)
    f, h = rng.uniform(size=(2, 1, 1, g.npix))
    kf, kh = g.heat_apply(f, 0.01), g.heat_apply(h, 0.01)
    assert abs(np.sum(g.area * h * kf) - np.sum(g.area * f * kh)) < 1e-13 * abs(np.sum(g.area * h * kf))


def test_sinkhorn_on_healpix():
    g = HealpixGrid(4)
    rng = np.random.default_rng(9)
    p, q = rng.uniform(0.5, 1.5, size=(2, 1, 1, g.npix))
    p /= np.sum(g.area * p)
    q /= np.sum(g.area * q)
    r = sk.divergence(g, p, q, 0.1, T=300, delta=1e-10, C=10)
    assert r["status"][0] == sk.OK
    assert r["S"][0] > 0
    rpp = sk.divergence(g, p, p, 0.1, T=300, delta=1e-10, C=10)
    assert abs(rpp["S"][0]) < 1e-12


def test_regional_bands_on_healpix():
    """Sec. 4.2 / App. E on HEALPix: with equal-area pixels, a band's pixel fraction approaches
    its exact area fraction (sin 23.5 deg for the Tropics, sin 10 deg for the ITCZ,
    (sin 60 - sin 30)/2 for each mid-latitude band, (1 - sin 66.5)/2 for the Arctic) to
    within the ring spacing; a constant field form has zero RMS everywhere, and the
    hemisphere sign field (mean zero on the symmetric grid) has RMS 1 in every band."""
    from oracle.regional import regional_rms, band_masks
    og = HealpixGrid(32)
    lat = og.lat_deg
    s = lambda d: np.sin(np.radians(d))
    exact = [s(23.5), s(10.0), (s(60.0) - s(30.0)) / 2, (s(60.0) - s(30.0)) / 2, (1 - s(66.5)) / 2]
    for mask, e in zip(band_masks(lat), exact):
        assert abs(mask.mean() - e) < 2.0 / og.nside
    a = og.a
    const = 3.0 * a[None]
    np.testing.assert_allclose(regional_rms(og, const), 0.0, atol=1e-12)
    # sign(lat) has mean zero (the grid is symmetric, the equator ring is 0): RMS 1 in the
    # bands off the equator; in the two equatorial bands the equator ring's zeros leave
    # sqrt(1 - n_eq / n_band)
    sign = np.sign(lat)[None] * a[None]
    got = regional_rms(og, sign)[0]
    eq = np.abs(lat) < 1e-9
    for r, mask in enumerate(band_masks(lat)):
        want = np.sqrt(1.0 - np.sum(mask & eq) / np.sum(mask))
        assert abs(got[r] - want) < 1e-12
    assert np.sum(eq) == 4 * og.nside
