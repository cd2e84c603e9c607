"""GPU parity on HEALPix grids (App. C.1 "HEALPix"; the paper's climate grid is nside = 64)
against the FP64 oracle, through the C ABI.  Fields are flat [batch][12 nside^2] arrays in
ring order."""
import math

import numpy as np
import pytest

from oracle.healpix import HealpixGrid
from oracle import sinkhorn as sk, convolution as cv
from tests.gpu_util import rel_max, f32, potentials_err, assert_s, BF16_S_LIMIT

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

PREC = {"fp32": shot.SHOT_FP32, "bf16x3": shot.SHOT_BF16X3, "tf32x3": shot.SHOT_TF32X3}
TOL = {"fp32": 2e-5, "bf16x3": 2e-4, "tf32x3": 2e-5}


def _grid(nside, lmax=-1, prec="fp32", mode=shot.SHOT_TABLE):
    return shot.shot_grid_init_healpix(nside, lmax, PREC[prec], mode), HealpixGrid(nside, None if lmax == -1 else lmax)


@pytest.mark.parametrize("nside", [1, 2, 8, 64])
def test_geometry_matches_oracle(nside):
    g, og = _grid(nside)
    assert shot.shot_grid_npix(g) == og.npix == 12 * nside * nside
    ln, off, ph = shot.shot_grid_rings(g)
    np.testing.assert_array_equal(ln, og.npx)
    np.testing.assert_array_equal(off, og.off[:-1])
    np.testing.assert_allclose(ph, og.phi0, rtol=0, atol=1e-15)
    x, w, a = shot.shot_grid_nodes(g)
    np.testing.assert_allclose(x, og.z, rtol=0, atol=1e-15)
    np.testing.assert_allclose(a, og.area, rtol=1e-15)
    info = shot.shot_grid_info(g)
    assert info["nlat"] == 4 * nside - 1 and info["lmax"] == 3 * nside - 1
    shot.shot_grid_free(g)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("nside,lmax,nf,t", [(1, -1, 1, 0.2), (2, -1, 3, 0.05), (4, -1, 5, 0.02),
                                             (8, 11, 2, 0.01), (16, -1, 24, 3e-3)])
def test_heat_apply_matches_oracle(prec, nside, lmax, nf, t):
    g, og = _grid(nside, lmax, prec)
    f, f64 = f32(np.random.default_rng(nside + nf).uniform(size=(nf, og.npix)))
    out = torch.empty((nf, og.npix), device="cuda")
    shot.shot_heat_apply(g, t, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_free(g)
    ref = og.heat_apply(f64[:, None, :], t)[:, 0]
    assert rel_max(out.cpu().numpy(), ref) < TOL[prec]


def test_recurrence_mode_matches_oracle():
    g, og = _grid(8, mode=shot.SHOT_RECURRENCE)
    f, f64 = f32(np.random.default_rng(8).uniform(size=(3, og.npix)))
    out = torch.empty((3, og.npix), device="cuda")
    shot.shot_heat_apply(g, 0.01, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_free(g)
    assert rel_max(out.cpu().numpy(), og.heat_apply(f64[:, None, :], 0.01)[:, 0]) < TOL["fp32"]


def test_climate_grid_nside64_full_size():
    g, og = _grid(64)
    f, f64 = f32(np.random.default_rng(64).uniform(size=(2, og.npix)))
    out = torch.empty((2, og.npix), device="cuda")
    shot.shot_heat_apply(g, 2.5e-3, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_free(g)
    assert rel_max(out.cpu().numpy(), og.heat_apply(f64[:, None, :], 2.5e-3)[:, 0]) < TOL["fp32"]


def _pairs(og, seed, npairs, masses=False):
    rng = np.random.default_rng(seed)
    p, q = rng.uniform(0.2, 1.0, size=(2, npairs, og.npix))
    p /= np.sum(og.area * p, axis=1)[:, None]
    q /= np.sum(og.area * q, axis=1)[:, None]
    if masses:
        p *= rng.uniform(0.5, 2.0, size=npairs)[:, None]
        q *= rng.uniform(0.5, 2.0, size=npairs)[:, None]
    return f32(p), f32(q)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("nside,eps,tau,T", [(4, 0.1, math.inf, 40), (8, 0.05, 1.0, 40)])
def test_sinkhorn_matches_oracle(prec, nside, eps, tau, T):
    g, og = _grid(nside, prec=prec)
    (p32, p), (q32, q) = _pairs(og, 100 + nside, 2, masses=not math.isinf(tau))
    rc, r = shot.shot_sinkhorn(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                               max_iter=T, tol=0.0, check_every=10)
    shot.shot_grid_free(g)
    ref = sk.sinkhorn(og, p[:, None, :], q[:, None, :], eps, tau, T=T, delta=0.0, C=10)
    assert rc == 0 and np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    tol = 1e-5 if prec == "fp32" else 5e-4
    u = r["u"].cpu().numpy()[:, None, :]
    v = r["v"].cpu().numpy()[:, None, :]
    assert potentials_err(og, eps, u, v, ref["phi"], ref["psi"]) < tol
    np.testing.assert_allclose(r["mass_pi"], ref["mass_pi"], rtol=1e-5 if prec == "fp32" else 1e-4)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_divergence_matches_oracle(prec):
    # the paper's climate setting in kind: eps = 0.01 is too sharp for nside 8, so 0.05
    g, og = _grid(8, prec=prec)
    (p32, p), (q32, q) = _pairs(og, 808, 2)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), 0.05,
                                 max_iter=60, tol=0.0, check_every=10)
    shot.shot_grid_free(g)
    ref = sk.divergence(og, p[:, None, :], q[:, None, :], 0.05, T=60, delta=0.0, C=10)
    assert np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    tol = 1e-5 if prec == "fp32" else 1e-4
    assert_s(r["S"], ref["S"], ref["runs"]["ot"][:2], tol, limited_by=BF16_S_LIMIT if prec == "bf16x3" else None)
    assert np.all(r["S"] > 0)


def test_gibbs_and_comparison_on_healpix():
    g, og = _grid(8)
    f, f64 = f32(np.random.default_rng(3).uniform(size=(2, og.npix)))
    out = torch.empty((2, og.npix), device="cuda")
    shot.shot_gibbs_apply(g, 0.05, torch.from_numpy(f).cuda(), out)
    torch.cuda.synchronize()
    assert rel_max(out.cpu().numpy(), cv.gibbs_apply(og, f64[:, None, :], 0.05)[:, 0]) < 2e-5
    mae = shot.shot_conv_compare(g, 0.05, torch.from_numpy(f).cuda())
    ref = cv.conv_mae(og, f64[:, None, :], 0.05)
    scale = float(np.abs(cv.gibbs_apply(og, f64[:, None, :], 0.05)).max())
    assert np.all(np.abs(mae - ref) <= 1e-3 * ref + 2e-5 * scale)
    shot.shot_grid_free(g)


def test_bad_nside_is_rejected():
    with pytest.raises(shot.ShotError):
        shot.shot_grid_init_healpix(0)


@pytest.mark.parametrize("nside,eps,tau,T,ck", [(4, 0.2, math.inf, 30, 7), (4, 0.2, 1.0, 30, 10)])
def test_unrolled_gradient_matches_oracle_fd(nside, eps, tau, T, ck):
    """The gradient of S (Sec. 4.2) on a HEALPix grid: directional derivatives of the unrolled
    adjoint against central differences of the oracle's S after the same T iterations."""
    from oracle.gradient import fd_directional
    g, og = _grid(nside)
    try:
        bal = math.isinf(tau)
        (p32, p), (q32, q) = _pairs(og, 300 + nside, 2, masses=not bal)
        rc, r = shot.shot_divergence_grad(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                                          max_iter=T, checkpoint_every=ck, mode=shot.SHOT_GRAD_UNROLLED)
        assert rc >= 0 and np.all(r["status"] >= 0)
        grad = r["grad"].cpu().numpy().astype(np.float64)
        rng = np.random.default_rng(17)
        for b in range(2):
            dirs = []
            for _ in range(3):
                d = p[b] * rng.normal(size=og.npix)
                if bal:
                    d -= np.mean(d)   # equal areas: keeps the mass
                d *= np.sqrt(np.sum(p[b] * p[b]) / np.sum(d * d))
                dirs.append(d[None, :])
            dirs = np.array(dirs)
            fd = fd_directional(og, p[b][None, :], q[b][None, :], eps, tau, T, dirs, h=1e-5)
            got = np.array([np.sum(grad[b] * d[0]) for d in dirs])
            assert np.max(np.abs(got - fd)) <= 1e-4 * np.max(np.abs(fd)), (got, fd)
    finally:
        shot.shot_grid_free(g)


def test_regional_rms_matches_oracle():
    from oracle.regional import regional_rms
    g, og = _grid(16)
    try:
        rng = np.random.default_rng(16)
        grad = (og.area * rng.normal(size=(3, og.npix))).astype(np.float32)
        got = shot.shot_regional_rms(g, torch.from_numpy(grad).cuda())
        ref = regional_rms(og, grad.astype(np.float64)[:, None, :])
        np.testing.assert_allclose(got, ref, rtol=1e-5)
    finally:
        shot.shot_grid_free(g)
