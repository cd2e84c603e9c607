"""GPU parity on the equiangular Clenshaw-Curtis grid (App. C.1; the paper's runtime
grid, Sec. 4.1) against the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sht as osht, sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32, potentials_err, assert_s, BF16_S_LIMIT

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

CC = shot.SHOT_QUAD_CLENSHAW_CURTIS
TOL_SHT = {"fp32": 2e-5, "bf16x3": 2e-4, "tf32x3": 2e-5}
PREC = {"fp32": shot.SHOT_FP32, "bf16x3": shot.SHOT_BF16X3, "tf32x3": shot.SHOT_TF32X3}


@pytest.fixture(scope="module")
def grid_cache():
    cache = {}

    def get(nlat, nlon=None, lmax=-1, prec="fp32", mode=shot.SHOT_TABLE):
        key = (nlat, nlon, lmax, prec, mode)
        if key not in cache:
            g = shot.shot_grid_init_quad(CC, nlat, nlon, lmax, PREC[prec], mode)
            og = OGrid(nlat, nlon, None if lmax == -1 else lmax, quadrature="cc")
            cache[key] = (g, og)
        return cache[key]
    yield get
    for g, _ in cache.values():
        shot.shot_grid_free(g)


@pytest.mark.parametrize("nlat,nlon", [(3, 6), (4, 8), (9, 18), (64, 128), (181, 375), (512, 1024)])
def test_cc_nodes_weights_match_oracle(grid_cache, nlat, nlon):
    # both sides are FP64; the device sums the closed form, the oracle the Chebyshev
    # interpolation form: agreement to a few ulps of the largest weight
    g, og = grid_cache(nlat, nlon)
    x, w, a = shot.shot_grid_nodes(g)
    assert x[0] == 1.0 and x[-1] == -1.0
    assert np.all(x == -x[::-1])
    assert np.max(np.abs(x - og.x)) < 4e-16
    assert np.max(np.abs(w - og.w)) < 1e-14 * og.w.max()
    assert abs(a.sum() * og.nlon - 4 * np.pi) < 1e-12


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("nlat,nlon,lmax,nf,t", [(3, 6, -1, 1, 0.1), (9, 18, -1, 3, 0.02),
                                                 (32, 64, -1, 40, 1e-2), (65, 135, -1, 5, 2.5e-3),
                                                 (33, 72, 16, 2, 0.01), (128, 256, -1, 3, 1e-3)])
def test_cc_heat_apply_matches_oracle(grid_cache, prec, nlat, nlon, lmax, nf, t):
    g, og = grid_cache(nlat, nlon, lmax, prec)
    f, f64 = f32(np.random.default_rng(11 * nlat + nf).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, t, torch.from_numpy(f).cuda(), out)
    ref = osht.heat_apply(og, f64, t)
    assert rel_max(out.cpu().numpy(), ref) < TOL_SHT[prec]


@pytest.mark.parametrize("nlat,nlon,nf", [(17, 36, 2), (64, 128, 3)])
def test_cc_recurrence_mode_matches_oracle(grid_cache, nlat, nlon, nf):
    # the pole rings hold Pbar_lm = 0 for every m >= 1: the seeds must skip them
    g, og = grid_cache(nlat, nlon, mode=shot.SHOT_RECURRENCE)
    f, f64 = f32(np.random.default_rng(nlat).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, 0.01, torch.from_numpy(f).cuda(), out)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 0.01)) < TOL_SHT["fp32"]


def test_cc_round_trip_below_half_band(grid_cache):
    # 2 lmax <= nlat - 1: analysis inverts synthesis exactly in exact arithmetic
    g, og = grid_cache(33, 64, 16)
    L = og.lmax + 1
    rng = np.random.default_rng(3)
    c = np.tril(rng.normal(size=(2, L, L))) + 1j * np.tril(rng.normal(size=(2, L, L)))
    c[..., :, 0] = c[..., :, 0].real
    f64 = osht.synthesis(og, c)
    f, _ = f32(f64)
    ct = torch.empty((2, L, L, 2), device="cuda")
    shot.shot_sht_analysis(g, torch.from_numpy(f).cuda(), ct)
    got = ct.cpu().numpy()
    scale = np.abs(c).max()
    assert np.abs(got[..., 0] - c.real).max() < 1e-5 * scale
    assert np.abs(got[..., 1] - c.imag).max() < 1e-5 * scale


def _fields(og, seed, npairs, masses=False):
    p, q = inputs.pairs("paper_uniform", seed, npairs, og.x, og.nlon, og.a_ring, masses=masses)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    return torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), p64, q64


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("nlat,nlon,eps,tau,T", [(17, 36, 0.1, math.inf, 40), (32, 64, 0.1, 1.0, 40)])
def test_cc_sinkhorn_matches_oracle(grid_cache, prec, nlat, nlon, eps, tau, T):
    g, og = grid_cache(nlat, nlon, prec=prec)
    unb = not math.isinf(tau)
    pt, qt, p, q = _fields(og, 3000 + nlat, 2, masses=unb)
    rc, r = shot.shot_sinkhorn(g, pt, qt, eps, tau, max_iter=T, tol=0.0, check_every=10)
    ref = sk.sinkhorn(og, p, q, eps, tau, T=T, delta=0.0, C=10)
    assert rc == 0 and np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    # BF16x3's per-product error (<= 3 * 2^-18) compounds over the T fixed-point
    # iterations, ~T * 1.5e-5 in u (6e-4 at T = 40); S, the metric's quantity, is held to
    # 1e-4 in test_cc_divergence_matches_oracle
    tol = 5e-4 if prec == "bf16x3" else 1e-5
    u, v = r["u"].cpu().numpy(), r["v"].cpu().numpy()
    assert potentials_err(og, eps, u, v, ref["phi"], ref["psi"]) < tol
    np.testing.assert_allclose(r["mass_pi"], ref["mass_pi"], rtol=1e-4 if prec == "bf16x3" else 1e-5)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32x3"])
def test_cc_divergence_matches_oracle(grid_cache, prec):
    g, og = grid_cache(24, prec=prec)
    pt, qt, p, q = _fields(og, 4024, 2)
    rc, r = shot.shot_divergence(g, pt, qt, 0.1, max_iter=60, tol=0.0, check_every=10)
    ref = sk.divergence(og, p, q, 0.1, T=60, delta=0.0, C=10)
    assert np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    tol = 1e-4 if prec == "bf16x3" else 1e-5
    assert_s(r["S"], ref["S"], ref["runs"]["ot"][:2], tol, limited_by=BF16_S_LIMIT if prec == "bf16x3" else None)
    assert np.all(r["S"] > 0)


def test_cc_512_full_size_heat_apply(grid_cache):
    # the paper's largest equiangular grid (L = 512 rings, 1024 longitudes)
    g, og = grid_cache(512)
    f, f64 = f32(np.random.default_rng(512).uniform(size=(2, 512, 1024)))
    out = torch.empty((2, 512, 1024), device="cuda")
    shot.shot_heat_apply(g, 1e-4, torch.from_numpy(f).cuda(), out)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 1e-4)) < TOL_SHT["fp32"]


def test_cc_rejects_bad_arguments():
    with pytest.raises(shot.ShotError):
        shot.shot_grid_init_quad(CC, 2, 4)       # needs nlat >= 3
    with pytest.raises(shot.ShotError):
        shot.shot_grid_init_quad(7, 8, 16)       # unknown quadrature
