"""GPU parity of the tcgen05 TF32x3 Legendre path against the FP64 oracle (C ABI).

The tf32 hi/lo split with three products is exact to ~2^-21 per product, so the bars are
the FP32 path's: transforms within 2e-5 of the largest output, potentials within 1e-5,
S within 1e-5 relative plus 4 * 2^-20 |OT(p, q)|.
"""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle.gradient import envelope
from oracle import sht as osht
from oracle import sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32, s_err, potentials_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL_SHT = 2e-5
TOL_PHI = 1e-5
TOL_S = 1e-5
QUAD = {"gl": (shot.SHOT_QUAD_GAUSS_LEGENDRE, "gl"), "cc": (shot.SHOT_QUAD_CLENSHAW_CURTIS, "cc")}


@pytest.fixture(scope="module")
def grid_cache():
    cache = {}

    def get(nlat, nlon=None, lmax=-1, quad="gl"):
        key = (nlat, nlon, lmax, quad)
        if key not in cache:
            q, oq = QUAD[quad]
            g = shot.shot_grid_init_quad(q, nlat, nlon, lmax, shot.SHOT_TF32X3)
            cache[key] = (g, OGrid(nlat, nlon, None if lmax == -1 else lmax, quadrature=oq))
        return cache[key]
    yield get
    for g, _ in cache.values():
        shot.shot_grid_free(g)


def test_tf32x3_grid_reports_precision(grid_cache):
    g, _ = grid_cache(16)
    assert shot.shot_grid_info(g)["precision"] == shot.SHOT_TF32X3


# sizes span one and several 128-row tiles and 32-node K chunks with ragged tails
@pytest.mark.parametrize("nlat,nlon,lmax,nf,quad", [(8, None, -1, 1, "gl"), (32, None, -1, 3, "gl"),
                                                    (33, 72, -1, 2, "gl"), (64, None, -1, 24, "gl"),
                                                    (180, None, -1, 5, "gl"), (20, 45, 13, 3, "gl"),
                                                    (32, None, -1, 128, "gl"), (48, None, -1, 40, "gl"),
                                                    (65, 135, -1, 4, "cc"),
                                                    (300, None, -1, 2, "gl")])
def test_tf32x3_analysis_matches_oracle(grid_cache, nlat, nlon, lmax, nf, quad):
    g, og = grid_cache(nlat, nlon, lmax, quad)
    L = og.lmax + 1
    f, f64 = f32(np.random.default_rng(nlat + nf).normal(size=(nf, og.nlat, og.nlon)))
    c = torch.empty((nf, L, L, 2), device="cuda")
    shot.shot_sht_analysis(g, torch.from_numpy(f).cuda(), c)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    got = c.cpu().numpy()
    ref = osht.analysis(og, f64)
    assert rel_max(got[..., 0], ref.real) < TOL_SHT
    assert rel_max(got[..., 1], ref.imag) < TOL_SHT


@pytest.mark.parametrize("nlat,nlon,lmax,nf,quad", [(8, None, -1, 1, "gl"), (32, None, -1, 5, "gl"),
                                                    (180, None, -1, 2, "gl"), (20, 45, 13, 3, "gl"),
                                                    (65, 135, -1, 4, "cc"), (64, None, -1, 100, "gl"),
                                                    (48, None, -1, 64, "gl")])
def test_tf32x3_synthesis_matches_oracle(grid_cache, nlat, nlon, lmax, nf, quad):
    g, og = grid_cache(nlat, nlon, lmax, quad)
    L = og.lmax + 1
    rng = np.random.default_rng(300 + nlat)
    c = rng.normal(size=(nf, L, L, 2)).astype(np.float32)
    iu = np.triu_indices(L, 1)
    c[:, iu[0], iu[1], :] = 0
    c[:, :, 0, 1] = 0
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_sht_synthesis(g, torch.from_numpy(c).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    ref = osht.synthesis(og, c[..., 0].astype(np.float64) + 1j * c[..., 1].astype(np.float64))
    assert rel_max(out.cpu().numpy(), ref) < TOL_SHT


@pytest.mark.parametrize("nlat,nf,t,quad", [(16, 2, 0.05, "gl"), (64, 24, 2.5e-3, "gl"), (180, 3, 1e-3, "gl"),
                                            (125, 5, 1e-3, "cc")])
def test_tf32x3_heat_apply_matches_oracle(grid_cache, nlat, nf, t, quad):
    g, og = grid_cache(nlat, quad=quad)
    f, f64 = f32(np.random.default_rng(nlat).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, t, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, t)) < TOL_SHT


def test_tf32x3_heat_apply_720_full_size(grid_cache):
    g, og = grid_cache(720)
    nf = 24
    f, f64 = f32(np.random.default_rng(7200).uniform(size=(nf, 720, 1440)))
    out = torch.empty((nf, 720, 1440), device="cuda")
    shot.shot_heat_apply(g, 1e-4, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    got = out.cpu().numpy()
    ref = osht.heat_apply(og, f64[:3], 1e-4)   # the oracle on a sample of the batch
    assert rel_max(got[:3], ref) < TOL_SHT


def test_tf32x3_more_accurate_than_bf16x3():
    """The same heat application on TF32X3, BF16X3 and FP32 grids: the TF32 split is the
    closer to the FP64 oracle by a wide margin (2^-21 against 2^-16 per product); both
    carry the FP32 error of the ring transforms, which bounds the ratio."""
    og = OGrid(96)
    f, f64 = f32(np.random.default_rng(96).uniform(size=(4, og.nlat, og.nlon)))
    ref = osht.heat_apply(og, f64, 1e-3)
    errs = {}
    for name, prec in (("tf32x3", shot.SHOT_TF32X3), ("bf16x3", shot.SHOT_BF16X3), ("fp32", shot.SHOT_FP32)):
        g = shot.shot_grid_init(96, None, -1, prec)
        try:
            out = torch.empty((4, og.nlat, og.nlon), device="cuda")
            shot.shot_heat_apply(g, 1e-3, torch.from_numpy(f).cuda(), out)
            shot.shot_grid_check(g)   # no bounded device-side wait expired
            errs[name] = rel_max(out.cpu().numpy(), ref)
        finally:
            shot.shot_grid_free(g)
    assert errs["tf32x3"] < errs["bf16x3"] / 4, errs
    assert errs["tf32x3"] < TOL_SHT, errs


@pytest.mark.parametrize("nlat,eps,tau,T", [(32, 0.1, math.inf, 60), (32, 0.1, 1.0, 60), (64, 0.02, 0.1, 30)])
def test_tf32x3_sinkhorn_matches_oracle(grid_cache, nlat, eps, tau, T):
    g, og = grid_cache(nlat)
    unb = not math.isinf(tau)
    p, q = inputs.pairs("paper_uniform", 1000 + nlat, 3, og.x, og.nlon, og.a_ring, masses=unb)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_sinkhorn(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                               max_iter=T, tol=0.0, check_every=10)
    ref = sk.sinkhorn(og, p64, q64, eps, tau, T=T, delta=0.0, C=10)
    assert rc == 0 and np.all(r["status"] == 0)
    u, v = r["u"].cpu().numpy(), r["v"].cpu().numpy()
    assert potentials_err(og, eps, u, v, ref["phi"], ref["psi"]) < TOL_PHI
    np.testing.assert_allclose(r["ot"], ref["ot"], rtol=TOL_PHI)


@pytest.mark.parametrize("nlat,eps,tau,T,tol", [(32, 0.1, math.inf, 600, 1e-5), (64, 0.02, 10.0, 40, 0.0)])
def test_tf32x3_divergence_matches_oracle(grid_cache, nlat, eps, tau, T, tol):
    g, og = grid_cache(nlat)
    unb = not math.isinf(tau)
    p, q = inputs.pairs("paper_uniform", 2000 + nlat, 2, og.x, og.nlon, og.a_ring, masses=unb)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                                 max_iter=T, tol=tol, check_every=10)
    ref = sk.divergence(og, p64, q64, eps, tau, T=T, delta=tol, C=10)
    assert np.all(r["status"] == ref["status"])
    ot_pq = ref["runs"]["ot"][:2]
    assert np.all(s_err(r["S"], ref["S"], ot_pq, TOL_S) <= 1.0)
    assert np.all(s_err(r["S_dual"], ref["S_dual"], ot_pq, TOL_S) <= 1.0)


def test_tf32x3_envelope_gradient_matches_oracle():
    # converged problem: the envelope formula applies; dS/dp is defined modulo c * a, so
    # the field forms are compared centred by their area means
    nlat, eps, T = 16, 1.0, 400
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat, None, -1, shot.SHOT_TF32X3)
    try:
        p, q = inputs.pairs("vmf3", 77, 1, og.x, og.nlon, og.a_ring)
        p32, p64 = f32(p)
        q32, q64 = f32(q)
        rc, r = shot.shot_divergence_grad(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps,
                                          max_iter=T, mode=shot.SHOT_GRAD_ENVELOPE)
        assert rc >= 0
        ref = envelope(og, p64[0], q64[0], eps, math.inf, T, delta=0.0, C=0)
        got = r["grad"].cpu().numpy()[0].astype(np.float64)
        a = og.a
        gf, rf = got / a, ref / a
        gf -= np.sum(a * gf) / np.sum(a)
        rf -= np.sum(a * rf) / np.sum(a)
        assert np.max(np.abs(gf - rf)) <= 1e-4 * np.max(np.abs(rf))
    finally:
        shot.shot_grid_free(g)
