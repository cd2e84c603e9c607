"""GPU parity of the on-the-fly recurrence mode (SHOT_RECURRENCE, FP32) against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sht as osht
from oracle import sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32, potentials_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL_SHT = 2e-5


@pytest.fixture(scope="module")
def grid_cache():
    cache = {}

    def get(nlat, nlon=None, lmax=-1):
        key = (nlat, nlon, lmax)
        if key not in cache:
            g = shot.shot_grid_init(nlat, nlon, lmax, shot.SHOT_FP32, shot.SHOT_RECURRENCE)
            cache[key] = (g, OGrid(nlat, nlon, None if lmax == -1 else lmax))
        return cache[key]
    yield get
    for g, _ in cache.values():
        shot.shot_grid_free(g)


@pytest.mark.parametrize("nlat,nlon,lmax,nf", [(8, None, -1, 1), (33, 72, -1, 3), (64, None, -1, 24),
                                               (180, None, -1, 2), (20, 45, 13, 3), (32, None, -1, 30)])
def test_recurrence_analysis_matches_oracle(grid_cache, nlat, nlon, lmax, nf):
    g, og = grid_cache(nlat, nlon, lmax)
    L = og.lmax + 1
    f, f64 = f32(np.random.default_rng(nlat + nf).normal(size=(nf, og.nlat, og.nlon)))
    c = torch.empty((nf, L, L, 2), device="cuda")
    shot.shot_sht_analysis(g, torch.from_numpy(f).cuda(), c)
    got = c.cpu().numpy()
    ref = osht.analysis(og, f64)
    assert rel_max(got[..., 0], ref.real) < TOL_SHT
    assert rel_max(got[..., 1], ref.imag) < TOL_SHT


@pytest.mark.parametrize("nlat,nf", [(8, 1), (64, 5), (180, 2)])
def test_recurrence_synthesis_matches_oracle(grid_cache, nlat, nf):
    g, og = grid_cache(nlat)
    L = og.lmax + 1
    rng = np.random.default_rng(500 + nlat)
    c = rng.normal(size=(nf, L, L, 2)).astype(np.float32)
    iu = np.triu_indices(L, 1)
    c[:, iu[0], iu[1], :] = 0
    c[:, :, 0, 1] = 0
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_sht_synthesis(g, torch.from_numpy(c).cuda(), out)
    ref = osht.synthesis(og, c[..., 0].astype(np.float64) + 1j * c[..., 1].astype(np.float64))
    assert rel_max(out.cpu().numpy(), ref) < TOL_SHT


def test_recurrence_heat_apply_720_matches_oracle_and_table(grid_cache):
    g, og = grid_cache(720)
    nf = 3
    f, f64 = f32(np.random.default_rng(7201).uniform(size=(nf, 720, 1440)))
    ft = torch.from_numpy(f).cuda()
    out = torch.empty((nf, 720, 1440), device="cuda")
    shot.shot_heat_apply(g, 1e-4, ft, out)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 1e-4)) < TOL_SHT
    gt = shot.shot_grid_init(720)
    try:
        out_t = torch.empty_like(out)
        shot.shot_heat_apply(gt, 1e-4, ft, out_t)
        assert rel_max(out.cpu().numpy(), out_t.cpu().numpy()) < TOL_SHT
    finally:
        shot.shot_grid_free(gt)


def test_recurrence_sinkhorn_matches_oracle(grid_cache):
    g, og = grid_cache(32)
    p, q = inputs.pairs("paper_uniform", 1032, 3, og.x, og.nlon, og.a_ring)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_sinkhorn(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), 0.1, max_iter=60,
                               tol=0.0, check_every=10)
    ref = sk.sinkhorn(og, p64, q64, 0.1, T=60, delta=0.0, C=10)
    assert rc == 0
    assert potentials_err(og, 0.1, r["u"].cpu().numpy(), r["v"].cpu().numpy(), ref["phi"], ref["psi"]) < 1e-5
