"""GPU parity of the recurrence mode (SHOT_RECURRENCE: no table, O(n) memory) against the FP64 oracle.

FP32 grids regenerate Pbar by the double-float recurrence on the CUDA cores; TF32X3 grids
regenerate it in shared memory from FP32 checkpoints every 16 degrees and contract on the
tensor cores (tcgen05 kind::tf32).  Both are held to the FP32 bars of the table path.
"""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sht as osht
from oracle import sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32, potentials_err, assert_s

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL_SHT = 2e-5
# BF16X3 grids in recurrence mode run the TF32x3 recurrence kernels: the same bars
PREC = {"fp32": shot.SHOT_FP32, "tf32x3": shot.SHOT_TF32X3, "bf16x3": shot.SHOT_BF16X3}
PRECS = ["fp32", "tf32x3", "bf16x3"]


@pytest.fixture(scope="module")
def grid_cache():
    cache = {}

    def get(nlat, nlon=None, lmax=-1, prec="fp32"):
        key = (nlat, nlon, lmax, prec)
        if key not in cache:
            g = shot.shot_grid_init(nlat, nlon, lmax, PREC[prec], shot.SHOT_RECURRENCE)
            cache[key] = (g, OGrid(nlat, nlon, None if lmax == -1 else lmax))
        return cache[key]
    yield get
    for g, _ in cache.values():
        shot.shot_grid_free(g)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nlat,nlon,lmax,nf", [(8, None, -1, 1), (33, 72, -1, 3), (64, None, -1, 24),
                                               (180, None, -1, 2), (20, 45, 13, 3), (32, None, -1, 30),
                                               (40, None, -1, 70)])
def test_recurrence_analysis_matches_oracle(grid_cache, nlat, nlon, lmax, nf, prec):
    g, og = grid_cache(nlat, nlon, lmax, prec)
    L = og.lmax + 1
    f, f64 = f32(np.random.default_rng(nlat + nf).normal(size=(nf, og.nlat, og.nlon)))
    c = torch.empty((nf, L, L, 2), device="cuda")
    shot.shot_sht_analysis(g, torch.from_numpy(f).cuda(), c)
    got = c.cpu().numpy()
    ref = osht.analysis(og, f64)
    shot.shot_grid_check(g)
    assert rel_max(got[..., 0], ref.real) < TOL_SHT
    assert rel_max(got[..., 1], ref.imag) < TOL_SHT


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nlat,nf", [(8, 1), (64, 5), (180, 2), (33, 70)])
def test_recurrence_synthesis_matches_oracle(grid_cache, nlat, nf, prec):
    g, og = grid_cache(nlat, prec=prec)
    L = og.lmax + 1
    rng = np.random.default_rng(500 + nlat)
    c = rng.normal(size=(nf, L, L, 2)).astype(np.float32)
    iu = np.triu_indices(L, 1)
    c[:, iu[0], iu[1], :] = 0
    c[:, :, 0, 1] = 0
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_sht_synthesis(g, torch.from_numpy(c).cuda(), out)
    ref = osht.synthesis(og, c[..., 0].astype(np.float64) + 1j * c[..., 1].astype(np.float64))
    shot.shot_grid_check(g)
    assert rel_max(out.cpu().numpy(), ref) < TOL_SHT


@pytest.mark.parametrize("prec", PRECS)
def test_recurrence_heat_apply_720_matches_oracle_and_table(grid_cache, prec):
    g, og = grid_cache(720, prec=prec)
    nf = 3
    f, f64 = f32(np.random.default_rng(7201).uniform(size=(nf, 720, 1440)))
    ft = torch.from_numpy(f).cuda()
    out = torch.empty((nf, 720, 1440), device="cuda")
    shot.shot_heat_apply(g, 1e-4, ft, out)
    shot.shot_grid_check(g)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 1e-4)) < TOL_SHT
    gt = shot.shot_grid_init(720, None, -1, PREC[prec])
    try:
        out_t = torch.empty_like(out)
        shot.shot_heat_apply(gt, 1e-4, ft, out_t)
        # the BF16X3 table grid carries ~2^-17 per table entry (its transforms' bar is 1e-4)
        assert rel_max(out.cpu().numpy(), out_t.cpu().numpy()) < (1e-4 if prec == "bf16x3" else TOL_SHT)
    finally:
        shot.shot_grid_free(gt)


@pytest.mark.parametrize("prec", PRECS)
def test_recurrence_sinkhorn_matches_oracle(grid_cache, prec):
    g, og = grid_cache(32, prec=prec)
    p, q = inputs.pairs("paper_uniform", 1032, 3, og.x, og.nlon, og.a_ring)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_sinkhorn(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), 0.1, max_iter=60,
                               tol=0.0, check_every=10)
    ref = sk.sinkhorn(og, p64, q64, 0.1, T=60, delta=0.0, C=10)
    assert rc == 0
    assert potentials_err(og, 0.1, r["u"].cpu().numpy(), r["v"].cpu().numpy(), ref["phi"], ref["psi"]) < 1e-5


@pytest.mark.parametrize("nlat,eps,tau,T", [(32, 0.1, math.inf, 60), (64, 0.02, 1.0, 40), (33, 0.1, math.inf, 40)])
def test_tf32_recurrence_divergence_matches_oracle(grid_cache, nlat, eps, tau, T):
    g, og = grid_cache(nlat, prec="tf32x3")
    unb = not math.isinf(tau)
    p, q = inputs.pairs("paper_uniform", 3300 + nlat, 2, og.x, og.nlon, og.a_ring, masses=unb)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                                 max_iter=T, tol=0.0, check_every=10)
    ref = sk.divergence(og, p64, q64, eps, tau, T=T, delta=0.0, C=10)
    assert rc == 0 and np.all(r["status"] == 0)
    np.testing.assert_allclose(r["ot3"], ref["runs"]["ot"], rtol=1e-5)
    assert_s(r["S"], ref["S"], ref["runs"]["ot"][:2], 1e-4)
    assert_s(r["S_dual"], ref["S_dual"], ref["runs"]["ot"][:2], 1e-4)


def test_tf32_recurrence_healpix_and_cc_heat_apply():
    """The checkpointed recurrence on the other node sets: Clenshaw-Curtis (poles included)
    and HEALPix rings, against the oracle's heat operator."""
    from oracle.healpix import HealpixGrid
    gc = shot.shot_grid_init_quad(shot.SHOT_QUAD_CLENSHAW_CURTIS, 49, 100, -1, shot.SHOT_TF32X3, shot.SHOT_RECURRENCE)
    gh = shot.shot_grid_init_healpix(8, -1, shot.SHOT_TF32X3, shot.SHOT_RECURRENCE)
    try:
        oc = OGrid(49, 100, quadrature="cc")
        f, f64 = f32(np.random.default_rng(49).uniform(size=(3, 49, 100)))
        out = torch.empty((3, 49, 100), device="cuda")
        shot.shot_heat_apply(gc, 0.01, torch.from_numpy(f).cuda(), out)
        shot.shot_grid_check(gc)
        assert rel_max(out.cpu().numpy(), osht.heat_apply(oc, f64, 0.01)) < TOL_SHT
        oh = HealpixGrid(8)
        fh, fh64 = f32(np.random.default_rng(8).uniform(size=(2, oh.npix)))
        outh = torch.empty((2, oh.npix), device="cuda")
        shot.shot_heat_apply(gh, 0.01, torch.from_numpy(fh).cuda(), outh)
        shot.shot_grid_check(gh)
        assert rel_max(outh.cpu().numpy(), oh.heat_apply(fh64[:, None, :], 0.01)[:, 0]) < TOL_SHT
    finally:
        shot.shot_grid_free(gc)
        shot.shot_grid_free(gh)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_tf32_recurrence_keeps_no_table(prec):
    """No table: the recurrence grid at 720 x 1440 holds checkpoints of 95 MB (a quarter of the
    table's entries) where the table grids hold the 0.38 GB FP32 table and its 0.75 GB
    transposed copy (TF32X3) or the bf16 hi/lo table (BF16X3)."""
    free0, _ = torch.cuda.mem_get_info()
    g = shot.shot_grid_init(720, None, -1, PREC[prec], shot.SHOT_RECURRENCE)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    shot.shot_grid_free(g)
    assert free0 - free1 < 200 * 2 ** 20, (free0 - free1) / 2 ** 20
