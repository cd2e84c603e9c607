"""GPU parity of the tcgen05 BF16x3 Legendre path against the FP64 oracle (C ABI).

Target: potentials and S within 1e-4 of the oracle (split-precision bar); transforms
within 1e-4 of the largest output.
"""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sht as osht
from oracle import sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32, potentials_err, assert_s, BF16_S_LIMIT

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module")
def grid_cache():
    cache = {}

    def get(nlat, nlon=None, lmax=-1):
        key = (nlat, nlon, lmax)
        if key not in cache:
            g = shot.shot_grid_init(nlat, nlon, lmax, shot.SHOT_BF16X3)
            cache[key] = (g, OGrid(nlat, nlon, None if lmax == -1 else lmax))
        return cache[key]
    yield get
    for g, _ in cache.values():
        shot.shot_grid_free(g)


@pytest.mark.parametrize("nlat,nlon,lmax,nf", [(8, None, -1, 1), (32, None, -1, 3), (33, 72, -1, 2),
                                               (64, None, -1, 24), (180, None, -1, 5), (20, 45, 13, 3),
                                               (32, None, -1, 128)])
def test_bf16x3_analysis_matches_oracle(grid_cache, nlat, nlon, lmax, nf):
    g, og = grid_cache(nlat, nlon, lmax)
    L = og.lmax + 1
    f, f64 = f32(np.random.default_rng(nlat + nf).normal(size=(nf, og.nlat, og.nlon)))
    c = torch.empty((nf, L, L, 2), device="cuda")
    shot.shot_sht_analysis(g, torch.from_numpy(f).cuda(), c)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    got = c.cpu().numpy()
    ref = osht.analysis(og, f64)
    assert rel_max(got[..., 0], ref.real) < TOL
    assert rel_max(got[..., 1], ref.imag) < TOL


@pytest.mark.parametrize("nlat,nlon,lmax,nf", [(8, None, -1, 1), (32, None, -1, 5), (180, None, -1, 2),
                                               (20, 45, 13, 3)])
def test_bf16x3_synthesis_matches_oracle(grid_cache, nlat, nlon, lmax, nf):
    g, og = grid_cache(nlat, nlon, lmax)
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
    assert rel_max(out.cpu().numpy(), ref) < TOL


@pytest.mark.parametrize("nlat,nf,t", [(16, 2, 0.05), (64, 24, 2.5e-3), (180, 3, 1e-3)])
def test_bf16x3_heat_apply_matches_oracle(grid_cache, nlat, nf, t):
    g, og = grid_cache(nlat)
    f, f64 = f32(np.random.default_rng(nlat).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, t, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, t)) < TOL


def test_bf16x3_heat_apply_720_full_size(grid_cache):
    g, og = grid_cache(720)
    nf = 24
    f, f64 = f32(np.random.default_rng(7200).uniform(size=(nf, 720, 1440)))
    out = torch.empty((nf, 720, 1440), device="cuda")
    shot.shot_heat_apply(g, 1e-4, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    got = out.cpu().numpy()
    ref = osht.heat_apply(og, f64[:3], 1e-4)   # the oracle on a sample of the batch
    assert rel_max(got[:3], ref) < TOL


@pytest.mark.parametrize("nlat,eps,tau,T", [(32, 0.1, math.inf, 60), (32, 0.1, 1.0, 60), (64, 0.02, 0.1, 30)])
def test_bf16x3_sinkhorn_matches_oracle(grid_cache, nlat, eps, tau, T):
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
    assert potentials_err(og, eps, u, v, ref["phi"], ref["psi"]) < TOL
    np.testing.assert_allclose(r["ot"], ref["ot"], rtol=TOL)


@pytest.mark.parametrize("nlat,eps,tau,T,tol", [(32, 0.1, math.inf, 600, 1e-5), (64, 0.02, 10.0, 40, 0.0)])
def test_bf16x3_divergence_matches_oracle(grid_cache, nlat, eps, tau, T, tol):
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
    assert_s(r["S"], ref["S"], ot_pq, TOL, limited_by=BF16_S_LIMIT)
    assert_s(r["S_dual"], ref["S_dual"], ot_pq, TOL, limited_by=BF16_S_LIMIT)


@pytest.mark.parametrize("nlat,nf", [(96, 24), (64, 40), (40, 64)])
def test_bf16x3_analysis_pipeline_depths_agree(monkeypatch, nlat, nf):
    """The tensor-core analysis at every pipeline depth (SHOT_TC_STAGES=1..4; the split spectra
    operand in its own ring of two buffers) matches the oracle, and the depths agree bit for
    bit: the K order of the accumulation does not depend on the depth.  Depths that do not fit
    in shared memory for the field count fall back to the deepest one that does."""
    og = OGrid(nlat)
    f, f64 = f32(np.random.default_rng(nlat + 7 * nf).uniform(size=(nf, og.nlat, og.nlon)))
    ref = osht.heat_apply(og, f64, 2e-3)
    outs = []
    for depth in ("1", "2", "3", "4"):
        monkeypatch.setenv("SHOT_TC_STAGES", depth)
        g = shot.shot_grid_init(nlat, None, -1, shot.SHOT_BF16X3)
        try:
            out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
            shot.shot_heat_apply(g, 2e-3, torch.from_numpy(f).cuda(), out)
            shot.shot_grid_check(g)   # no bounded device-side wait expired
            outs.append(out.cpu().numpy())
        finally:
            shot.shot_grid_free(g)
    assert rel_max(outs[0], ref) < TOL
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
