"""GPU parity of the fused per-order tensor-core heat kernel (BF16x3 analysis and synthesis
of each (m, parity) block in one CTA, the table read a second time as an MN-major operand)
against the FP64 oracle and against the two-kernel tensor-core path (C ABI)."""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sht as osht
from oracle import sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32, s_err_prec, potentials_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL = 1e-4


def _grid(monkeypatch, fused, nlat, nlon=None, lmax=-1, quad=shot.SHOT_QUAD_GAUSS_LEGENDRE):
    monkeypatch.setenv("SHOT_FUSED_HEAT", "1" if fused else "0")
    return shot.shot_grid_init_quad(quad, nlat, nlon, lmax, shot.SHOT_BF16X3)


@pytest.mark.parametrize("nlat,nlon,lmax,nf,t", [(8, None, -1, 1, 0.1), (32, None, -1, 3, 0.01),
                                                 (33, 72, -1, 2, 0.02), (65, 135, -1, 24, 3e-3),
                                                 (180, None, -1, 5, 1e-3), (20, 45, 13, 3, 0.05),
                                                 (256, None, -1, 32, 1e-3), (64, None, -1, 40, 3e-3)])
def test_fused_heat_apply_matches_oracle(monkeypatch, nlat, nlon, lmax, nf, t):
    # nf = 40 exceeds the fused kernel's 32 fields: the two-kernel path runs instead
    g = _grid(monkeypatch, True, nlat, nlon, lmax)
    og = OGrid(nlat, nlon, None if lmax == -1 else lmax)
    f, f64 = f32(np.random.default_rng(17 * nlat + nf).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, t, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    shot.shot_grid_free(g)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, t)) < TOL


@pytest.mark.parametrize("nlat,nf", [(24, 6), (96, 24)])
def test_fused_agrees_with_two_kernel_path(monkeypatch, nlat, nf):
    og = OGrid(nlat)
    f, _ = f32(np.random.default_rng(nlat).uniform(size=(nf, og.nlat, og.nlon)))
    outs = []
    for fused in (True, False):
        g = _grid(monkeypatch, fused, nlat)
        out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
        shot.shot_heat_apply(g, 2e-3, torch.from_numpy(f).cuda(), out)
        shot.shot_grid_check(g)   # no bounded device-side wait expired
        shot.shot_grid_free(g)
        outs.append(out.cpu().numpy())
    # same products and the same accumulation order per tile: agreement far below the tolerance
    assert rel_max(outs[0], outs[1]) < 1e-6


def test_fused_cc_grid(monkeypatch):
    g = _grid(monkeypatch, True, 33, 72, -1, shot.SHOT_QUAD_CLENSHAW_CURTIS)
    og = OGrid(33, 72, quadrature="cc")
    f, f64 = f32(np.random.default_rng(5).uniform(size=(4, 33, 72)))
    out = torch.empty((4, 33, 72), device="cuda")
    shot.shot_heat_apply(g, 0.01, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    shot.shot_grid_free(g)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 0.01)) < TOL


@pytest.mark.parametrize("nlat,eps,tau,T", [(32, 0.1, math.inf, 60), (48, 0.05, 1.0, 40)])
def test_fused_divergence_matches_oracle(monkeypatch, nlat, eps, tau, T):
    g = _grid(monkeypatch, True, nlat)
    og = OGrid(nlat)
    unb = not math.isinf(tau)
    p, q = inputs.pairs("paper_uniform", 6000 + nlat, 2, og.x, og.nlon, og.a_ring, masses=unb)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                                 max_iter=T, tol=0.0, check_every=10)
    shot.shot_grid_free(g)
    ref = sk.divergence(og, p64, q64, eps, tau, T=T, delta=0.0, C=10)
    assert np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    assert np.all(s_err_prec(r["S"], ref["S"], ref["runs"]["ot"][:2], TOL, "bf16x3") <= 1.0)


def test_fused_720_full_size(monkeypatch):
    g = _grid(monkeypatch, True, 720)
    og = OGrid(720)
    f, f64 = f32(np.random.default_rng(720).uniform(size=(3, 720, 1440)))
    out = torch.empty((3, 720, 1440), device="cuda")
    shot.shot_heat_apply(g, 1e-4, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    shot.shot_grid_free(g)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 1e-4)) < TOL


@pytest.mark.parametrize("fused,split", [(False, False), (False, True), (True, False), (True, True)])
def test_spectra_formats_agree_with_oracle(monkeypatch, fused, split):
    # the solver's spectra as FP32 (split in shared memory) or as bf16 hi/lo written by the
    # inverse DFT (TMA'd as an MN-major operand), with the two-kernel or the fused path
    monkeypatch.setenv("SHOT_SPLIT_SPECTRA", "1" if split else "0")
    g = _grid(monkeypatch, fused, 40)
    og = OGrid(40)
    p, q = inputs.pairs("paper_uniform", 7040, 3, og.x, og.nlon, og.a_ring)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), 0.05,
                                 max_iter=50, tol=0.0, check_every=10)
    shot.shot_grid_free(g)
    ref = sk.divergence(og, p64, q64, 0.05, T=50, delta=0.0, C=10)
    assert np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    assert np.all(s_err_prec(r["S"], ref["S"], ref["runs"]["ot"][:3], TOL, "bf16x3") <= 1.0)


@pytest.mark.parametrize("nlat,nf", [(36, 3), (96, 24)])
def test_transposed_analysis_matches_oracle(monkeypatch, nlat, nf):
    # the opt-in transposed analysis (fields on M, degree rows on N): same heat operator
    monkeypatch.setenv("SHOT_ANA_TRANSPOSED", "1")
    g = _grid(monkeypatch, False, nlat)
    og = OGrid(nlat)
    f, f64 = f32(np.random.default_rng(nlat * 3).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, 3e-3, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    p, q = inputs.pairs("paper_uniform", 9000 + nlat, 2, og.x, og.nlon, og.a_ring)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), 0.05,
                                 max_iter=40, tol=0.0, check_every=10)
    shot.shot_grid_free(g)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 3e-3)) < TOL
    ref = sk.divergence(og, p64, q64, 0.05, T=40, delta=0.0, C=10)
    assert np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    assert np.all(s_err_prec(r["S"], ref["S"], ref["runs"]["ot"][:2], TOL, "bf16x3") <= 1.0)


def _merged_grid(monkeypatch, merged, nlat, nlon=None, lmax=-1):
    monkeypatch.setenv("SHOT_MERGED_HEAT", "1" if merged else "0")
    return shot.shot_grid_init(nlat, nlon, lmax, shot.SHOT_BF16X3)


@pytest.mark.parametrize("nlat,nlon,lmax,nf,t", [(8, None, -1, 1, 0.1), (33, 72, -1, 2, 0.02),
                                                 (64, None, -1, 24, 3e-3), (180, None, -1, 5, 1e-3),
                                                 (20, 45, 13, 3, 0.05), (256, None, -1, 32, 1e-3)])
def test_merged_heat_apply_matches_oracle(monkeypatch, nlat, nlon, lmax, nf, t):
    """Analysis and synthesis of each block in one persistent CTA (SHOT_MERGED_HEAT=1)."""
    g = _merged_grid(monkeypatch, True, nlat, nlon, lmax)
    og = OGrid(nlat, nlon, None if lmax == -1 else lmax)
    f, f64 = f32(np.random.default_rng(23 * nlat + nf).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, t, torch.from_numpy(f).cuda(), out)
    shot.shot_grid_check(g)   # no bounded device-side wait expired
    shot.shot_grid_free(g)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, t)) < TOL


@pytest.mark.parametrize("nlat,nf", [(96, 24), (180, 7), (720, 24)])
def test_merged_agrees_with_two_kernel_path_bitwise(monkeypatch, nlat, nf):
    """The merged kernel issues the two-kernel path's MMAs in the same K order and the same
    epilogue arithmetic: the heat applications agree bit for bit."""
    og = OGrid(nlat)
    f = np.random.default_rng(nlat).uniform(size=(nf, og.nlat, og.nlon)).astype(np.float32)
    outs = []
    for merged in (True, False):
        g = _merged_grid(monkeypatch, merged, nlat)
        out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
        shot.shot_heat_apply(g, 1e-3, torch.from_numpy(f).cuda(), out)
        shot.shot_grid_check(g)
        outs.append(out.cpu().numpy())
        shot.shot_grid_free(g)
    np.testing.assert_array_equal(outs[0], outs[1])


def test_merged_divergence_matches_oracle(monkeypatch):
    nlat, eps, tau, T = 64, 0.02, 1.0, 30
    g = _merged_grid(monkeypatch, True, nlat)
    og = OGrid(nlat)
    p, q = inputs.pairs("paper_uniform", 2400, 2, og.x, og.nlon, og.a_ring, masses=True)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                                 max_iter=T, tol=0.0, check_every=10)
    shot.shot_grid_free(g)
    ref = sk.divergence(og, p64, q64, eps, tau, T=T, delta=0.0, C=10)
    assert np.all(r["status"] == ref["status"])
    ot_pq = ref["runs"]["ot"][:2]
    assert np.all(s_err_prec(r["S"], ref["S"], ot_pq, TOL, "bf16x3") <= 1.0)
