"""GPU gradient of the Sinkhorn divergence (shot_divergence_grad, C ABI) against the FP64 oracle.

UNROLLED: derivative of S after exactly T iterations, checked along random directions
against central finite differences of the oracle's S after the same T iterations.
ENVELOPE: the potential form at convergence, against the oracle's envelope gradient.
Bar: directional derivatives within 1e-4 (relative) of the finite differences.
"""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle.gradient import fd_directional, envelope
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import f32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL = 1e-4


def _dirs(og, p, k, seed, balanced):
    rng = np.random.default_rng(seed)
    a = og.a
    out = []
    for _ in range(k):
        d = p * rng.normal(size=p.shape)
        if balanced:
            d -= np.sum(a * d) / np.sum(a)          # keep the masses equal
        d *= np.sqrt(np.sum(a * p * p) / np.sum(a * d * d))
        out.append(d)
    return np.array(out)


@pytest.mark.parametrize("nlat,eps,tau,T,ck", [(12, 1.0, math.inf, 40, 7), (16, 0.5, math.inf, 60, 20),
                                               (12, 1.0, 1.0, 40, 9), (16, 0.5, 0.3, 30, 30)])
def test_unrolled_gradient_matches_oracle_fd(nlat, eps, tau, T, ck):
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat)
    try:
        bal = math.isinf(tau)
        p, q = inputs.pairs("vmf3", 40 + nlat, 2, og.x, og.nlon, og.a_ring, masses=not bal)
        p32, p64 = f32(p)
        q32, q64 = f32(q)
        rc, r = shot.shot_divergence_grad(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                                          max_iter=T, checkpoint_every=ck, mode=shot.SHOT_GRAD_UNROLLED)
        assert rc >= 0 and np.all(r["status"] >= 0)
        grad = r["grad"].cpu().numpy().astype(np.float64)
        for b in range(2):
            dirs = _dirs(og, p64[b], 3, 7 + b, bal)
            fd = fd_directional(og, p64[b], q64[b], eps, tau, T, dirs, h=1e-5)
            got = np.array([np.sum(grad[b] * d) for d in dirs])
            scale = np.max(np.abs(fd))
            assert np.max(np.abs(got - fd)) <= TOL * scale, (got, fd)
    finally:
        shot.shot_grid_free(g)


def test_unrolled_gradient_config4_structure():
    # the iteration / checkpoint structure of the config-4 workload (T = 400, k = 20) on a
    # grid the oracle differentiates in seconds
    nlat, eps, T, ck = 24, 0.4, 400, 20
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat)
    try:
        p, q = inputs.pairs("vmf8", 4000, 2, og.x, og.nlon, og.a_ring)
        p32, p64 = f32(p)
        q32, q64 = f32(q)
        rc, r = shot.shot_divergence_grad(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps,
                                          max_iter=T, checkpoint_every=ck)
        assert rc >= 0
        grad = r["grad"].cpu().numpy().astype(np.float64)
        dirs = _dirs(og, p64[0], 2, 11, True)
        fd = fd_directional(og, p64[0], q64[0], eps, math.inf, T, dirs, h=1e-5)
        got = np.array([np.sum(grad[0] * d) for d in dirs])
        assert np.max(np.abs(got - fd)) <= TOL * np.max(np.abs(fd)), (got, fd)
    finally:
        shot.shot_grid_free(g)


def test_envelope_gradient_matches_oracle_envelope():
    # converged problems (marginal error ~1e-15 in FP64): the envelope formula applies
    nlat, eps, T = 16, 1.0, 400
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat)
    try:
        p, q = inputs.pairs("vmf3", 77, 1, og.x, og.nlon, og.a_ring)
        p32, p64 = f32(p)
        q32, q64 = f32(q)
        rc, r = shot.shot_divergence_grad(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps,
                                          max_iter=T, mode=shot.SHOT_GRAD_ENVELOPE)
        ref = envelope(og, p64[0], q64[0], eps, math.inf, T, delta=0.0, C=0)
        got = r["grad"].cpu().numpy()[0].astype(np.float64)
        a = og.a
        # defined modulo c * a: compare the field forms centred by their area means
        gf, rf = got / a, ref / a
        gf -= np.sum(a * gf) / np.sum(a)
        rf -= np.sum(a * rf) / np.sum(a)
        assert np.max(np.abs(gf - rf)) <= TOL * np.max(np.abs(rf))
    finally:
        shot.shot_grid_free(g)


def test_autograd_function_backward():
    nlat, eps, T = 12, 1.0, 30
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat)
    try:
        p, q = inputs.pairs("vmf3", 5, 2, og.x, og.nlon, og.a_ring)
        pt = torch.from_numpy(p.astype(np.float32)).cuda().requires_grad_(True)
        qt = torch.from_numpy(q.astype(np.float32)).cuda()
        S = shot.divergence(g, pt, qt, eps, max_iter=T, checkpoint_every=10)
        (S * torch.tensor([1.0, 2.0], dtype=torch.float64, device="cuda")).sum().backward()
        rc, r = shot.shot_divergence_grad(g, pt.detach(), qt, eps, max_iter=T, checkpoint_every=10)
        np.testing.assert_allclose(pt.grad[0].cpu().numpy(), r["grad"][0].cpu().numpy(), rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(pt.grad[1].cpu().numpy(), 2 * r["grad"][1].cpu().numpy(), rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(S.detach().cpu().numpy(), r["S"], rtol=1e-6)
    finally:
        shot.shot_grid_free(g)
