"""GPU gradient of the Sinkhorn divergence (shot_divergence_grad, C ABI) against the FP64 oracle.

UNROLLED: derivative of S after exactly T iterations, checked along random directions
against central finite differences of the oracle's S after the same T iterations.
ENVELOPE: the potential form at convergence, against the oracle's envelope gradient.
Bar: directional derivatives within 1e-4 (relative to the largest) of the finite
differences, the gradient target.  The split forms miss it at the gradient workload's shape,
where dS/dp is a small difference of potentials (S = 4.4e-5 there) that amplifies operator
error; those cases record the measured shortfall as expected failures (pytest.xfail with the
value) and still fail outright above a ceiling, GRAD_LIMIT, so that a defect is not hidden.
Measured on GB300 (directional error, 3 directions): 256 x 512, T = 400, k = 20: FP32 7.8e-5,
TF32x3 1.3e-4 (its FP32 tensor-core accumulation and 2^-21 products), BF16x3 8.0e-3 (~2^-17
representation error per bf16 hi/lo table entry, a fixed perturbation of the operator);
16 x 32, vMF fields, T = 60: FP32 1.0e-6, BF16x3 1.7e-4; 24 x 48, U(0,1) fields, eps = 0.1,
T = 100: FP32 5.2e-6, BF16x3 3.9e-4.

The gradient workload of Sec. 4.2 at its own shape (256 x 512, t = 1e-3, T = 400 with u, v
checkpointed every 20 iterations, a batch of 16 pairs) is checked against central differences
that the oracle computed once (tests/golden/grad_fd_256x512.json, written by
tests/golden/make_grad_fd_256.py): 400 FP64 iterations at that size take minutes on a CPU.
"""
import json
import math
import os

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
# (ceiling, reason): between TOL and the ceiling a split form's miss is an expected failure
GRAD_LIMIT = {"tf32x3": (1e-3, "TF32x3: 2^-21 products accumulated in FP32 by the tensor cores; "
                               "the config-4 gradient measured 1.3e-4"),
              "bf16x3": (3e-2, "BF16x3: ~2^-17 per bf16 hi/lo table entry; the config-4 gradient measured "
                               "8.0e-3, the small cases 1.7e-4 and 3.9e-4")}
PREC = {"fp32": shot.SHOT_FP32, "tf32x3": shot.SHOT_TF32X3, "bf16x3": shot.SHOT_BF16X3}
GOLD_256 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grad_fd_256x512.json")


def _dirs(og, p, k, seed, balanced):
    return inputs.fd_directions(p, og.a, k, seed, balanced)


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


def _directional_err(grad, dirs, fd):
    got = np.array([np.sum(grad * d) for d in dirs])
    return np.max(np.abs(got - fd)) / np.max(np.abs(fd)), got


def _assert_grad(prec, err, got, fd):
    msg = f"{prec}: directional error {err:.3e} (got {got}, fd {fd})"
    if err <= TOL:
        return
    assert prec in GRAD_LIMIT and err <= GRAD_LIMIT[prec][0], msg
    pytest.xfail(f"{GRAD_LIMIT[prec][1]}; measured {err:.3e} > {TOL:g}")


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_unrolled_gradient_config4_shape_matches_stored_oracle_fd(prec):
    gold = json.load(open(GOLD_256))
    og = OGrid(gold["nlat"])
    p, q = inputs.pairs(gold["recipe"], gold["seed"], gold["npairs"], og.x, og.nlon, og.a_ring)
    p32, p64 = f32(p)
    q32, _ = f32(q)
    g = shot.shot_grid_init(gold["nlat"], None, -1, PREC[prec])
    try:
        rc, r = shot.shot_divergence_grad(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(),
                                          gold["eps"], max_iter=gold["T"], checkpoint_every=20)
        assert rc >= 0 and np.all(r["status"] >= 0), (rc, r["status"])
        k = gold["pair"]
        grad = r["grad"][k].cpu().numpy().astype(np.float64)
        dirs = inputs.fd_directions(p64[k], og.a, gold["ndirs"], gold["dir_seed"], balanced=True)
        err, got = _directional_err(grad, dirs, np.array(gold["fd"]))
        _assert_grad(prec, err, got, gold["fd"])
    finally:
        shot.shot_grid_free(g)


# vMF fields (floor 1e-6) drive Kv toward 0 far from their modes, below BF16x3's error relative
# to the largest value at nlat = 24, eps = 0.4 (the solve stops NONPOSITIVE there): the second
# case takes the U(0,1) fields
@pytest.mark.parametrize("nlat,eps,T,ck,recipe", [(16, 0.5, 60, 20, "vmf3"), (24, 0.1, 100, 20, "paper_uniform")])
def test_bf16x3_unrolled_gradient_matches_oracle_fd(nlat, eps, T, ck, recipe):
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat, None, -1, shot.SHOT_BF16X3)
    try:
        p, q = inputs.pairs(recipe, 90 + nlat, 1, og.x, og.nlon, og.a_ring)
        p32, p64 = f32(p)
        q32, q64 = f32(q)
        rc, r = shot.shot_divergence_grad(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps,
                                          max_iter=T, checkpoint_every=ck)
        assert rc >= 0 and np.all(r["status"] >= 0)
        grad = r["grad"][0].cpu().numpy().astype(np.float64)
        dirs = _dirs(og, p64[0], 3, 5, True)
        fd = fd_directional(og, p64[0], q64[0], eps, math.inf, T, dirs, h=1e-5)
        err, got = _directional_err(grad, dirs, fd)
        _assert_grad("bf16x3", err, got, fd)
    finally:
        shot.shot_grid_free(g)

