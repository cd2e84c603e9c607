"""GPU parity of Algorithm 1 and the Sinkhorn divergence against the FP64 oracle (C ABI)."""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32, s_err, potentials_err, assert_s, BF16_S_LIMIT, FP32_S_LIMIT

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

# FP32 targets: potentials and S within 1e-5 of the FP64 oracle (relative).
TOL_PHI = 1e-5
TOL_S = 1e-5


@pytest.fixture(scope="module")
def grid_cache():
    cache = {}

    def get(nlat, nlon=None):
        key = (nlat, nlon)
        if key not in cache:
            cache[key] = (shot.shot_grid_init(nlat, nlon), OGrid(nlat, nlon))
        return cache[key]
    yield get
    for g, _ in cache.values():
        shot.shot_grid_free(g)


def _fields(og, recipe, seed, npairs, masses=False):
    p, q = inputs.pairs(recipe, seed, npairs, og.x, og.nlon, og.a_ring, masses=masses)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    return torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), p64, q64


@pytest.mark.parametrize("nlat,nlon,eps,tau,T", [(16, None, 0.1, math.inf, 40), (32, None, 0.1, math.inf, 60),
                                                 (32, None, 0.1, 1.0, 60), (64, None, 0.01, 0.1, 30),
                                                 (33, 72, 0.1, math.inf, 30)])
def test_sinkhorn_fixed_iterations_match_oracle(grid_cache, nlat, nlon, eps, tau, T):
    g, og = grid_cache(nlat, nlon)
    unb = not math.isinf(tau)
    pt, qt, p, q = _fields(og, "paper_uniform", 1000 + nlat, 3, masses=unb)
    rc, r = shot.shot_sinkhorn(g, pt, qt, eps, tau, max_iter=T, tol=0.0, check_every=10)
    ref = sk.sinkhorn(og, p, q, eps, tau, T=T, delta=0.0, C=10)
    assert rc == 0 and np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    assert np.all(r["iters"] == T)
    u, v = r["u"].cpu().numpy(), r["v"].cpu().numpy()
    assert potentials_err(og, eps, u, v, ref["phi"], ref["psi"]) < TOL_PHI
    for b in range(3):   # FP32 also meets the bar without removing the gauge
        assert rel_max(eps * np.log(u[b]), ref["phi"][b]) < TOL_PHI
        assert rel_max(eps * np.log(v[b]), ref["psi"][b]) < TOL_PHI
    np.testing.assert_allclose(r["ot"], ref["ot"], rtol=TOL_PHI)
    np.testing.assert_allclose(r["mass_pi"], ref["mass_pi"], rtol=1e-5)
    np.testing.assert_allclose(r["err"], ref["err"], rtol=1e-2, atol=1e-6)


def test_sinkhorn_converges_at_same_check(grid_cache):
    g, og = grid_cache(32)
    pt, qt, p, q = _fields(og, "paper_uniform", 77, 2)
    rc, r = shot.shot_sinkhorn(g, pt, qt, 0.1, max_iter=2000, tol=1e-5, check_every=10)
    ref = sk.sinkhorn(og, p, q, 0.1, T=2000, delta=1e-5, C=10)
    assert np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    np.testing.assert_array_equal(r["iters"], ref["iters"])
    assert np.all(r["err"] < 1e-5)


def test_l1_norm_and_not_converged_warning(grid_cache):
    g, og = grid_cache(16)
    pt, qt, p, q = _fields(og, "paper_uniform", 5, 1)
    rc, r = shot.shot_sinkhorn(g, pt, qt, 0.1, max_iter=20, tol=1e-12, check_every=10,
                               flags=shot.SHOT_FLAG_NORM_L1)
    ref = sk.sinkhorn(og, p, q, 0.1, T=20, delta=1e-12, C=10, norm="l1")
    assert rc == shot.SHOT_WARN_NOT_CONVERGED and r["status"][0] == ref["status"][0] == sk.NOT_CONVERGED
    np.testing.assert_allclose(r["err"], ref["err"], rtol=1e-2)


def test_breakdown_reported_at_oracle_iteration(grid_cache):
    # App. C.4: truncated-kernel negativity; literal vMF inputs at nlat 32, t = 1e-2
    g, og = grid_cache(32)
    pt, qt, p, q = _fields(og, "vmf3", 1001, 1)
    rc, r = shot.shot_sinkhorn(g, pt, qt, 4e-2, max_iter=50, tol=1e-10, check_every=10)
    ref = sk.sinkhorn(og, p, q, 4e-2, T=50, delta=1e-10, C=10)
    assert ref["status"][0] == sk.NONPOSITIVE
    assert rc == shot.SHOT_ERR_NONPOSITIVE and r["status"][0] == shot.SHOT_ERR_NONPOSITIVE
    assert r["iters"][0] == ref["iters"][0]
    assert np.isnan(r["ot"][0])


# tol >= 1e-6: the FP32 path resolves the relative marginal error down to ~3e-7
@pytest.mark.parametrize("nlat,eps,tau,T,tol", [(16, 0.2, math.inf, 400, 2e-6), (32, 0.1, math.inf, 600, 1e-6),
                                                (32, 0.1, 1.0, 80, 0.0), (64, 0.01, 10.0, 40, 0.0)])
def test_divergence_matches_oracle(grid_cache, nlat, eps, tau, T, tol):
    g, og = grid_cache(nlat)
    unb = not math.isinf(tau)
    pt, qt, p, q = _fields(og, "paper_uniform", 2000 + nlat, 2, masses=unb)
    rc, r = shot.shot_divergence(g, pt, qt, eps, tau, max_iter=T, tol=tol, check_every=10)
    ref = sk.divergence(og, p, q, eps, tau, T=T, delta=tol, C=10)
    assert np.all(r["status"] == ref["status"])
    np.testing.assert_array_equal(r["iters3"], ref["runs"]["iters"])
    ot_pq = ref["runs"]["ot"][:2]
    assert np.all(s_err(r["S"], ref["S"], ot_pq, TOL_S) <= 1.0)
    assert np.all(s_err(r["S_dual"], ref["S_dual"], ot_pq, TOL_S) <= 1.0)
    if not unb:
        assert np.all(r["S"] > 0)


def test_divergence_of_identical_measures_is_zero(grid_cache):
    g, og = grid_cache(16)
    pt, qt, p, q = _fields(og, "paper_uniform", 9, 2)
    rc, r = shot.shot_divergence(g, pt, pt, 0.2, max_iter=100, tol=0.0)
    assert np.all(r["S"] == 0.0)


@pytest.mark.parametrize("tau", [math.inf, 1.0])
def test_divergence_with_zero_marginal_entries(grid_cache, tau):
    # p vanishes on a polar cap and q on a longitude sector: those nodes give u = 0 (v = 0)
    # and contribute their limit 0 to the objective (a reading of the paper's dual form).
    # The empty regions stay within about one kernel width (sqrt(2t) ~ 0.3 rad here): over a
    # much larger empty cap K u falls by orders of magnitude, v grows accordingly and the
    # FP32 SHT's absolute error turns into a relative error of v there (a conditioning
    # limit of the FP32 path, not of the update)
    g, og = grid_cache(24)
    rng = np.random.default_rng(24)
    p, q = rng.uniform(size=(2, 2, og.nlat, og.nlon))
    p[:, :2] = 0.0
    q[:, :, : og.nlon // 8] = 0.0
    p /= np.sum(og.a * p, axis=(1, 2))[:, None, None]
    q /= np.sum(og.a * q, axis=(1, 2))[:, None, None]
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    rc, r = shot.shot_divergence(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), 0.2, tau,
                                 max_iter=60, tol=0.0, check_every=10)
    ref = sk.divergence(og, p64, q64, 0.2, tau, T=60, delta=0.0, C=10)
    assert np.all(r["status"] == 0) and np.all(ref["status"] == 0)
    assert np.all(np.isfinite(r["S"])) and np.all(np.isfinite(ref["S"]))
    assert np.all(s_err(r["S"], ref["S"], ref["runs"]["ot"][:2], TOL_S) <= 1.0)


@pytest.mark.parametrize("nlat,pairs,tau", [(256, 8, math.inf), (75, 3, 1.0), (45, 1, math.inf)])
def test_persistent_update_kernel_matches_one_item_per_cta(nlat, pairs, tau):
    """The solver's update half-steps run in a persistent kernel that prefetches the next
    (ring pair, field group) item's spectra and marginals; the per-item arithmetic is that of
    the one-item-per-CTA kernel (SHOT_IDFT_PERSISTENT=0), so u, v and S agree bit for bit.
    Sizes: several items per CTA (256), an odd grid with an equator ring (75, 45), a partial
    field group (3 problems)."""
    import os
    og = OGrid(nlat)
    p, q = inputs.pairs("paper_uniform", 4000 + nlat, pairs, og.x, og.nlon, og.a_ring,
                        masses=not math.isinf(tau))
    pt = torch.from_numpy(p.astype(np.float32)).cuda()
    qt = torch.from_numpy(q.astype(np.float32)).cuda()
    res = []
    for flag in ("1", "0"):
        os.environ["SHOT_IDFT_PERSISTENT"] = flag
        try:
            g = shot.shot_grid_init(nlat)
        finally:
            del os.environ["SHOT_IDFT_PERSISTENT"]
        try:
            u3 = torch.empty((3 * pairs, og.nlat, og.nlon), device="cuda")
            v3 = torch.empty_like(u3)
            rc, r = shot.shot_divergence(g, pt, qt, 0.05, tau, max_iter=40, tol=0.0, check_every=10, u3=u3, v3=v3)
            assert rc == 0
            res.append((u3.cpu().numpy(), v3.cpu().numpy(), np.asarray(r["S"])))
        finally:
            shot.shot_grid_free(g)
    for a, b in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_sinkhorn_on_ring_length_with_prime_13(prec):
    """nlon = 130 = 2*5*13: the solver's fused transforms run the generic radix-13 stage."""
    nlat, eps, T = 65, 0.05, 40
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat, None, -1, shot.SHOT_FP32 if prec == "fp32" else shot.SHOT_BF16X3)
    try:
        p, q = inputs.pairs("paper_uniform", 130, 2, og.x, og.nlon, og.a_ring)
        p32, p64 = f32(p)
        q32, q64 = f32(q)
        rc, r = shot.shot_sinkhorn(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps,
                                   max_iter=T, tol=0.0, check_every=10)
        ref = sk.sinkhorn(og, p64, q64, eps, math.inf, T=T, delta=0.0, C=10)
        assert rc == 0 and np.all(r["status"] == 0)
        u, v = r["u"].cpu().numpy(), r["v"].cpu().numpy()
        assert potentials_err(og, eps, u, v, ref["phi"], ref["psi"]) < (TOL_PHI if prec == "fp32" else 1e-4)
    finally:
        shot.shot_grid_free(g)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_unbalanced_potentials_beyond_fp32_exponent_range(prec):
    """tau/eps = 1000 with masses 0.63 and 1.58 (App. C.2's unbalanced branch): the
    potentials settle near -+tau log(m(q)/m(p))/2, so eps log u ~ -4.6 and u ~ e^{-460},
    far outside FP32.  The solver keeps each scaling as an FP32 buffer times an FP64
    factor; ot, m(pi), the potentials (SHOT_FLAG_POTENTIALS) and S still match the FP64
    oracle, whose scalings stay inside the FP64 range."""
    nlat, eps, tau, T = 64, 0.01, 10.0, 40
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat, None, -1, shot.SHOT_FP32 if prec == "fp32" else shot.SHOT_BF16X3)
    tol = TOL_PHI if prec == "fp32" else 1e-4
    try:
        p, q = inputs.pairs("paper_uniform", 6400, 2, og.x, og.nlon, og.a_ring)
        p32, p64 = f32(p * np.array([0.63, 1.58])[:, None, None])
        q32, q64 = f32(q * np.array([1.58, 0.63])[:, None, None])
        pt, qt = torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda()
        rc, r = shot.shot_sinkhorn(g, pt, qt, eps, tau, max_iter=T, tol=0.0, check_every=10,
                                   flags=shot.SHOT_FLAG_POTENTIALS)
        ref = sk.sinkhorn(og, p64, q64, eps, tau, T=T, delta=0.0, C=10)
        assert np.all(ref["status"] == 0)
        assert np.max(np.abs(ref["phi"])) / eps > 200.0   # e^{phi/eps} is outside FP32
        assert rc == 0 and np.all(r["status"] == 0)
        phi, psi = r["u"].cpu().numpy(), r["v"].cpu().numpy()
        assert rel_max(phi, ref["phi"]) < tol and rel_max(psi, ref["psi"]) < tol
        np.testing.assert_allclose(r["ot"], ref["ot"], rtol=tol)
        # m(pi) = sum a e^{(phi + psi)/eps} H...: a relative change d of the potentials moves it by
        # (|phi| + |psi|) d / eps, so FP32 potentials (d = 2^-24) of size ~4.7 at eps = 0.01
        # carry ~5e-5 of m(pi) (the potentials themselves are within tol above)
        tol_m = max(tol, 2.0 ** -24 * (np.max(np.abs(ref["phi"])) + np.max(np.abs(ref["psi"]))) / eps)
        np.testing.assert_allclose(r["mass_pi"], ref["mass_pi"], rtol=tol_m)
        rc, rd = shot.shot_divergence(g, pt, qt, eps, tau, max_iter=T, tol=0.0, check_every=10)
        refd = sk.divergence(og, p64, q64, eps, tau, T=T, delta=0.0, C=10)
        assert rc == 0 and np.all(rd["status"] == 0)
        assert_s(rd["S"], refd["S"], refd["runs"]["ot"][:2], tol, limited_by=BF16_S_LIMIT if prec == "bf16x3" else None)
    finally:
        shot.shot_grid_free(g)


def test_potentials_flag_returns_eps_log_scalings(grid_cache):
    g, og = grid_cache(32)
    pt, qt, p, q = _fields(og, "paper_uniform", 81, 2, masses=True)
    for tau in (math.inf, 1.0):
        rc, r = shot.shot_sinkhorn(g, pt, qt, 0.1, tau, max_iter=30, tol=0.0, check_every=10)
        rc2, r2 = shot.shot_sinkhorn(g, pt, qt, 0.1, tau, max_iter=30, tol=0.0, check_every=10,
                                     flags=shot.SHOT_FLAG_POTENTIALS)
        assert rc == rc2 == 0
        np.testing.assert_array_equal(r["ot"], r2["ot"])
        u, v = r["u"].cpu().double().numpy(), r["v"].cpu().double().numpy()
        assert rel_max(r2["u"].cpu().numpy(), 0.1 * np.log(u)) < 1e-6
        assert rel_max(r2["v"].cpu().numpy(), 0.1 * np.log(v)) < 1e-6


@pytest.mark.parametrize("prec,tau", [("fp32", math.inf), ("bf16x3", math.inf), ("fp32", 1.0)])
def test_full_size_first_iteration_matches_oracle(prec, tau):
    """GL 720 x 1440 (the headline grid, t = 1e-4) through the solver's own launch path
    (persistent update kernel, graph-free single block, final pass): after one iteration of
    Alg. 1 the returned u, v equal the oracle's first iteration (u' = (p / K 1)^g,
    v' = (q / K u')^g, then the gauge or the translation-invariant step) at every node."""
    from oracle.sht import heat_apply
    nlat, eps = 720, 4e-4
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat, None, -1, shot.SHOT_FP32 if prec == "fp32" else shot.SHOT_BF16X3)
    try:
        unb = not math.isinf(tau)
        # unit masses also for tau = 1: with masses U[0.5, 2] the translation-invariant constant
        # at eps = 4e-4 is e^{+-c/eps} ~ e^{+-800}, beyond FP64 (and so beyond the oracle)
        p, q = inputs.pairs("paper_uniform", 7201, 2, og.x, og.nlon, og.a_ring)
        p32, p64 = f32(p)
        q32, q64 = f32(q)
        rc, r = shot.shot_sinkhorn(g, torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), eps, tau,
                                   max_iter=1, tol=0.0, check_every=0)
        assert rc == 0 and np.all(r["status"] == 0)
        gam = 1.0 if not unb else tau / (tau + eps)
        u1 = (p64 / heat_apply(og, np.ones_like(p64), eps / 4)) ** gam
        v1 = (q64 / heat_apply(og, u1, eps / 4)) ** gam
        if not unb:
            s = np.sum(u1, axis=(1, 2))[:, None, None]
            u1, v1 = u1 / s, v1 * s
        else:
            a = og.a
            A = np.sum(a * p64 * u1 ** (-eps / tau), axis=(1, 2))
            B = np.sum(a * q64 * v1 ** (-eps / tau), axis=(1, 2))
            c = (0.5 * tau * (np.log(A) - np.log(B)))[:, None, None]
            u1, v1 = u1 * np.exp(c / eps), v1 * np.exp(-c / eps)
        tol = TOL_PHI if prec == "fp32" else 1e-4
        for b in range(2):
            assert rel_max(r["u"][b].cpu().numpy(), u1[b]) < tol
            assert rel_max(r["v"][b].cpu().numpy(), v1[b]) < tol
    finally:
        shot.shot_grid_free(g)


@pytest.mark.parametrize("tau", [math.inf, 1.0])
def test_warm_start_continues_the_iteration(grid_cache, tau):
    """SHOT_FLAG_WARM_START: T1 iterations, then T2 more from the returned (u, v), equal the
    oracle's T1 + T2 iterations (Alg. 1's next u-step reads v only; the stored pair carries the
    gauge / translation-invariant state)."""
    g, og = grid_cache(32)
    unb = not math.isinf(tau)
    pt, qt, p, q = _fields(og, "paper_uniform", 515, 2, masses=unb)
    rc, r1 = shot.shot_sinkhorn(g, pt, qt, 0.1, tau, max_iter=20, tol=0.0, check_every=10)
    assert rc == 0
    rc, r2 = shot.shot_sinkhorn(g, pt, qt, 0.1, tau, max_iter=25, tol=0.0, check_every=10,
                                flags=shot.SHOT_FLAG_WARM_START, u=r1["u"], v=r1["v"])
    assert rc == 0 and np.all(r2["iters"] == 25)
    ref = sk.sinkhorn(og, p, q, 0.1, tau, T=45, delta=0.0, C=10)
    u, v = r2["u"].cpu().numpy(), r2["v"].cpu().numpy()
    if unb:
        for b in range(2):
            assert rel_max(0.1 * np.log(u[b]), ref["phi"][b]) < TOL_PHI
            assert rel_max(0.1 * np.log(v[b]), ref["psi"][b]) < TOL_PHI
    else:
        assert potentials_err(og, 0.1, u, v, ref["phi"], ref["psi"]) < TOL_PHI
    np.testing.assert_allclose(r2["ot"], ref["ot"], rtol=TOL_PHI)


@pytest.mark.parametrize("prec,tau", [("fp32", math.inf), ("fp32", 1.0), ("bf16x3", math.inf)])
def test_symmetric_self_terms_match_oracle(prec, tau):
    """SHOT_FLAG_SYMMETRIC_SELF: the self terms by the symmetric averaged update, T fixed
    iterations on both sides, against the oracle's same iteration; S and the self terms' OT."""
    nlat, eps, T = 32, 0.1, 40
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat, None, -1, shot.SHOT_FP32 if prec == "fp32" else shot.SHOT_BF16X3)
    tol = TOL_S if prec == "fp32" else 1e-4
    try:
        unb = not math.isinf(tau)
        pt, qt, p, q = _fields(og, "paper_uniform", 8080, 2, masses=unb)
        rc, r = shot.shot_divergence(g, pt, qt, eps, tau, max_iter=T, tol=0.0, check_every=10,
                                     flags=shot.SHOT_FLAG_SYMMETRIC_SELF)
        ref = sk.divergence_symmetric_self(og, p, q, eps, tau, T=T, delta=0.0, C=10)
        assert rc == 0 and np.all(r["status"] == 0) and np.all(ref["status"] == 0)
        np.testing.assert_allclose(r["ot3"][2:], ref["self"]["ot"], rtol=tol)
        np.testing.assert_allclose(r["ot3"][:2], ref["pq"]["ot"], rtol=tol)
        assert_s(r["S"], ref["S"], ref["pq"]["ot"], tol, limited_by=BF16_S_LIMIT if prec == "bf16x3" else FP32_S_LIMIT)
    finally:
        shot.shot_grid_free(g)


def test_symmetric_self_terms_reach_the_same_divergence(grid_cache):
    """Converged, the symmetric self terms give Alg. 1's divergence (same fixed point) and stop
    earlier."""
    g, og = grid_cache(32)
    pt, qt, p, q = _fields(og, "paper_uniform", 8181, 2)
    rc, a = shot.shot_divergence(g, pt, qt, 0.1, max_iter=2000, tol=1e-6, check_every=10)
    rc2, b = shot.shot_divergence(g, pt, qt, 0.1, max_iter=2000, tol=1e-6, check_every=10,
                                  flags=shot.SHOT_FLAG_SYMMETRIC_SELF)
    assert rc == 0 and rc2 == 0
    ref = sk.divergence(og, p, q, 0.1, T=2000, delta=1e-9, C=10)
    assert np.all(s_err(b["S"], ref["S"], ref["runs"]["ot"][:2], 1e-4) <= 1.0), (b["S"], ref["S"])
    assert np.all(s_err(a["S"], ref["S"], ref["runs"]["ot"][:2], 1e-4) <= 1.0)
    assert np.all(b["iters3"][2:] <= a["iters3"][2:])
