"""Accuracy at the headline shape: the batched heat-kernel Sinkhorn on the 720 x 1440
Gauss-Legendre grid, t = 1e-4 (eps = 4t, Sec. 3.2), against the FP64 oracle after the same
T = 20 iterations of Alg. 1 (App. C), for every precision of the Legendre contractions.

One pair of the benchmark's fields (the runtime experiment's U(0,1) fields of Sec. 4.1,
seed 5000, pair 0) gives the three problems (p,q), (p,p), (q,q) of eq. (sinkhorn-divergence).
Compared, each against its precision's target (FP32 1e-5, split forms 1e-4):
  * the gauge-fixed potentials phi = eps log u, psi = eps log v (App. C.2), relative to their
    largest magnitude;
  * the scalings u, v element by element (|u_gpu / u_ref - 1| = |d phi| / eps);
  * the marginal error of App. C.3 (itself relative to ||p||) recomputed by the oracle from
    the GPU's u and v, against the oracle's own: |e_gpu - e_ref| <= target;
  * S and S_dual of eq. (sinkhorn-divergence) by the contract's metric
    |dS| / max(|S|, 1e-3 |OT(p,q)|).
The bf16 hi/lo form misses the S and element-wise bars here: its table carries ~2^-17
relative representation error per entry, a fixed perturbation of the operator that the
difference S = OT(p,q) - (OT(p,p) + OT(q,q))/2 (S ~ 5e-3 |OT| on these fields) does not
cancel; those cases are expected failures and record the measured shortfall.
"""
import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sinkhorn as sk
from oracle import sht as osht
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import f32, s_err, potentials_err, rel_elem, assert_s, BF16_S_LIMIT

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

NLAT, T_HEAT, T_ITERS, SEED = 720, 1e-4, 20, 5000
EPS = 4.0 * T_HEAT
TOL = {"fp32": 1e-5, "tf32x3": 1e-4, "bf16x3": 1e-4, "tf32x3_rec": 1e-4}
PREC = {"fp32": (shot.SHOT_FP32, shot.SHOT_TABLE), "tf32x3": (shot.SHOT_TF32X3, shot.SHOT_TABLE),
        "bf16x3": (shot.SHOT_BF16X3, shot.SHOT_TABLE),
        # TF32x3 contractions on P regenerated from checkpoints (recurrence mode, no table)
        "tf32x3_rec": (shot.SHOT_TF32X3, shot.SHOT_RECURRENCE)}
ALL = ["fp32", "tf32x3", "tf32x3_rec", "bf16x3"]
BF16_MISS = pytest.mark.xfail(strict=True, reason="bf16 hi/lo operands: ~2^-17 per table entry; the element-wise "
                                                  "scalings miss 1e-4 at 720 (measured 3.2e-4)")


@pytest.fixture(scope="module")
def ref720():
    og = OGrid(NLAT)
    og.pbar()
    p, q = inputs.pairs("paper_uniform", SEED, 1, og.x, og.nlon, og.a_ring)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    ref = sk.divergence(og, p64, q64, EPS, T=T_ITERS, C=10)
    assert np.all(ref["status"] == 0)
    return dict(og=og, p32=p32, q32=q32, p64=p64, q64=q64, ref=ref, gpu={})


def _gpu(ref720, prec):
    """One shot_divergence solve per precision (cached for the module's tests)."""
    if prec not in ref720["gpu"]:
        g = shot.shot_grid_init(NLAT, 2 * NLAT, -1, *PREC[prec])
        try:
            pt = torch.from_numpy(ref720["p32"]).cuda()
            qt = torch.from_numpy(ref720["q32"]).cuda()
            u3 = torch.empty((3,) + pt.shape[1:], device="cuda")
            v3 = torch.empty_like(u3)
            rc, r = shot.shot_divergence(g, pt, qt, EPS, max_iter=T_ITERS, tol=0.0, check_every=10, u3=u3, v3=v3)
            assert rc == 0 and np.all(r["status"] == 0), (rc, r["status"])
            r["u"] = u3.cpu().numpy().astype(np.float64)
            r["v"] = v3.cpu().numpy().astype(np.float64)
        finally:
            shot.shot_grid_free(g)
        ref720["gpu"][prec] = r
    return ref720["gpu"][prec]


@pytest.mark.parametrize("prec", ALL)
def test_potentials_and_marginals_match_oracle_at_720(ref720, prec):
    r, ref, og = _gpu(ref720, prec), ref720["ref"], ref720["og"]
    runs = ref["runs"]
    tol = TOL[prec]
    e_pot = potentials_err(og, EPS, r["u"], r["v"], runs["phi"], runs["psi"])
    assert e_pot <= tol, f"{prec}: gauge-fixed potentials {e_pot:.3e} > {tol:g}"
    # App. C.3's marginal error of the GPU's scalings, recomputed with the oracle's K
    P = np.concatenate([ref720["p64"], ref720["p64"], ref720["q64"]])
    e_gpu = sk.marginal_error(og, r["u"], osht.heat_apply(og, r["v"], T_HEAT), P)
    d = np.abs(e_gpu - runs["err"])
    assert np.all(d <= tol), f"{prec}: marginal error {e_gpu} vs oracle {runs['err']} (diff {d})"
    np.testing.assert_allclose(r["ot3"], runs["ot"], rtol=tol)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "tf32x3_rec", pytest.param("bf16x3", marks=BF16_MISS)])
def test_scalings_elementwise_match_oracle_at_720(ref720, prec):
    r, runs = _gpu(ref720, prec), ref720["ref"]["runs"]
    for name in ("u", "v"):
        e = rel_elem(r[name], runs[name], floor=0.0)
        assert e <= TOL[prec], f"{prec}: {name} element-wise {e:.3e} > {TOL[prec]:g}"


@pytest.mark.parametrize("prec", ALL)
def test_divergence_matches_oracle_at_720(ref720, prec):
    r, ref = _gpu(ref720, prec), ref720["ref"]
    ot_pq = ref["runs"]["ot"][:1]
    lim = BF16_S_LIMIT if prec == "bf16x3" else None
    assert_s(r["S"], ref["S"], ot_pq, TOL[prec], limited_by=lim)
    assert_s(r["S_dual"], ref["S_dual"], ot_pq, TOL[prec], limited_by=lim)
