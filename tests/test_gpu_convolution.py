"""GPU parity of the explicit Gibbs-kernel convolution and the heat-vs-matrix comparison
(App. "Convolution on S^2") against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import convolution as cv
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import rel_max, f32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

CC = shot.SHOT_QUAD_CLENSHAW_CURTIS
GL = shot.SHOT_QUAD_GAUSS_LEGENDRE
EPS8 = np.logspace(-3, 1, 8)   # the comparison's eps range, 8 values log-spaced


def test_normaliser_matches_oracle():
    for eps in EPS8:
        assert abs(shot.shot_gibbs_normaliser(eps) / cv.gibbs_normaliser(eps) - 1.0) < 1e-12


@pytest.mark.parametrize("quad,nlat,nlon,nf", [(CC, 9, 18, 1), (CC, 16, 32, 3), (CC, 33, 72, 5), (GL, 24, 48, 2)])
@pytest.mark.parametrize("eps", [1e-3, 0.1, 10.0])
def test_gibbs_apply_matches_oracle(quad, nlat, nlon, nf, eps):
    g = shot.shot_grid_init_quad(quad, nlat, nlon)
    og = OGrid(nlat, nlon, quadrature="cc" if quad == CC else "gl")
    f, f64 = f32(np.random.default_rng(nlat + nf).uniform(size=(nf, nlat, nlon)))
    out = torch.empty((nf, nlat, nlon), device="cuda")
    shot.shot_gibbs_apply(g, eps, torch.from_numpy(f).cuda(), out)
    torch.cuda.synchronize()
    shot.shot_grid_free(g)
    # FP32 sums of n <= 2200 positive terms and FP32 distances: 2e-5 of the largest output
    assert rel_max(out.cpu().numpy(), cv.gibbs_apply(og, f64, eps)) < 2e-5


@pytest.mark.parametrize("L", [8, 16, 32])
def test_conv_compare_matches_oracle(L):
    g = shot.shot_grid_init_quad(CC, L, 2 * L)
    og = OGrid(L, 2 * L, quadrature="cc")
    f, f64 = f32(inputs.field("vmf_k10", 42, og.x, og.nlon, og.a_ring)[None])
    ft = torch.from_numpy(f).cuda()
    for eps in EPS8:
        got = shot.shot_conv_compare(g, eps, ft)[0]
        ref = float(cv.conv_mae(og, f64, eps)[0])
        # the MAE differences two FP32 outputs of size ~max|K f|: absolute floor 2e-5 of that
        scale = float(np.abs(cv.gibbs_apply(og, f64, eps)).max())
        assert abs(got - ref) <= 1e-3 * ref + 2e-5 * scale, (eps, got, ref)
    shot.shot_grid_free(g)


def test_conv_compare_error_falls_with_resolution():
    # at eps = 1e-2 the discretisation dominates: finer grids, smaller MAE (the paper's trend)
    maes = []
    for L in (8, 16, 32, 64):
        g = shot.shot_grid_init_quad(CC, L, 2 * L)
        x, _, a = shot.shot_grid_nodes(g)
        f, _ = f32(inputs.field("vmf_k10", 42, x, 2 * L, a)[None])
        maes.append(shot.shot_conv_compare(g, 1e-2, torch.from_numpy(f).cuda())[0])
        shot.shot_grid_free(g)
    assert maes[0] > maes[1] > maes[2]


def test_gibbs_rejects_bad_arguments():
    g = shot.shot_grid_init_quad(CC, 8, 16)
    x = torch.zeros((1, 8, 16), device="cuda")
    with pytest.raises(shot.ShotError):
        shot.shot_gibbs_apply(g, 0.0, x, torch.empty_like(x))
    with pytest.raises(shot.ShotError):
        shot.shot_gibbs_apply(g, 0.1, x, x)
    with pytest.raises(shot.ShotError):
        shot.shot_gibbs_normaliser(-1.0)
    shot.shot_grid_free(g)
