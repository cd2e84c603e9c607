"""GPU parity of the grid, SHT and heat convolution against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sht as osht
from tests.gpu_util import rel_max, f32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

# FP32 arithmetic: ring FFT (log2 nlon stages) + a sum over <= nlat/2 nodes per output.
# Rounding grows like sqrt(terms) * 2^-24 relative to the largest term; 2e-5 of the
# largest output leaves a factor >= 10 of margin up to nlat = 720.
TOL_SHT = 2e-5


@pytest.fixture(scope="module")
def grid_cache():
    cache = {}

    def get(nlat, nlon=None, lmax=-1):
        key = (nlat, nlon, lmax)
        if key not in cache:
            g = shot.shot_grid_init(nlat, nlon, lmax)
            og = OGrid(nlat, nlon, None if lmax == -1 else lmax)
            cache[key] = (g, og)
        return cache[key]
    yield get
    for g, _ in cache.values():
        shot.shot_grid_free(g)


@pytest.mark.parametrize("nlat,nlon", [(2, 4), (7, 15), (32, 64), (180, 360), (720, 1440)])
def test_nodes_weights_match_oracle(grid_cache, nlat, nlon):
    # both sides run Newton on P_nlat in FP64; the weights go through P'(x) from an
    # nlat-step recurrence whose rounding grows ~ nlat * 2^-53 (the oracle is 7e-13 off a
    # 40-digit reference at nlat 256), hence 1e-11 relative
    g, og = grid_cache(nlat, nlon)
    x, w, a = shot.shot_grid_nodes(g)
    assert np.max(np.abs(x - og.x)) < 4e-15
    assert np.max(np.abs(w - og.w) / og.w) < 1e-11
    assert np.max(np.abs(a - og.a_ring) / og.a_ring) < 1e-11
    assert np.all(x[: nlat // 2] == -x[::-1][: nlat // 2])   # exact mirror


@pytest.mark.parametrize("nlat,nlon,lmax,nf", [(4, 8, -1, 1), (9, 18, -1, 3), (12, 30, 11, 2),
                                               (32, 64, -1, 5), (64, 128, -1, 40), (180, 360, -1, 2),
                                               (20, 45, 13, 3)])
def test_analysis_matches_oracle(grid_cache, nlat, nlon, lmax, nf):
    g, og = grid_cache(nlat, nlon, lmax)
    L = og.lmax + 1
    f, f64 = f32(np.random.default_rng(nlat + nf).normal(size=(nf, og.nlat, og.nlon)))
    c = torch.empty((nf, L, L, 2), device="cuda")
    shot.shot_sht_analysis(g, torch.from_numpy(f).cuda(), c)
    got = c.cpu().numpy()
    ref = osht.analysis(og, f64)
    assert rel_max(got[..., 0], ref.real) < TOL_SHT
    assert rel_max(got[..., 1], ref.imag) < TOL_SHT
    assert np.all(got[:, np.triu_indices(L, 1)[0], np.triu_indices(L, 1)[1]] == 0)


@pytest.mark.parametrize("nlat,nlon,lmax,nf", [(4, 8, -1, 1), (9, 18, -1, 3), (32, 64, -1, 5),
                                               (180, 360, -1, 2), (20, 45, 13, 3)])
def test_synthesis_matches_oracle(grid_cache, nlat, nlon, lmax, nf):
    g, og = grid_cache(nlat, nlon, lmax)
    L = og.lmax + 1
    rng = np.random.default_rng(100 + nlat)
    c = rng.normal(size=(nf, L, L, 2)).astype(np.float32)
    c[..., 0][:, np.triu_indices(L, 1)[0], np.triu_indices(L, 1)[1]] = 0
    c[..., 1][:, np.triu_indices(L, 1)[0], np.triu_indices(L, 1)[1]] = 0
    c[:, :, 0, 1] = 0
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_sht_synthesis(g, torch.from_numpy(c).cuda(), out)
    ref = osht.synthesis(og, c[..., 0].astype(np.float64) + 1j * c[..., 1].astype(np.float64))
    assert rel_max(out.cpu().numpy(), ref) < TOL_SHT


@pytest.mark.parametrize("nlat,nlon,lmax,nf,t", [(4, 8, -1, 1, 0.1), (9, 18, -1, 3, 0.02),
                                                 (32, 64, -1, 40, 1e-2), (64, 128, -1, 7, 2.5e-3),
                                                 (180, 360, -1, 3, 1e-3), (12, 30, 11, 2, 0.0),
                                                 (20, 45, 13, 5, 0.05)])
def test_heat_apply_matches_oracle(grid_cache, nlat, nlon, lmax, nf, t):
    g, og = grid_cache(nlat, nlon, lmax)
    f, f64 = f32(np.random.default_rng(7 * nlat + nf).uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, t, torch.from_numpy(f).cuda(), out)
    ref = osht.heat_apply(og, f64, t)
    assert rel_max(out.cpu().numpy(), ref) < TOL_SHT


def test_heat_apply_720_full_size(grid_cache):
    g, og = grid_cache(720)
    nf = 3
    f, f64 = f32(np.random.default_rng(720).uniform(size=(nf, 720, 1440)))
    out = torch.empty((nf, 720, 1440), device="cuda")
    shot.shot_heat_apply(g, 1e-4, torch.from_numpy(f).cuda(), out)
    ref = osht.heat_apply(og, f64, 1e-4)
    assert rel_max(out.cpu().numpy(), ref) < TOL_SHT


def test_heat_apply_rejects_bad_arguments(grid_cache):
    g, _ = grid_cache(8)
    x = torch.zeros((1, 8, 16), device="cuda")
    with pytest.raises(shot.ShotError):
        shot.shot_heat_apply(g, -1.0, x, torch.empty_like(x))
    with pytest.raises(shot.ShotError):
        shot.shot_heat_apply(g, 0.1, x, x)
    with pytest.raises(shot.ShotError):
        shot.shot_grid_init(8, 14)      # nlon < 2 lmax + 1
    with pytest.raises(shot.ShotError):
        shot.shot_grid_init(8, 6402)    # longer than the shared-memory ring FFT takes


# Ring lengths with prime factors above 5 run a generic FFT stage per such prime (O(p) work
# per output; the roots of unity tabulated in the plan): 42 = 2*3*7, 66 = 2*3*11,
# 98 = 2*7^2, 130 = 2*5*13, 362 = 2*181 (a prime radix of 181).
@pytest.mark.parametrize("nlat,nlon,nf", [(21, 42, 3), (33, 66, 2), (49, 98, 4), (65, 130, 24), (181, 362, 2)])
def test_any_ring_length_heat_and_sht_match_oracle(grid_cache, nlat, nlon, nf):
    g, og = grid_cache(nlat, nlon)
    L = og.lmax + 1
    rng = np.random.default_rng(nlon + nf)
    f, f64 = f32(rng.uniform(size=(nf, og.nlat, og.nlon)))
    out = torch.empty((nf, og.nlat, og.nlon), device="cuda")
    shot.shot_heat_apply(g, 2e-3, torch.from_numpy(f).cuda(), out)
    assert rel_max(out.cpu().numpy(), osht.heat_apply(og, f64, 2e-3)) < TOL_SHT
    c = torch.empty((nf, L, L, 2), device="cuda")
    shot.shot_sht_analysis(g, torch.from_numpy(f).cuda(), c)
    ref = osht.analysis(og, f64)
    got = c.cpu().numpy()
    assert rel_max(got[..., 0], ref.real) < TOL_SHT
    assert rel_max(got[..., 1], ref.imag) < TOL_SHT
