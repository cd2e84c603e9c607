"""GPU regional attribution (shot_regional_rms) against the oracle's definition."""
import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle.regional import regional_rms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402


@pytest.mark.parametrize("nlat", [32, 90, 180])
def test_regional_rms_matches_oracle(nlat):
    og = OGrid(nlat)
    g = shot.shot_grid_init(nlat)
    try:
        rng = np.random.default_rng(nlat)
        grad = (og.a * rng.normal(size=(3, og.nlat, og.nlon))).astype(np.float32)
        got = shot.shot_regional_rms(g, torch.from_numpy(grad).cuda())
        ref = regional_rms(og, grad.astype(np.float64))
        np.testing.assert_allclose(got, ref, rtol=1e-5)
    finally:
        shot.shot_grid_free(g)
