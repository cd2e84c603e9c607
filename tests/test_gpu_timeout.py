"""Failure detection on the device path, without a GPU fault: the bounded waits of the
tcgen05 Legendre kernels.

Every mbarrier wait in those kernels gives up after a limit that the launch passes in (by
default 2^30 SM cycles).  Here one heat apply on a small grid runs with a limit of a few
hundred cycles, far below a TMA copy's latency, so its first waits expire: each CTA raises its
abort flag, lets its own copies land and its MMAs finish, frees its tensor memory and returns.
The host then reads SHOT_ERR_TIMEOUT from shot_grid_check (which clears the flag), and the
next heat apply on the same grid, with the default limit, matches the FP64 oracle, so no
tensor memory and no flag was left behind.  Nothing here traps or waits without a bound.
"""
import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sht as osht
from tests.gpu_util import rel_max, f32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

# (precision, Legendre mode, transform tolerance of that form)
FORMS = {"bf16x3": (shot.SHOT_BF16X3, shot.SHOT_TABLE, 1e-4),
         "tf32x3": (shot.SHOT_TF32X3, shot.SHOT_TABLE, 2e-5),
         "tf32x3_rec": (shot.SHOT_TF32X3, shot.SHOT_RECURRENCE, 2e-5)}
TINY = 300   # SM cycles: well below the latency of one TMA copy


@pytest.mark.parametrize("form", list(FORMS))
def test_expired_wait_reports_timeout_and_grid_recovers(form):
    prec, mode, tol = FORMS[form]
    nlat, nf, t = 32, 3, 0.01
    og = OGrid(nlat)
    f, f64 = f32(np.random.default_rng(7).uniform(size=(nf, og.nlat, og.nlon)))
    ref = osht.heat_apply(og, f64, t)
    g = shot.shot_grid_init(nlat, None, -1, prec, mode)
    try:
        x = torch.from_numpy(f).cuda()
        out = torch.empty_like(x)
        shot.shot_heat_apply(g, t, x, out)
        shot.shot_grid_check(g)   # the default limit: no wait expires
        assert rel_max(out.cpu().numpy(), ref) < tol

        shot.shot_grid_set_wait_limit(g, TINY)
        out.fill_(0.0)
        shot.shot_heat_apply(g, t, x, out)
        with pytest.raises(shot.ShotError) as e:
            shot.shot_grid_check(g)
        assert e.value.code == shot.SHOT_ERR_TIMEOUT
        shot.shot_grid_check(g)   # the check cleared the flag

        shot.shot_grid_set_wait_limit(g, 0)   # back to the default
        for _ in range(2):   # tensor memory was freed: later launches allocate it again
            out.fill_(0.0)
            shot.shot_heat_apply(g, t, x, out)
            shot.shot_grid_check(g)
            assert rel_max(out.cpu().numpy(), ref) < tol
    finally:
        shot.shot_grid_free(g)


def test_wait_limit_rejects_a_null_grid():
    with pytest.raises(shot.ShotError) as e:
        shot.shot_grid_set_wait_limit(None, 100)
    assert e.value.code == shot.SHOT_ERR_INVALID_ARG
