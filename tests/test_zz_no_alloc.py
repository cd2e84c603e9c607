"""The allocation-free heat convolution, checked against shot_heat_apply.

Callers that cannot allocate device memory where they need K_t (a pool that must not
grow, a step that forbids allocation, a stream being captured by someone else, a fixed
start-up memory budget) use shot_heat_apply_noalloc, whose scratch is a fixed
library-owned device array.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import rel_max

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL_SHT = 2e-5   # the tolerance the FP32 heat-convolution parity tests use


def _call_abi(g, t, x, y):
    """Through the C ABI directly (ctypes), as a caller without the binding would."""
    lib = shot.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.shot_heat_apply_noalloc(g, ctypes.c_double(t), ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()), x.shape[0], stream)


def test_noalloc_matches_heat_apply_twice():
    g = shot.shot_grid_init(64)
    try:
        rng = np.random.default_rng(64)
        for call, (nf, t) in enumerate([(5, 2.5e-3), (3, 1e-2)]):
            f = torch.from_numpy(rng.uniform(size=(nf, 64, 128)).astype(np.float32)).cuda()
            ref = torch.empty_like(f)
            shot.shot_heat_apply(g, t, f, ref)
            out = torch.full_like(f, float("nan"))
            rc = _call_abi(g, t, f, out)
            assert rc == shot.SHOT_OK, (call, shot.last_error())
            torch.cuda.synchronize()
            assert rel_max(out.cpu().numpy(), ref.cpu().numpy()) <= TOL_SHT, call
    finally:
        shot.shot_grid_free(g)


# a Gauss-Legendre FP32 grid in table and recurrence mode, and a HEALPix grid: (make, field shape)
GRIDS = {
    "gl_table": (lambda: shot.shot_grid_init(48), (3, 48, 96)),
    "gl_recurrence": (lambda: shot.shot_grid_init(48, None, -1, shot.SHOT_FP32, shot.SHOT_RECURRENCE), (3, 48, 96)),
    "healpix": (lambda: shot.shot_grid_init_healpix(8, -1, shot.SHOT_FP32, shot.SHOT_TABLE), (3, 12 * 8 * 8)),
}


@pytest.mark.parametrize("kind", list(GRIDS))
def test_noalloc_first_on_fresh_grid_allocates_nothing(kind):
    """On a grid that has never run a transform (no workspace yet) the allocation-free call
    comes first; after the first call has resolved the scratch array's device address, a
    second call leaves the device's free memory unchanged.  Only then does shot_heat_apply
    (which creates the grid's workspace) run, for the comparison."""
    make, shape = GRIDS[kind]
    g = make()
    try:
        t = 1e-2
        f = torch.from_numpy(np.random.default_rng(8).uniform(size=shape).astype(np.float32)).cuda()
        out = torch.full_like(f, float("nan"))
        ref = torch.empty_like(f)
        torch.cuda.synchronize()
        assert _call_abi(g, t, f, out) == shot.SHOT_OK, shot.last_error()
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        out.fill_(float("nan"))
        assert _call_abi(g, t, f, out) == shot.SHOT_OK, shot.last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0 - free1)
        shot.shot_heat_apply(g, t, f, ref)
        torch.cuda.synchronize()
        assert rel_max(out.cpu().numpy(), ref.cpu().numpy()) <= TOL_SHT
    finally:
        shot.shot_grid_free(g)


def test_noalloc_rejects_requests_beyond_its_scratch():
    g = shot.shot_grid_init(180)
    try:
        nf = 64   # spectra alone need ~16 MB > 8 MB
        f = torch.zeros((nf, 180, 360), device="cuda")
        out = torch.empty_like(f)
        rc = _call_abi(g, 1e-3, f, out)
        assert rc == shot.SHOT_ERR_INVALID_ARG
        assert "scratch" in shot.last_error()
    finally:
        shot.shot_grid_free(g)
