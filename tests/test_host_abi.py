"""Host-side logic of the C ABI that runs without a GPU: the matrix-convolution normaliser C(eps)
(computed on the host by composite Simpson) against the oracle's adaptive quadrature, and the
argument checks, which reject bad calls with SHOT_ERR_INVALID_ARG and a message before any CUDA
work."""
import ctypes
import math

import numpy as np
import pytest

from oracle import convolution as cv


@pytest.fixture(scope="module")
def lib():
    from paper_2605_18389_gb300 import shot
    import os
    if not os.path.exists(shot.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return shot.lib()


@pytest.mark.parametrize("eps", np.logspace(-3, 1, 8))
def test_gibbs_normaliser_matches_oracle(lib, eps):
    """C(eps) = 2 pi int_0^pi e^{-theta^2/eps} sin(theta) dtheta (App. "Convolution on S^2")."""
    c = ctypes.c_double()
    assert lib.shot_gibbs_normaliser(float(eps), ctypes.byref(c)) == 0
    assert abs(c.value / cv.gibbs_normaliser(float(eps)) - 1.0) < 1e-9


def _last_error(lib):
    buf = ctypes.create_string_buffer(512)
    lib.shot_last_error(buf, 512)
    return buf.value.decode()


def test_bad_arguments_are_rejected_without_a_gpu(lib):
    from paper_2605_18389_gb300 import shot
    c = ctypes.c_double()
    assert lib.shot_gibbs_normaliser(-1.0, ctypes.byref(c)) == shot.SHOT_ERR_INVALID_ARG
    assert "eps" in _last_error(lib)
    assert lib.shot_gibbs_normaliser(float("nan"), ctypes.byref(c)) == shot.SHOT_ERR_INVALID_ARG
    # no grid: every call that needs one refuses before touching the device
    assert lib.shot_heat_apply(None, 1e-3, None, None, 1, None) == shot.SHOT_ERR_INVALID_ARG
    assert "bad argument" in _last_error(lib)
    assert lib.shot_sinkhorn(None, None, None, 1, 0.1, math.inf, 10, 0.0, 10, 0, None, None, None, None, None,
                             None, None, None, None) == shot.SHOT_ERR_INVALID_ARG
    assert lib.shot_divergence(None, None, None, 1, 0.1, math.inf, 10, 0.0, 10, 0, None, None, None, None, None,
                               None, None, None) == shot.SHOT_ERR_INVALID_ARG
    assert "solver" in _last_error(lib)
    n = ctypes.c_longlong()
    assert lib.shot_launch_count(ctypes.byref(n)) == 0 and n.value >= 0
