"""Batched uneven grids in one solve (shot_divergence_multi) and graph-replayed blocks.

Each set's result must equal the oracle's divergence of that set alone (per-problem tau on
a shared grid), and the multi-grid solve must equal the single-grid calls.
"""
import math

import numpy as np
import pytest

from oracle.grid import Grid as OGrid
from oracle import sinkhorn as sk
from paper_2605_18389_gb300 import inputs
from tests.gpu_util import f32, s_err, assert_s, FP32_S_LIMIT

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2605_18389_gb300 import shot  # noqa: E402

TOL_S = 1e-5


def _set(og, seed, npairs, masses):
    p, q = inputs.pairs("paper_uniform", seed, npairs, og.x, og.nlon, og.a_ring, masses=masses)
    p32, p64 = f32(p)
    q32, q64 = f32(q)
    return torch.from_numpy(p32).cuda(), torch.from_numpy(q32).cuda(), p64, q64


def test_multi_grid_sets_match_oracle_and_single_calls():
    eps, T = 0.1, 40   # well-posed on all four grids (the oracle breaks down at eps 0.02 on nlat 16)
    specs = [(16, 1.0), (16, math.inf), (24, 0.1), (32, 10.0)]   # grid nlat, tau
    grids = {n: (shot.shot_grid_init(n), OGrid(n)) for n in (16, 24, 32)}
    try:
        sets, refs, singles = [], [], []
        for i, (n, tau) in enumerate(specs):
            g, og = grids[n]
            pt, qt, p64, q64 = _set(og, 900 + i, 2, not math.isinf(tau))
            sets.append(dict(grid=g, p=pt, q=qt, eps=eps, tau=tau))
            refs.append(sk.divergence(og, p64, q64, eps, tau, T=T, delta=0.0, C=10))
        rc, outs = shot.shot_divergence_multi(sets, max_iter=T, tol=0.0, check_every=10)
        assert rc >= 0
        for st, o, ref in zip(sets, outs, refs):
            assert np.all(o["status"] == 0)
            rc1, r1 = shot.shot_divergence(st["grid"], st["p"], st["q"], eps, st["tau"], max_iter=T, tol=0.0,
                                           check_every=10)
            singles.append(r1)
            np.testing.assert_allclose(o["S"], r1["S"], rtol=1e-6, atol=1e-9)
        for o, ref in zip(outs, refs):   # S against the oracle last (FP32: see FP32_S_LIMIT)
            ot_pq = ref["runs"]["ot"][: len(o["S"])]
            assert_s(o["S"], ref["S"], ot_pq, TOL_S, limited_by=FP32_S_LIMIT)
            assert_s(o["S_dual"], ref["S_dual"], ot_pq, TOL_S, limited_by=FP32_S_LIMIT)
    finally:
        for g, _ in grids.values():
            shot.shot_grid_free(g)


def test_graph_replay_equals_profiled_eager_launches():
    # blocks are captured into a CUDA graph unless per-launch profiling is on: same numbers
    og = OGrid(24)
    g = shot.shot_grid_init(24)
    try:
        pt, qt, _, _ = _set(og, 5, 3, False)
        rc, r_graph = shot.shot_divergence(g, pt, qt, 0.05, max_iter=60, tol=0.0, check_every=10)
        shot.shot_profile_enable(True)
        try:
            rc, r_eager = shot.shot_divergence(g, pt, qt, 0.05, max_iter=60, tol=0.0, check_every=10)
        finally:
            shot.shot_profile_enable(False)
            shot.shot_profile_read()
        np.testing.assert_array_equal(r_graph["S"], r_eager["S"])
    finally:
        shot.shot_grid_free(g)


def test_configuration3_sets_with_scalings_beyond_fp32():
    """Configuration 3's kind of batch at eps = 0.01 (t = 2.5e-3): tau in {0.1, 1, 10} with
    masses far apart (0.6 vs 1.7 and 1.8 vs 0.55) on one grid in one solve.  At tau = 10 the
    potentials reach ~6 = 600 eps, so the scalings leave FP32 (the solver carries them as FP32
    buffers times FP64 factors); S matches the FP64 oracle for every set."""
    eps, T = 0.01, 40
    g, og = shot.shot_grid_init(64), OGrid(64)
    try:
        sets, refs = [], []
        for i, tau in enumerate((0.1, 1.0, 10.0)):
            p, q = inputs.pairs("paper_uniform", 3300 + i, 2, og.x, og.nlon, og.a_ring)
            p32, p64 = f32(p * np.array([0.6, 1.8])[:, None, None])
            q32, q64 = f32(q * np.array([1.7, 0.55])[:, None, None])
            sets.append(dict(grid=g, p=torch.from_numpy(p32).cuda(), q=torch.from_numpy(q32).cuda(), eps=eps,
                             tau=tau))
            refs.append(sk.divergence(og, p64, q64, eps, tau, T=T, delta=0.0, C=10))
        assert np.max(np.abs(refs[2]["runs"]["phi"])) / eps > 200.0
        rc, outs = shot.shot_divergence_multi(sets, max_iter=T, tol=0.0, check_every=10)
        assert rc >= 0
        for o, ref in zip(outs, refs):
            assert np.all(o["status"] == 0) and np.all(ref["status"] == 0)
            ot_pq = ref["runs"]["ot"][: len(o["S"])]
            assert np.all(s_err(o["S"], ref["S"], ot_pq, TOL_S) <= 1.0), (o["S"], ref["S"])
    finally:
        shot.shot_grid_free(g)


def test_configuration3_grids_in_one_solve_match_oracle():
    """Configuration 3's own grids, 64/96/128/180 rings (nlon = 2 nlat), in one
    shot_divergence_multi solve: one set per grid, tau cycling through {0.1, 1, 10} plus a
    balanced set, masses U[0.5, 2] per field, eps = 0.01 (t = 2.5e-3), 20 iterations.  Each set's
    S and S_dual against the FP64 oracle, and against the same set solved alone."""
    eps, T = 0.01, 20
    specs = [(64, 0.1), (96, 1.0), (128, 10.0), (180, math.inf)]
    grids = {n: (shot.shot_grid_init(n), OGrid(n)) for n, _ in specs}
    try:
        sets, refs = [], []
        for i, (n, tau) in enumerate(specs):
            g, og = grids[n]
            pt, qt, p64, q64 = _set(og, 3900 + i, 1, not math.isinf(tau))
            sets.append(dict(grid=g, p=pt, q=qt, eps=eps, tau=tau))
            refs.append(sk.divergence(og, p64, q64, eps, tau, T=T, delta=0.0, C=10))
        rc, outs = shot.shot_divergence_multi(sets, max_iter=T, tol=0.0, check_every=10)
        assert rc >= 0
        for st, o in zip(sets, outs):
            assert np.all(o["status"] == 0)
            rc1, r1 = shot.shot_divergence(st["grid"], st["p"], st["q"], eps, st["tau"], max_iter=T, tol=0.0,
                                           check_every=10)
            np.testing.assert_allclose(o["S"], r1["S"], rtol=1e-6, atol=1e-9)
        for o, ref in zip(outs, refs):
            assert np.all(ref["status"] == 0)
            ot_pq = ref["runs"]["ot"][: len(o["S"])]
            assert_s(o["S"], ref["S"], ot_pq, TOL_S, limited_by=FP32_S_LIMIT)
            assert_s(o["S_dual"], ref["S_dual"], ot_pq, TOL_S, limited_by=FP32_S_LIMIT)
    finally:
        for g, _ in grids.values():
            shot.shot_grid_free(g)
