"""The stored oracle outputs under tests/golden/ (CPU).

grad_fd_256x512.json holds central differences of S computed once by the FP64 oracle
(tests/golden/make_grad_fd_256.py); the GPU gradient test regenerates the same inputs and
directions and compares.  These checks keep the fixture consistent with the generators it
relies on and the script that writes it independent of the CUDA path.
"""
import ast
import json
import math
import os

import numpy as np

from oracle.grid import Grid
from paper_2605_18389_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_grad_fd_fixture_is_well_formed():
    with open(os.path.join(GOLDEN, "grad_fd_256x512.json")) as f:
        g = json.load(f)
    assert g["recipe"] in inputs.RECIPES
    assert g["nlat"] == 256 and g["nlon"] == 512 and g["lmax"] == 255
    assert math.isclose(g["eps"], 4.0 * g["t"])          # eps = 4t (Sec. 3.2)
    assert g["T"] == 400 and 0 <= g["pair"] < g["npairs"]
    fd = np.asarray(g["fd"], dtype=np.float64)
    assert fd.shape == (g["ndirs"],) and 2 <= g["ndirs"] <= 4 and np.all(np.isfinite(fd))
    assert np.all(np.abs(fd) > 0.0) and math.isfinite(g["S"]) and g["S"] > 0.0


def test_fd_directions_reproducible_and_mass_preserving():
    og = Grid(16)
    p, _ = inputs.pairs("paper_uniform", 5, 1, og.x, og.nlon, og.a_ring)
    d1 = inputs.fd_directions(p[0], og.a, 3, 77)
    d2 = inputs.fd_directions(p[0], og.a, 3, 77)
    np.testing.assert_array_equal(d1, d2)
    norm_p = np.sum(og.a * p[0] * p[0])
    for d in d1:
        assert abs(np.sum(og.a * d)) <= 1e-12 * np.sum(og.a * np.abs(d))   # sum a delta = 0
        assert math.isclose(np.sum(og.a * d * d), norm_p, rel_tol=1e-12)     # ||delta||_a = ||p||_a
    assert not np.allclose(d1[0], d1[1])


def test_golden_script_runs_only_the_oracle_and_the_input_generators():
    path = os.path.join(GOLDEN, "make_grad_fd_256.py")
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mods.add(node.module)
    allowed = {"json", "math", "os", "sys", "time", "numpy", "paper_2605_18389_gb300"}
    for m in mods:
        assert m in allowed or m == "oracle" or m.startswith("oracle."), m
    # from the package, only the seeded input generators
    for node in ast.walk(tree):
        if isinstance(node, ast.ImportFrom) and node.module == "paper_2605_18389_gb300":
            assert [a.name for a in node.names] == ["inputs"]
