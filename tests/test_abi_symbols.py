"""The C-ABI library loads and exports every entry point include/shot.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "shot.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\bint\s+(shot_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("shot_grid_init", "shot_heat_apply", "shot_sinkhorn", "shot_divergence"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2605_18389_gb300 import shot
    if not os.path.exists(shot.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    lib = ctypes.CDLL(shot.LIB_PATH)
    for n in declared():
        assert hasattr(lib, n), n
    # and the binding knows each of them, with the same name
    assert set(declared()) <= set(shot.SIGNATURES)


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2605_18389_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), f
