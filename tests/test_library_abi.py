"""CPU-side checks of the C-ABI library: it builds, loads, and exports every entry point that
include/tobk.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tobk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tobk_[A-Za-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1909_13585_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "tobk_create" in names and "tobk_solve_equilibrium" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    import paper_1909_13585_gb300 as pkg
    assert set(_declared()) == set(pkg.EXPORTED)


def test_product_path_has_no_oracle_import():
    pkg_dir = os.path.join(ROOT, "paper_1909_13585_gb300")
    for dp, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
