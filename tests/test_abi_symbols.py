"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gp.h declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

from paper_1902_09215_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["gp_create_population", "gp_crossover", "gp_evaluate", "gp_fitness",
              "gp_tree_size", "gp_tree_read", "gp_destroy_population", "gp_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi(libpath):
    from paper_1902_09215_gb300 import gp
    for n in declared_functions():
        assert n in gp.EXPORTED, n
        if n not in ("gp_evaluate_ex",):
            assert hasattr(gp, n), n


def test_status_strings(libpath):
    from paper_1902_09215_gb300 import gp
    assert gp.gp_status_string(0) == "GP_OK"
    assert "malformed" in gp.gp_status_string(3)
    assert "unknown" in gp.gp_status_string(99)


def test_library_targets_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert "-fmad=false" in _build.NVCC_FLAGS and "-prec-div=true" in _build.NVCC_FLAGS


def test_product_path_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_1902_09215_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(from\s+oracle|import\s+oracle|liboracle|gp_oracle|oracle/)", src), f
