"""The C-ABI library builds for sm_103a and exports every entry point that
include/dfl.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

import paper_2404_19634_gb300 as dfl

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "dfl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dfl_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return dfl.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dfl_create", "dfl_static", "dfl_apply_batch", "dfl_update",
                     "dfl_membership", "dfl_modularity", "dfl_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) == set(dfl._SIGS)


def test_build_targets_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in dfl.NVCC_FLAGS
    assert not any("sm_90" in f or "sm_100" in f for f in dfl.NVCC_FLAGS)
