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


def test_c_caller_compiles_and_links(libpath, tmp_path):
    """The header is plain C99 (no C++ needed by a caller) and a C program
    using the basic calls links against the library as built."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = os.path.join(os.path.dirname(__file__), "c_api_example.c")
    exe = str(tmp_path / "c_api_example")
    libdir = os.path.dirname(libpath)
    out = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                          "-I", os.path.dirname(HEADER), src, "-o", exe, "-L", libdir, "-ldfl",
                          "-Wl,-rpath," + libdir],
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert os.path.exists(exe)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every entry point raises."""
    monkeypatch.setattr(dfl, "_lib", None)
    monkeypatch.setattr(dfl, "_LIB", str(tmp_path / "absent" / "libdfl.so"))
    with pytest.raises(RuntimeError, match="not built"):
        dfl.Dfl(2, [0, 1, 2], [1, 0], [1, 1])
    with pytest.raises(RuntimeError, match="not built"):
        dfl.default_options()


def test_product_package_does_not_use_the_oracle():
    """The oracle is test infrastructure: nothing in the package imports,
    loads or runs it."""
    pkg = os.path.dirname(dfl.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert not re.search(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|dfl_oracle|liboracle", text), f
