"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/dot.h declares (no GPU needed: no compute call is made here)."""
import os
import re
import subprocess

import pytest

from paper_1706_05586_gb300 import build as B
from paper_1706_05586_gb300 import dot as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "dot.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dot_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    if not os.path.exists(B.LIB):
        B.build()
    return B.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("dot_create", "dot_set_grid", "dot_set_pals", "dot_set_sampling", "dot_misfit",
                 "dot_gradient", "dot_jacobian_mua", "dot_jacobian_p", "dot_get_stats"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (dot_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_symbol(lib_path):
    assert sorted(D.SIGNATURES) == _declared()
    lib = D.load(lib_path)
    for name in D.SIGNATURES:
        assert hasattr(lib, name)
    assert D.dot_last_error() == ""


def test_library_is_built_for_sm_103a(lib_path):
    # cuobjdump is not used; the build flags are the evidence
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_binding_fails_loudly_without_library(tmp_path):
    saved = D._lib
    try:
        D._lib = None
        with pytest.raises(ImportError):
            D.load(str(tmp_path / "missing.so"))
    finally:
        D._lib = saved
