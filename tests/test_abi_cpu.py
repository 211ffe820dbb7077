"""CPU-only checks of the C-ABI library: it builds, loads and exports every declared symbol.

No compute call is made here (there is no GPU on the build host).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "ihsbin.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ihsbin_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def so_path():
    from paper_2210_12212_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for want in ["ihsbin_sketch", "ihsbin_build_basis", "ihsbin_eval_path", "ihsbin_problem_create"]:
        assert want in names


def test_library_exports_every_declared_symbol(so_path):
    lib = ctypes.CDLL(so_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(so_path):
    from paper_2210_12212_gb300 import ihsbin as ihs
    assert set(ihs.EXPORTED) >= set(declared_functions())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2210_12212_gb300 import ihsbin as ihs
    saved = ihs._lib
    ihs._lib = None
    try:
        with pytest.raises(RuntimeError):
            ihs.load(str(tmp_path / "missing.so"))
    finally:
        ihs._lib = saved
