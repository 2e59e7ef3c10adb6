"""The C-ABI library builds, loads and exports every symbol its header declares (no GPU
needed; no compute call is made)."""
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1611_06765_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "pnmcc.h")).read()
    return sorted(set(re.findall(r"\b(pnm_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    from paper_1611_06765_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_opts_and_errors_without_gpu(lib):
    import ctypes as C
    from paper_1611_06765_gb300 import _lib
    o = _lib.pnm_solve_opts()
    lib.pnm_default_opts(C.byref(o))
    assert o.precision == 0 and o.mix_alpha == 0.5 and o.tol_dE == 1e-10 and o.max_iter == 500
    # a null context is rejected before any CUDA call
    n = C.c_int()
    assert lib.pnm_num_systems(None, C.byref(n)) == _lib.PNM_EINVAL
    assert b"null" in lib.pnm_last_error()


def test_no_cpu_fallback_in_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1611_06765_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
