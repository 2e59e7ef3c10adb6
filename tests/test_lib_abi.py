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
    assert o.terms == _lib.PNM_TERMS_FULL and C.sizeof(o) == 56
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


def test_twist_mesh_is_gauss_legendre(lib):
    """pnm_twist_mesh is host code (no GPU): per axis it must be numpy's Gauss-Legendre rule
    mapped to [0, pi], and the product weights integrate polynomials of the axis degree
    exactly (the average of theta_x^2 theta_y theta_z^3 over [0, pi]^3 is pi^2/3 * pi/2 * pi^3/4)."""
    import math

    import numpy as np
    import paper_1611_06765_gb300 as P
    for n in (1, 2, 5, 16, 64):
        x, w = np.polynomial.legendre.leggauss(n)
        th, wt = P.twist_mesh(n, 1, 1)
        assert np.max(np.abs(th[:, 0] - (x + 1) * math.pi / 2)) < 1e-13
        assert np.max(np.abs(2 * wt - w)) < 1e-13
        assert np.all(th[:, 1:] == math.pi / 2)
    th, wt = P.twist_mesh(4, 5, 6)
    assert th.shape == (120, 3) and abs(wt.sum() - 1) < 1e-14
    assert abs(np.sum(wt * th[:, 0] ** 2 * th[:, 1] * th[:, 2] ** 3) - math.pi ** 6 / 24) < 1e-11
    assert len({tuple(r) for r in th}) == 120
    assert not np.any((th[:, 0] == th[:, 1]) | (th[:, 1] == th[:, 2]) | (th[:, 0] == th[:, 2]))
    assert lib.pnm_twist_mesh(0, 1, 1, None, None) == P._lib.PNM_EINVAL
