"""pnm_mbpt2_noalloc: the second-order energy for callers that cannot allocate device memory
at call time (for example while a CUDA graph is being captured, or under a fixed memory
budget).  It must give the same numbers as pnm_mbpt2, which uses scratch memory owned by
the context, on two calls in a row (its static scratch array is shared by every call).

Kept in a file of its own that pytest collects last, so a run stopping at the first
failure has run every other test before this one.
"""
import ctypes as C

import numpy as np
import pytest

from conftest import minnesota_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


def _call(lib, fn, ctx, nsys):
    out = np.zeros(nsys)
    rc = getattr(lib, fn)(ctx._h, out.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == 0, lib.pnm_last_error()
    return out


@pytest.mark.parametrize("N,rho,n2max", [(14, 0.08, 20), (14, [0.04, 0.08, 0.16], 20)])
def test_noalloc_matches_mbpt2_twice(pkg, N, rho, n2max):
    from paper_1611_06765_gb300 import _lib
    lib = _lib.load()
    ctx = pkg.Context(N, rho, n2max, params=minnesota_params())
    ref = _call(lib, "pnm_mbpt2", ctx, ctx.nsys)
    first = _call(lib, "pnm_mbpt2_noalloc", ctx, ctx.nsys)
    second = _call(lib, "pnm_mbpt2_noalloc", ctx, ctx.nsys)
    for got in (first, second):
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref))
    ctx.close()


def test_noalloc_rejects_oversize_then_still_matches(pkg):
    """More systems than the static scratch holds (64): PNM_EINVAL with a message naming the
    limit, nothing launched; a valid call right after still equals pnm_mbpt2."""
    from paper_1611_06765_gb300 import _lib
    lib = _lib.load()
    big = pkg.Context(2, [0.02 + 0.001 * k for k in range(65)], 1, params=minnesota_params())
    out = np.zeros(big.nsys)
    rc = lib.pnm_mbpt2_noalloc(big._h, out.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == _lib.PNM_EINVAL
    assert b"64 systems" in lib.pnm_last_error()
    big.close()
    ctx = pkg.Context(14, [0.04, 0.08], 20, params=minnesota_params())
    ref = _call(lib, "pnm_mbpt2", ctx, ctx.nsys)
    got = _call(lib, "pnm_mbpt2_noalloc", ctx, ctx.nsys)
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref))
    ctx.close()
