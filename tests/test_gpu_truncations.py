"""Truncated CCD (Eqs. ccd1, ccd2 and the linear terms of Eq. ccd3) and the third-order
diagrams (pnm_mbpt3) on the GPU against the FP64 oracle."""
import math

import numpy as np
import pytest

from conftest import minnesota_params
from oracle import channel

pytestmark = pytest.mark.gpu

TERMS = {"pp": 1, "pphh": 2, "linear": 3}


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


@pytest.fixture(scope="module")
def sys14(pkg):
    g = pkg.Context(14, 0.08, 20, params=minnesota_params())
    yield g, channel.OracleSystem(14, 0.08, 20, minnesota_params())
    g.close()


@pytest.mark.parametrize("terms", ["pp", "pphh", "linear"])
def test_truncated_iteration_matches_oracle(pkg, sys14, terms):
    g, o = sys14
    dE_o, it_o, h_o, _ = o.ccd(alpha=0.5, tol=1e-10, maxit=400, terms=terms)
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=400, terms=TERMS[terms])
    assert it[0] == it_o
    assert np.max(np.abs(g.history() - h_o) / np.abs(h_o)) < 1e-10
    abij, t_o = o.amplitudes()
    t_o = o.t_gather(g.amplitude_labels())
    assert np.max(np.abs(g.get_amplitudes() - t_o)) <= 1e-10 * np.max(np.abs(t_o))


def test_full_solve_after_truncations_and_mbpt3(pkg, sys14):
    """The fixed intermediates of a truncation and the MBPT3 pass leave nothing behind."""
    g, o = sys14
    g.solve(alpha=0.5, tol=1e-10, max_iter=400, terms=pkg.PNM_TERMS_PP)
    g.mbpt3()
    dE_o, it_o, _, _ = o.ccd(alpha=0.5, tol=1e-10, maxit=300)
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    assert it[0] == it_o and abs(dE[0] - dE_o) <= 1e-10 * abs(dE_o)


def test_truncations_are_fp64_only(pkg, sys14):
    g, _ = sys14
    with pytest.raises(pkg.PnmError) as e:
        g.solve(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-10, terms=pkg.PNM_TERMS_PPHH)
    assert e.value.code == -1


@pytest.mark.parametrize("N,rhos,n2,theta", [
    (14, [0.08], 20, None), (14, [0.04, 0.12], 20, None), (2, [0.08], 9, None),
    (14, [0.08], 20, [(2.9, 0.5, 1.7)]), (66, [0.16], 36, None)])
def test_mbpt3_matches_oracle(pkg, N, rhos, n2, theta):
    g = pkg.Context(N, rhos, n2, params=minnesota_params(), theta=theta)
    e3 = g.mbpt3()
    for s, rho in enumerate(rhos):
        o = channel.OracleSystem(N, rho, n2, minnesota_params(), theta=None if theta is None else theta[s])
        ref = o.mbpt3()
        assert np.max(np.abs(e3[s] - ref) / np.abs(ref)) < 1e-11, (s, e3[s], ref)
    g.close()


def test_first_truncated_step_is_mbpt3(pkg, sys14):
    """One unmixed step from the MBPT2 amplitudes adds the diagrams it contains (GPU only)."""
    g, _ = sys14
    d4, d5, d3 = g.mbpt3()[0]
    for terms, ref in ((pkg.PNM_TERMS_PP, d4), (pkg.PNM_TERMS_PPHH, d4 + d5),
                       (pkg.PNM_TERMS_LINEAR, d4 + d5 + d3)):
        g.solve(alpha=1.0, tol=1e-30, max_iter=1, terms=terms, allow=(pkg.PNM_ENOTCONV,))
        h = g.history()
        assert math.isclose(h[1] - h[0], ref, rel_tol=1e-11), terms
