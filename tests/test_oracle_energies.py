"""Pins of the oracle's HF energies, E_ref and MBPT2 (arXiv:1611.06765 Eq. Hnormalorder and
the E_Ref expression, Eq. ccdGuess, Table tab:ecomparison)."""
import math

import numpy as np
import pytest

from conftest import minnesota_params, read_golden
from oracle import channel


def _gauss_sum(L, params, m):
    """sum over R, S of (V/L^3)(pi/kappa)^{3/2} exp(-q^2/4kappa) at q^2 = (2 pi / L)^2 m."""
    VR, kR, _, _, VS, kS, _ = params
    q2 = (2 * math.pi / L) ** 2 * m
    return sum(V / L ** 3 * (math.pi / k) ** 1.5 * math.exp(-q2 / (4 * k)) for V, k in ((VR, kR), (VS, kS)))


def test_eref_closed_form_N14():
    """For N = 14 the holes are 7 momenta {0, +-e_x, +-e_y, +-e_z} times two spins.  Only
    opposite-spin pairs interact, each with 1/2 [Vt(0) + Vt(k_i - k_j)].  Counting ordered
    momentum pairs (m, m'): 7 with |dn|^2 = 0, 12 with 1, 24 with 2, 6 with 4, the
    potential part 1/2 sum_ij <ij|v|ij> = 1/2 [56 Vt(0) + 12 Vt(1) + 24 Vt(2) + 6 Vt(4)]."""
    P = minnesota_params()
    N, rho = 14, 0.08
    S = channel.OracleSystem(N, rho, 4, P)
    L = S.L
    T = P[6] * (2 * math.pi / L) ** 2 * 12
    G = lambda m: _gauss_sum(L, P, m)
    pot = 0.5 * (56 * G(0) + 12 * G(1) + 24 * G(2) + 6 * G(4))
    assert math.isclose(S.eref(), T + pot, rel_tol=1e-13)


def test_hf_energies_are_diagonal_fock():
    """eps_p = h0_pp + sum_i <pi|v|pi>, checked against single elements."""
    P = minnesota_params()
    S = channel.OracleSystem(14, 0.08, 4, P)
    ekin, eps = S.energies()
    for p in (0, 5, 14, 30, 65):
        assert math.isclose(eps[p], ekin[p] + sum(S.v(p, i, p, i) for i in range(14)), rel_tol=1e-13)


def test_eref_two_neutrons():
    """N = 2: only the pair (0 down, 0 up) at k = 0; E_ref = Vt(0)."""
    P = minnesota_params()
    S = channel.OracleSystem(2, 0.08, 4, P)
    assert math.isclose(S.eref(), _gauss_sum(S.L, P, 0), rel_tol=1e-13)


@pytest.mark.parametrize("N,rho,n2max", [(14, 0.08, 4), (14, 0.08, 20), (2, 0.08, 20)])
def test_mbpt2_equals_first_ccd_iteration(N, rho, n2max):
    """One unmixed update from zero amplitudes gives the MBPT2 energy (text after
    Eq. ccdGuess)."""
    S = channel.OracleSystem(N, rho, n2max, minnesota_params())
    e_m2 = S.mbpt2()
    _, it, hist, _ = S.ccd(alpha=1.0, tol=0.0, maxit=1, init="zero")
    assert it == 1 and hist[0] == 0.0
    assert math.isclose(hist[1], e_m2, rel_tol=1e-12)


def _table():
    return [(float(r[0]), float(r[1]), float(r[2])) for r in read_golden("ecomparison.txt")]


@pytest.mark.parametrize("rho,e_mbpt2,e_ccd", _table())
def test_mbpt2_matches_ecomparison(rho, e_mbpt2, e_ccd):
    """Table tab:ecomparison, N = 66, n^2 <= 42: (E_ref + dE_MBPT2)/N to the printed three
    decimals.  hbar^2/2m is not printed, so the tolerance is one unit of the last digit."""
    S = channel.OracleSystem(66, rho, 42, minnesota_params())
    e = (S.eref() + S.mbpt2()) / 66
    assert abs(e - e_mbpt2) < 1.0e-3
