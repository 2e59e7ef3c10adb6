"""Truncated CCD (Eqs. ccd1 and ccd2 of Sec. "Coupled cluster theory": the pp ladder, then
the pp and hh ladders, with the bare interaction) and the third-order energy (diagrams (3),
(4), (5) of Fig. goldstone), in the oracle.

Pins that do not come from the oracle itself:
  - Eqs. ccd1 and ccd2 are linear: per channel they are the Sylvester equation
    (E_pp + V_pp) T + T (V_hh - E_hh) = -v (V_hh = 0 for ccd1), solved here by scipy;
  - for two neutrons the sum of the three diagrams is the third-order Rayleigh-Schroedinger
    energy of the exact two-body Hamiltonian with the Moller-Plesset split, and MBPT2 its
    second order;
  - the dense engine (numpy, the paper's formulas) agrees with the channel engine;
  - one unmixed step of the truncated iteration from the MBPT2 amplitudes adds exactly the
    diagrams it contains to E2.
"""
import math

import numpy as np
import pytest
from scipy.linalg import solve_sylvester

from conftest import minnesota_params
from oracle import channel, dense, exact2, pw


def _sylvester_amplitudes(S, with_hh):
    """Amplitudes of Eq. ccd1 (with_hh False) or ccd2 by a direct solve per channel, as
    {(a, b, i, j): t} over restricted pairs."""
    tab = S.channel_tables()
    _, eps = S.energies()
    out = {}
    ho = po = 0
    for c, (nh, npp) in enumerate(zip(tab["nhh"], tab["npp"])):
        hh = tab["hh"][ho:ho + nh]
        pp = tab["pp"][po:po + npp]
        ho += nh
        po += npp
        Vpp = S.vpp_block(c)
        Vhh = np.array([[S.v(k, l, i, j) for (i, j) in hh] for (k, l) in hh]) if with_hh else np.zeros((nh, nh))
        v = np.array([[S.v(a, b, i, j) for (i, j) in hh] for (a, b) in pp])
        Epp = np.diag([eps[a] + eps[b] for a, b in pp])
        Ehh = np.diag([eps[i] + eps[j] for i, j in hh])
        T = solve_sylvester(Epp + Vpp, Vhh - Ehh, -v)
        for x, (a, b) in enumerate(pp):
            for y, (i, j) in enumerate(hh):
                out[(a, b, i, j)] = T[x, y]
    return out


@pytest.mark.parametrize("n2", [4, 20])
@pytest.mark.parametrize("terms", ["pp", "pphh"])
def test_ladder_truncations_solve_their_linear_equations(n2, terms):
    S = channel.OracleSystem(14, 0.08, n2, minnesota_params())
    dE, it, _, _ = S.ccd(alpha=0.5, tol=1e-13, maxit=2000, terms=terms)
    assert it < 2000
    ref = _sylvester_amplitudes(S, terms == "pphh")
    abij, t = S.amplitudes()
    tr = np.array([ref[tuple(r)] for r in abij.tolist()])
    assert np.max(np.abs(t - tr)) < 1e-9 * np.max(np.abs(tr))
    e_ref = sum(S.v(a, b, i, j) * x for (a, b, i, j), x in ref.items())
    assert math.isclose(dE, e_ref, rel_tol=1e-10)


@pytest.fixture(scope="module")
def cfg0():
    P = minnesota_params()
    N, rho, n2 = 14, 0.08, 4
    st = pw.basis(n2)
    L = pw.box_length(N, rho)
    D = dense.DenseCCD(pw.kinetic(st, L, P[6]), pw.v_dense(st, L, P), N)
    return D, channel.OracleSystem(N, rho, n2, P)


@pytest.mark.parametrize("terms", ["pp", "pphh", "linear"])
def test_dense_and_channel_truncations_agree(cfg0, terms):
    D, S = cfg0
    _, it1, h1, _ = D.solve(alpha=0.5, tol=1e-10, maxit=300, terms=terms)
    _, it2, h2, _ = S.ccd(alpha=0.5, tol=1e-10, maxit=300, terms=terms)
    assert it1 == it2
    assert np.max(np.abs(h1 - h2) / np.abs(h2)) < 1e-12


def test_dense_and_channel_mbpt3_agree(cfg0):
    D, S = cfg0
    a, b = D.mbpt3(), S.mbpt3()
    assert np.max(np.abs(a - b) / np.abs(b)) < 1e-12


def test_first_truncated_step_adds_its_diagrams(cfg0):
    _, S = cfg0
    d4, d5, d3 = S.mbpt3()
    for terms, ref in (("pp", d4), ("pphh", d4 + d5), ("linear", d4 + d5 + d3)):
        h = S.ccd(alpha=1.0, tol=1e-30, maxit=1, terms=terms)[2]
        assert math.isclose(h[1] - h[0], ref, rel_tol=1e-11), terms


@pytest.mark.parametrize("n2,theta", [(4, None), (9, None), (9, (3.8, 0.2, 0.1))])
def test_two_neutron_mbpt3_is_rayleigh_schroedinger(n2, theta):
    S = channel.OracleSystem(2, 0.08, n2, minnesota_params(), theta=theta)
    ekin, eps = S.energies()
    e2, e3 = exact2.rs_third_order(S.states(), ekin, eps, S.v, (0, 1))
    assert math.isclose(S.mbpt2(), e2, rel_tol=1e-12)
    d = S.mbpt3()
    assert math.isclose(d.sum(), e3, rel_tol=1e-10)
    assert abs(d[2]) > 0.5 * abs(e3)      # the ring diagram is not negligible here


def test_printed_diagram_3_misses_third_order():
    """Eq. (diag3) as printed (<bk|v|ic>) vanishes for two neutrons, so with (4) and (5) it
    does not give the Rayleigh-Schroedinger third order; the reading <kb|v|cj> does."""
    P = minnesota_params()
    st = pw.basis(4)
    L = pw.box_length(2, 0.08)
    v = pw.v_dense(st, L, P)
    D = dense.DenseCCD(pw.kinetic(st, L, P[6]), v, 2)
    t0 = D.mbpt2_guess()
    o, u = slice(0, 2), slice(2, len(st))
    printed = np.einsum("abij,bkic,acik->", t0, v[u, o, o, u], t0)
    assert abs(printed) < 1e-15
    e2, e3 = exact2.rs_third_order(st, pw.kinetic(st, L, P[6]), D.eps, lambda p, q, r, s: v[p, q, r, s], (0, 1))
    d4, d5, d3 = D.mbpt3()
    assert abs(d4 + d5 + printed - e3) > 0.1 * abs(e3)
    assert math.isclose(d4 + d5 + d3, e3, rel_tol=1e-10)
