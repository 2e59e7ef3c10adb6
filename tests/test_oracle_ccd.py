"""Pins of the oracle's CCD engines (arXiv:1611.06765 Eqs. ccd, ccd3, ccdcorr and the
intermediates of Sec. "Developing a CCD code").

- The dense engine (every term of Eq. ccd as printed) against the paper's pairing-model
  table tab:selectedbenchmarks and its closed-form MBPT2.
- The dense engine against the channel engine (intermediates, restricted blocks).
- Two neutrons: CCD is exact, so it must equal exact diagonalisation.
- Table tab:ecomparison (N = 66) for the CCD column.
"""
import math

import numpy as np
import pytest

from conftest import minnesota_params, read_golden
from oracle import channel, dense, exact2, pairing, pw


def _pairing_rows():
    return [tuple(float(x) for x in r) for r in read_golden("pairing_selectedbenchmarks.txt")]


def test_pairing_hamiltonian_matches_paper():
    rows = read_golden("pairing_hamiltonian.txt")
    for g in (-1.0, 0.5, 1.0):
        expect = np.zeros((6, 6))
        for r, c, cd, cg in rows:
            expect[int(r), int(c)] = expect[int(c), int(r)] = float(cd) * 1.0 + float(cg) * g
        _, H = pairing.fci_ground(g)
        assert np.allclose(H, expect, atol=1e-15)


@pytest.mark.parametrize("g,eref,mbpt2,eccd", _pairing_rows())
def test_pairing_table(g, eref, mbpt2, eccd):
    h0, v = pairing.hamiltonian(g)
    D = dense.DenseCCD(h0, v, 4)
    assert math.isclose(D.eref, eref, abs_tol=1e-12)
    e2 = D.energy(D.mbpt2_guess())
    # closed form printed below Eq. (smartMBPT)'s pairing example
    closed = -g * g / 4 * (1 / (4 + g) + 1 / (6 + g) + 1 / (2 + g) + 1 / (4 + g))
    assert math.isclose(e2, closed, rel_tol=1e-12, abs_tol=1e-15)
    assert abs(e2 - mbpt2) < 5e-6
    dE, it, _, _ = D.solve(alpha=0.5, tol=1e-12, maxit=2000)
    assert it < 2000
    assert abs(dE - eccd) < 5e-6


def test_pairing_g_minus_one_needs_mixing():
    """Text below tab:selectedbenchmarks: g = -1 does not settle without mixing."""
    h0, v = pairing.hamiltonian(-1.0)
    D = dense.DenseCCD(h0, v, 4)
    dE, it, _, _ = D.solve(alpha=1.0, tol=1e-12, maxit=300)
    assert it == 300 or abs(dE - (-0.21895)) > 1e-3


@pytest.fixture(scope="module")
def cfg0():
    P = minnesota_params()
    N, rho, n2 = 14, 0.08, 4
    st = pw.basis(n2)
    v = pw.v_dense(st, pw.box_length(N, rho), P)
    D = dense.DenseCCD(pw.kinetic(st, pw.box_length(N, rho), P[6]), v, N)
    S = channel.OracleSystem(N, rho, n2, P)
    return D, S


def test_dense_and_channel_engines_agree(cfg0):
    D, S = cfg0
    N = 14
    assert math.isclose(D.eref, S.eref(), rel_tol=1e-13)
    dE1, it1, h1, t1 = D.solve(alpha=0.5, tol=1e-10, maxit=300)
    dE2, it2, h2, _ = S.ccd(alpha=0.5, tol=1e-10, maxit=300)
    assert it1 == it2
    assert np.max(np.abs(h1 - h2) / np.abs(h2)) < 1e-12
    abij, tc = S.amplitudes()
    td = t1[abij[:, 0] - N, abij[:, 1] - N, abij[:, 2], abij[:, 3]]
    assert np.max(np.abs(td - tc)) < 1e-12 * np.max(np.abs(tc))


def test_dense_energy_and_antisymmetry(cfg0):
    D, _ = cfg0
    t = D.mbpt2_guess()
    t = 0.5 * D.step(t) + 0.5 * t
    assert np.allclose(t, -t.transpose(1, 0, 2, 3), atol=0)
    assert np.allclose(t, -t.transpose(0, 1, 3, 2), atol=0)


@pytest.mark.parametrize("n2max", [4, 20])
def test_two_neutrons_ccd_is_exact(n2max):
    P = minnesota_params()
    S = channel.OracleSystem(2, 0.08, n2max, P)
    ekin, _ = S.energies()
    E0, Eref, _ = exact2.ground_state(S.states(), ekin, S.v, (0, 1))
    assert math.isclose(Eref, S.eref(), rel_tol=1e-13)
    dE, it, _, _ = S.ccd(alpha=0.5, tol=1e-13, maxit=500)
    assert it < 500
    assert abs(dE - (E0 - Eref)) < 1e-10 * abs(E0)


def test_two_neutrons_dense_is_exact():
    P = minnesota_params()
    N, rho, n2 = 2, 0.08, 4
    st = pw.basis(n2)
    L = pw.box_length(N, rho)
    v = pw.v_dense(st, L, P)
    D = dense.DenseCCD(pw.kinetic(st, L, P[6]), v, N)
    E0, Eref, _ = exact2.ground_state(st, pw.kinetic(st, L, P[6]), lambda p, q, r, s: v[p, q, r, s], (0, 1))
    dE, _, _, _ = D.solve(alpha=0.5, tol=1e-13, maxit=500)
    assert abs(dE - (E0 - Eref)) < 1e-10 * abs(E0)


def _ccd_rows():
    # The rho = 0.08 CCD entry (9.136) is not reproduced by this reading (9.105); the
    # MBPT2 column of the same row is.  It is kept out of the pin set.
    return [r for r in [(float(a), float(b), float(c)) for a, b, c in read_golden("ecomparison.txt")]
            if r[0] in (0.04, 0.06)]


@pytest.mark.parametrize("rho,e_mbpt2,e_ccd", _ccd_rows())
def test_ccd_matches_ecomparison(rho, e_mbpt2, e_ccd):
    S = channel.OracleSystem(66, rho, 42, minnesota_params())
    er = S.eref()
    dE, it, _, _ = S.ccd(alpha=0.5, tol=1e-8, maxit=200)
    assert it < 200
    assert abs((er + dE) / 66 - e_ccd) < 1.0e-3


def _library_labels(S):
    """(a, b, i, j) of each restricted amplitude in the library layout (per channel n_hh x
    n_pp, hh rows, pp contiguous)."""
    tab = S.channel_tables()
    out = []
    ho = po = 0
    for nh, npp in zip(tab["nhh"], tab["npp"]):
        hh = tab["hh"][ho:ho + nh]
        pp = tab["pp"][po:po + npp]
        for i, j in hh:
            for a, b in pp:
                out.append((a, b, i, j))
        ho += nh
        po += npp
    return np.array(out, dtype=np.int64).reshape(-1, 4)


def test_ph_term_matches_dense(cfg0):
    """The channel engine's P(ij)P(ab) sum_kc t_ik^ac chi_kb^cj (cross-channel T, C, Q) equals
    the dense Eq. (ccd3) terms it stands for, P(ij)P(ab) sum_kc <kb|v|cj> t_ik^ac +
    P(ij) sum_klcd <kl|v|cd> t_ik^ac t_jl^bd, on random antisymmetric amplitudes."""
    D, S = cfg0
    N = 14
    lab = _library_labels(S)
    rng = np.random.default_rng(21)
    t = rng.normal(0.0, 0.05, len(lab))
    td = np.zeros_like(D.D)
    a, b, i, j = lab[:, 0] - N, lab[:, 1] - N, lab[:, 2], lab[:, 3]
    td[a, b, i, j] = t
    td[b, a, i, j] = -t
    td[a, b, j, i] = -t
    td[b, a, j, i] = t
    lin = dense.P_ij(dense.P_ab(np.einsum("kbcj,acik->abij", D.v_kbcj, td)))
    quad = dense.P_ij(np.einsum("klcd,acik,bdjl->abij", D.v_klcd, td, td, optimize=True))
    ref = (lin + quad)[a, b, i, j]
    got = S.ph_apply(t)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    bound = S.ph_apply(t, absval=True)
    assert np.all(bound >= np.abs(got) - 1e-15)


def _scan():
    """Rows (n2max, hbar2_2m, rho, states, E_MBPT2/N, E_CCD/N) of the oracle scan of the readings
    of Table tab:ecomparison (tests/golden/ecomparison_scan.py wrote them from the oracle)."""
    return [(int(a), float(b), float(c), int(d), float(e), float(f))
            for a, b, c, d, e, f, _ in read_golden("ecomparison_scan.txt")]


def test_no_scanned_reading_gives_the_printed_rho008_ccd_entry():
    """Table tab:ecomparison prints E_CCD/N = 9.136 at rho = 0.08 beside E_MBPT2/N = 9.075.
    Among the spherical bases n^2 <= 36 ... 46 and hbar^2/2m in {20.721, 20.7355}, exactly one
    reading reproduces the other five entries of the three rows to one unit of the printed
    third decimal (n^2 <= 42, 2378 states, 20.721), and none gives 9.136 together with MBPT2
    9.075: the CCD - MBPT2 gap at rho = 0.08 stays between 0.025 and 0.035 MeV for every reading
    (printed: 0.061), so the printed CCD entry is taken as a misprint."""
    printed = {(float(r), "mbpt2"): float(m) for r, m, _ in read_golden("ecomparison.txt")}
    printed.update({(float(r), "ccd"): float(c) for r, _, c in read_golden("ecomparison.txt")})
    rows = _scan()
    readings = sorted({(n2, h) for n2, h, *_ in rows})
    full_match = []
    for n2, h in readings:
        got = {(rho, kind): val for n, hh, rho, _, m, c in rows if (n, hh) == (n2, h)
               for kind, val in (("mbpt2", m), ("ccd", c))}
        ok = {k: abs(got[k] - v) <= 1.0e-3 for k, v in printed.items()}
        if all(v for k, v in ok.items() if k != (0.08, "ccd")):
            full_match.append((n2, h))
        assert not (ok[(0.08, "ccd")] and ok[(0.08, "mbpt2")]), (n2, h)
        gap = got[(0.08, "ccd")] - got[(0.08, "mbpt2")]
        assert 0.025 < gap < 0.035, (n2, h, gap)
    assert full_match == [(42, 20.721)]
    assert abs(printed[(0.08, "ccd")] - printed[(0.08, "mbpt2")] - 0.061) < 1e-9


@pytest.mark.slow
@pytest.mark.parametrize("rho", [0.04, 0.06, 0.08])
def test_ecomparison_scan_rows_reproduce(rho):
    """The stored scan rows of the reading kept (n^2 <= 42, hbar^2/2m = 20.721) are the oracle's."""
    row = [r for r in _scan() if r[0] == 42 and r[1] == 20.721 and r[2] == rho][0]
    P = minnesota_params()
    S = channel.OracleSystem(66, rho, 42, P)
    er = S.eref()
    assert abs((er + S.mbpt2()) / 66 - row[4]) < 2e-6
    dE, _, _, _ = S.ccd(alpha=0.5, tol=1e-10 * 66, maxit=400)
    assert abs((er + dE) / 66 - row[5]) < 2e-6
