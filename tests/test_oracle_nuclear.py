"""Nuclear matter in the oracle: protons and neutrons with the full Minnesota operator
(Sec. "Two-body interaction": V = 1/2 (V_R + 1/2(1+P_s) V_T + 1/2(1-P_s) V_S)(1 - P_s P_t)),
channels keyed by (P, S_z, T_z) (Sec. "Infinite nuclear matter" and the channel index of Sec.
"Developing a CCD code").

Pins that do not come from the oracle itself:
  - pure proton matter is pure neutron matter (no Coulomb term: charge symmetry), energy by
    energy and channel by channel;
  - the interaction written out by hand with spin and isospin Kronecker deltas (numpy) equals
    the oracle's 16 x 16 operator algebra element by element, and the dense engine on it
    (Eq. ccd3 term by term) reproduces the channel engine's E_ref, MBPT2, CCD and MBPT3;
  - E_ref in closed form: with every spin-isospin state of a momentum filled, the trace of each
    operator over the 16 two-nucleon labels gives 1/2 sum_{k,k'} [6 V_R + 3 V_T + 3 V_S at
    q = 0 and at q = k - k'] (the V_T term is present only because np pairs exist);
  - antisymmetry, hermiticity, conservation of P, S_z, T_z, and p <-> n label symmetry of V.
"""
import math

import numpy as np
import pytest

from conftest import minnesota_params
from oracle import channel, dense, pw


def test_proton_matter_is_neutron_matter():
    P = minnesota_params()
    n = channel.OracleSystem(14, 0.08, 20, P)
    p = channel.OracleSystem(0, 0.08, 20, P, Z=14)
    assert np.array_equal(p.states()[:, :4], n.states())
    assert np.all(p.states()[:, 4] == -1)
    tn, tp = n.channel_tables(), p.channel_tables()
    assert np.array_equal(tn["nhh"], tp["nhh"]) and np.array_equal(tn["npp"], tp["npp"])
    for f in ("eref", "mbpt2"):
        assert math.isclose(getattr(n, f)(), getattr(p, f)(), rel_tol=1e-13), f
    a = n.ccd(alpha=0.5, tol=1e-10, maxit=300)
    b = p.ccd(alpha=0.5, tol=1e-10, maxit=300)
    assert a[1] == b[1] and np.max(np.abs(a[2] - b[2]) / np.abs(a[2])) < 1e-12
    assert np.max(np.abs(n.mbpt3() - p.mbpt3())) < 1e-12 * np.max(np.abs(n.mbpt3()))


@pytest.fixture(scope="module", params=[1, 2])
def snm4(request):
    P = minnesota_params()
    n2 = request.param
    st = pw.basis(n2, species="np")
    L = pw.box_length(4, 0.16)
    v = pw.v_dense_nucleons(st, L, P)
    return st, L, v, channel.OracleSystem(2, 0.16, n2, P, Z=2)


def test_hand_written_interaction_matches_operator_algebra(snm4):
    st, L, v, S = snm4
    assert np.array_equal(S.states(), st.astype(np.int32))
    rng = np.random.default_rng(3)
    n = len(st)
    vmax = np.max(np.abs(v))
    hits = 0
    for _ in range(4000):
        p, q, r = (int(x) for x in rng.integers(0, n, 3))
        # a partner that conserves momentum, spin and isospin, so most samples are nonzero
        tgt = st[p] + st[q] - st[r]
        cand = np.where(np.all(st == tgt, axis=1))[0]
        s = int(cand[0]) if len(cand) else int(rng.integers(0, n))
        assert abs(v[p, q, r, s] - S.v(p, q, r, s)) <= 1e-13 * vmax
        hits += abs(v[p, q, r, s]) > 0
    assert hits > 500


def test_dense_engine_matches_channel_engine(snm4):
    st, L, v, S = snm4
    P = minnesota_params()
    D = dense.DenseCCD(pw.kinetic(st, L, P[6]), v, 4)
    assert math.isclose(D.eref, S.eref(), rel_tol=1e-13)
    assert math.isclose(D.energy(D.mbpt2_guess()), S.mbpt2(), rel_tol=1e-12)
    _, it1, h1, _ = D.solve(alpha=0.5, tol=1e-10, maxit=300)
    _, it2, h2, _ = S.ccd(alpha=0.5, tol=1e-10, maxit=300)
    assert it1 == it2 and np.max(np.abs(h1 - h2) / np.abs(h2)) < 1e-12
    assert np.max(np.abs(D.mbpt3() - S.mbpt3()) / np.abs(S.mbpt3())) < 1e-11


@pytest.mark.parametrize("A,rho,n2", [(4, 0.16, 4), (28, 0.16, 9), (28, 0.08, 9)])
def test_reference_energy_closed_form(A, rho, n2):
    P = minnesota_params()
    VR, kR, VT, kT, VS, kS, h = P
    S = channel.OracleSystem(A // 2, rho, n2, P, Z=A // 2)
    st = S.states()
    assert np.sum(st[:A, 4] == 1) == A // 2
    ks = np.unique(st[:A, :3], axis=0)
    assert len(ks) * 4 == A
    L = S.L
    k0 = 2 * math.pi / L
    T = h * k0 * k0 * 4 * np.sum(ks ** 2)
    g = lambda V, kap, q2: V / L ** 3 * (math.pi / kap) ** 1.5 * math.exp(-q2 / (4 * kap))
    w = lambda q2: 6 * g(VR, kR, q2) + 3 * g(VT, kT, q2) + 3 * g(VS, kS, q2)
    epot = 0.0
    for a in ks:
        for b in ks:
            epot += 0.5 * (w(0.0) + w(k0 * k0 * float(np.sum((a - b) ** 2))))
    assert math.isclose(S.eref(), T + epot, rel_tol=1e-12)
    # without V_T the np pairs lose exactly their triplet part
    P0 = (VR, kR, 0.0, kT, VS, kS, h)
    S0 = channel.OracleSystem(A // 2, rho, n2, P0, Z=A // 2)
    w0 = lambda q2: 6 * g(VR, kR, q2) + 3 * g(VS, kS, q2)
    epot0 = sum(0.5 * (w0(0.0) + w0(k0 * k0 * float(np.sum((a - b) ** 2)))) for a in ks for b in ks)
    assert math.isclose(S0.eref(), T + epot0, rel_tol=1e-12)


def test_interaction_symmetries():
    P = minnesota_params()
    S = channel.OracleSystem(2, 0.16, 2, P, Z=2)
    st = S.states()
    n = len(st)
    swap = {}
    for p in range(n):                     # p <-> n label exchange
        tgt = st[p].copy()
        tgt[4] = -tgt[4]
        swap[p] = int(np.where(np.all(st == tgt, axis=1))[0][0])
    rng = np.random.default_rng(5)
    for _ in range(1500):
        p, q, r, s = (int(x) for x in rng.integers(0, n, 4))
        x = S.v(p, q, r, s)
        assert abs(x + S.v(q, p, r, s)) < 1e-13 and abs(x + S.v(p, q, s, r)) < 1e-13
        assert abs(x - S.v(r, s, p, q)) < 1e-13
        assert abs(x - S.v(swap[p], swap[q], swap[r], swap[s])) < 1e-13
        cons = np.array_equal(st[p] + st[q], st[r] + st[s])
        if not cons:
            assert x == 0.0
