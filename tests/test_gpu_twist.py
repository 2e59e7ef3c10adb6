"""Twisted boundary conditions on the GPU (``pnm_create_twisted``, ``pnm_twist_mesh``)
against the FP64 oracle: reordered basis and channel tables bit-exact, energies and the CCD
iteration as in the periodic parity tests, and a batched twist-averaged solve (one system
per mesh point, all in one grouped context) in FP64 and in the mixed path.
"""
import math

import numpy as np
import pytest

from conftest import minnesota_params
from oracle import channel, exact2

pytestmark = pytest.mark.gpu

TWISTS = [(0.4, 1.3, 2.6), (2.9, 0.5, 1.7), (2.0, 2.0, 0.7)]


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 20), (66, 0.16, 36)])
def test_twisted_tables_bit_exact(pkg, N, rho, n2):
    twists = TWISTS if N == 14 else TWISTS[:1]
    g = pkg.Context(N, rho, n2, params=minnesota_params(), theta=twists)
    for s, th in enumerate(twists):
        o = channel.OracleSystem(N, rho, n2, minnesota_params(), theta=th)
        nv, eps, nh = g.basis(s)
        assert nh == N
        assert np.array_equal(nv.astype(np.int32), o.states())
        _, eps_o = o.energies()
        assert np.max(np.abs(eps - eps_o)) <= 1e-12 * np.max(np.abs(eps_o))
        keys, sizes, pairs = g.channels(s, kind=0)
        t = o.channel_tables()
        nhh = int(t["nhh"].sum())
        assert np.array_equal(keys, t["keys"]) and np.array_equal(sizes[:, 0], t["nhh"])
        assert np.array_equal(pairs[:nhh], t["hh"]) and np.array_equal(pairs[nhh:], t["pp"])
        keys, sizes, pairs = g.channels(s, kind=1)
        x = o.cross_tables()
        n1 = int(x["nph"].sum())
        assert np.array_equal(keys, x["keys"]) and np.array_equal(sizes[:, 0], x["nph"])
        assert np.array_equal(sizes[:, 1], x["nhp"])
        assert np.array_equal(pairs[:n1], x["ph"]) and np.array_equal(pairs[n1:], x["hp"])
        assert math.isclose(g.eref()[s], o.eref(), rel_tol=1e-12)
        assert math.isclose(g.mbpt2()[s], o.mbpt2(), rel_tol=1e-11)
    g.close()


def test_twisted_ccd_fp64_history_and_amplitudes(pkg):
    N, rho, n2 = 14, 0.08, 20
    th = TWISTS[1]
    g = pkg.Context(N, rho, n2, params=minnesota_params(), theta=th)
    o = channel.OracleSystem(N, rho, n2, minnesota_params(), theta=th)
    dE_o, it_o, h_o, _ = o.ccd(alpha=0.5, tol=1e-10, maxit=300)
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    assert it[0] == it_o
    assert np.max(np.abs(g.history() - h_o) / np.abs(h_o)) < 1e-10
    t_o = o.t_gather(g.amplitude_labels())
    assert np.max(np.abs(g.get_amplitudes() - t_o)) <= 1e-10 * np.max(np.abs(t_o))
    g.close()


def test_twisted_two_neutrons_exact(pkg):
    th = (3.8, 0.2, 0.1)
    g = pkg.Context(2, 0.08, 9, params=minnesota_params(), theta=th)
    o = channel.OracleSystem(2, 0.08, 9, minnesota_params(), theta=th)
    ekin, _ = o.energies()
    E0, Eref, _ = exact2.ground_state(o.states(), ekin, o.v, (0, 1))
    dE, _, _, _ = g.solve(alpha=0.5, tol=1e-13, max_iter=500)
    assert abs(dE[0] - (E0 - Eref)) < 1e-10 * abs(E0)
    g.close()


def test_degenerate_twist_rejected(pkg):
    """Twists whose Fermi level is degenerate for N = 14 (the oracle rejects them too)."""
    nodes = pkg.twist_mesh(5, 1, 1)[0][:, 0]
    for bad in [(nodes[0], nodes[0], nodes[2]), (1.0, 1.0, 2.2), (0.5, 0.5, 2.0)]:
        with pytest.raises(ValueError):
            channel.OracleSystem(14, 0.08, 20, minnesota_params(), theta=bad)
        with pytest.raises(pkg.PnmError) as e:
            pkg.Context([14, 14], 0.08, 20, params=minnesota_params(), theta=[TWISTS[0], bad])
        assert e.value.code == -1 and "system 1" in str(e.value)


@pytest.fixture(scope="module")
def tabc(pkg):
    """Twist-averaged N=14, n^2<=20, rho=0.08 on a 2x3x4 Gauss-Legendre mesh (24 systems)."""
    th, w = pkg.twist_mesh(2, 3, 4)
    g = pkg.Context(14, 0.08, 20, params=minnesota_params(), theta=th)
    orc = []
    for t in th:
        o = channel.OracleSystem(14, 0.08, 20, minnesota_params(), theta=t)
        orc.append((o.eref(), o.ccd(alpha=0.5, tol=1e-10, maxit=300)))
    yield pkg, g, th, w, orc
    g.close()


def test_twist_average_fp64_matches_oracle(tabc):
    P, g, th, w, orc = tabc
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    for s, (eref_o, (dE_o, it_o, _, _)) in enumerate(orc):
        assert it[s] == it_o
        assert abs(dE[s] - dE_o) <= 1e-10 * abs(dE_o)
    ta = np.sum(w * (g.eref() + dE)) / 14
    ta_o = sum(wi * (e + r[0]) for wi, (e, r) in zip(w, orc)) / 14
    assert abs(ta - ta_o) <= 1e-10 * abs(ta_o)


def test_twist_average_mixed_within_1e6(tabc):
    """BF16x3 ladders + 2 FP64 sweeps, stopped by |dE change|/N < 1e-6 MeV: each twist and
    the average within 1e-6 MeV per neutron of the oracle's converged energies."""
    P, g, th, w, orc = tabc
    dE, it, _, _ = g.solve(precision=P.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-6,
                           max_iter=300, refine_sweeps=2)
    err = [(dE[s] - r[0]) / 14 for s, (_, r) in enumerate(orc)]
    assert max(abs(e) for e in err) < 1e-6, err
    assert abs(np.sum(w * np.array(err))) < 1e-6
