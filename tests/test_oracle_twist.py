"""The oracle under twisted boundary conditions (Sec. "Twist-averaged boundary conditions":
k = (2 pi n + theta)/L, states ordered by energy and the lowest N filled, E averaged over a
Gauss-Legendre twist mesh with weight w_x w_y w_z / pi^3).

Pins that do not come from the oracle itself:
  - theta = 0 is the periodic system, state by state;
  - a twist that keeps the set of occupied momenta leaves every energy denominator unchanged
    (the twist enters eps_i + eps_j - eps_a - eps_b only through k_i + k_j - k_a - k_b = 0), so
    MBPT2 and CCD are those of the periodic system and E_ref moves by the closed form
    hbar^2/2m (2 pi / L)^2 N |theta / 2 pi|^2 (the occupied n sum to zero);
  - reflecting one axis (theta_x -> -theta_x) or swapping two axes maps the system onto itself;
  - two neutrons: CCD equals exact diagonalisation in the two-body sector of the occupied
    pair, also when the twist moves that pair away from n = 0;
  - the dense engine (numpy, Eq. ccd3 term by term) agrees with the channel engine;
  - twist averaging brings T/N and the HF potential energy per particle close to their
    infinite-matter values, T_inf = 3/5 hbar^2 k_F^2 / 2m and the two-Fermi-sphere integral
    of the paper, with much less spread over N than periodic boundaries (Figs. 3 and 4).
"""
import itertools
import math

import numpy as np
import pytest
from scipy.integrate import quad

from conftest import minnesota_params
from oracle import channel, dense, exact2, pw


def _mesh(ns):
    """Product Gauss-Legendre mesh on [0, pi]^3 (numpy's leggauss per axis)."""
    axes = []
    for n in ns:
        x, w = np.polynomial.legendre.leggauss(n)
        axes.append(((x + 1) * math.pi / 2, w * math.pi / 2))
    pts = []
    for idx in itertools.product(*[range(n) for n in ns]):
        th = tuple(axes[a][0][i] for a, i in enumerate(idx))
        w = np.prod([axes[a][1][i] for a, i in enumerate(idx)]) / math.pi ** 3
        pts.append((th, w))
    return pts


def test_zero_twist_is_periodic():
    P = minnesota_params()
    a = channel.OracleSystem(14, 0.08, 20, P)
    b = channel.OracleSystem(14, 0.08, 20, P, theta=(0.0, 0.0, 0.0))
    assert np.array_equal(a.states(), b.states())
    assert np.array_equal(a.energies()[1], b.energies()[1])
    ta, tb = a.channel_tables(), b.channel_tables()
    assert all(np.array_equal(ta[k], tb[k]) for k in ta)
    assert np.array_equal(pw.basis(20), pw.basis(20, (0.0, 0.0, 0.0)))


def test_twist_keeping_the_fermi_sea_moves_only_the_kinetic_energy():
    P = minnesota_params()
    N, rho, n2 = 14, 0.08, 20
    theta = (0.3, 0.7, 1.1)
    a = channel.OracleSystem(N, rho, n2, P)
    b = channel.OracleSystem(N, rho, n2, P, theta=theta)
    occ = lambda o: sorted(map(tuple, o.states()[:N].tolist()))
    assert occ(a) == occ(b)
    phi2 = sum((t / (2 * math.pi)) ** 2 for t in theta)
    shift = P[6] * (2 * math.pi / a.L) ** 2 * N * phi2
    assert math.isclose(b.eref() - a.eref(), shift, rel_tol=1e-10)
    assert math.isclose(b.mbpt2(), a.mbpt2(), rel_tol=1e-12)
    ea = a.ccd(alpha=0.5, tol=1e-10, maxit=300)[0]
    eb = b.ccd(alpha=0.5, tol=1e-10, maxit=300)[0]
    assert math.isclose(ea, eb, rel_tol=1e-11)


def test_reflection_and_axis_swap_symmetry():
    P = minnesota_params()
    N, rho, n2 = 14, 0.08, 20
    base = (0.4, 1.3, 2.6)
    ref = channel.OracleSystem(N, rho, n2, P, theta=base)
    per = channel.OracleSystem(N, rho, n2, P)
    assert abs(ref.mbpt2() - per.mbpt2()) > 1e-3 * abs(per.mbpt2())   # the Fermi sea moved
    e0 = (ref.eref(), ref.mbpt2(), ref.ccd(alpha=0.5, tol=1e-11, maxit=300)[0])
    for th in [(-0.4, 1.3, 2.6), (0.4, -1.3, 2.6), (1.3, 0.4, 2.6), (2.6, 1.3, 0.4)]:
        o = channel.OracleSystem(N, rho, n2, P, theta=th)
        e = (o.eref(), o.mbpt2(), o.ccd(alpha=0.5, tol=1e-11, maxit=300)[0])
        for x, y in zip(e, e0):
            assert math.isclose(x, y, rel_tol=1e-10), (th, e, e0)


def test_dense_engine_agrees_at_a_twist():
    P = minnesota_params()
    N, rho, n2 = 14, 0.08, 4
    theta = (2.9, 0.5, 1.7)
    st = pw.basis(n2, theta)
    L = pw.box_length(N, rho)
    D = dense.DenseCCD(pw.kinetic(st, L, P[6], theta), pw.v_dense(st, L, P), N)
    S = channel.OracleSystem(N, rho, n2, P, theta=theta)
    assert np.array_equal(S.states(), st.astype(np.int32))
    assert math.isclose(D.eref, S.eref(), rel_tol=1e-13)
    _, it1, h1, _ = D.solve(alpha=0.5, tol=1e-10, maxit=300)
    _, it2, h2, _ = S.ccd(alpha=0.5, tol=1e-10, maxit=300)
    assert it1 == it2
    assert np.max(np.abs(h1 - h2) / np.abs(h2)) < 1e-12


@pytest.mark.parametrize("theta", [(0.9, 0.2, 0.5), (3.8, 0.2, 0.1)])
def test_two_neutrons_twisted_is_exact(theta):
    P = minnesota_params()
    S = channel.OracleSystem(2, 0.08, 9, P, theta=theta)
    st = S.states()
    assert np.array_equal(st[0, :3], st[1, :3])
    ekin, _ = S.energies()
    E0, Eref, _ = exact2.ground_state(st, ekin, S.v, (0, 1))
    assert math.isclose(Eref, S.eref(), rel_tol=1e-13)
    dE, it, _, _ = S.ccd(alpha=0.5, tol=1e-13, maxit=500)
    assert it < 500
    assert abs(dE - (E0 - Eref)) < 1e-10 * abs(E0)
    if theta[0] > math.pi:
        assert st[0, 0] == -1                      # the pair sits at n = (-1, 0, 0)


def test_degenerate_fermi_level_is_rejected():
    P = minnesota_params()
    x, _ = np.polynomial.legendre.leggauss(5)
    th = (x + 1) * math.pi / 2
    with pytest.raises(ValueError):
        channel.OracleSystem(14, 0.08, 20, P, theta=(th[0], th[0], th[2]))


def _hf_inf(rho, P):
    """HF potential energy per particle of infinite neutron matter: the paper's integral over
    two Fermi spheres of <k1 k2|v|k1 k2>, reduced to one dimension with the overlap volume of
    two spheres of radius k_F at distance q, pi/12 (4 k_F + q)(2 k_F - q)^2."""
    VR, kR, _, _, VS, kS, _ = P
    W = lambda q: (VR * (math.pi / kR) ** 1.5 * math.exp(-q * q / (4 * kR))
                   + VS * (math.pi / kS) ** 1.5 * math.exp(-q * q / (4 * kS)))
    kF = (3 * math.pi ** 2 * rho) ** (1 / 3)
    vol = 4 * math.pi * kF ** 3 / 3
    direct = W(0.0) * vol ** 2
    exch = quad(lambda q: 4 * math.pi * q * q * W(q) * math.pi / 12 * (4 * kF + q) * (2 * kF - q) ** 2,
                0.0, 2 * kF)[0]
    return (direct + exch) / (2 * rho * (2 * math.pi) ** 6)


def test_twist_average_reduces_finite_size_effects():
    P = minnesota_params()
    rho = 0.08
    kF = (3 * math.pi ** 2 * rho) ** (1 / 3)
    t_inf = 0.6 * P[6] * kF ** 2
    hf_inf = _hf_inf(rho, P)
    mesh = _mesh((4, 5, 6))
    tp, ta, hp, ha = {}, {}, {}, {}
    for N, n2 in ((14, 4), (38, 9), (54, 9), (66, 9), (114, 12)):
        o = channel.OracleSystem(N, rho, n2, P)
        tp[N] = o.energies()[0][:N].sum() / N
        hp[N] = o.eref() / N - tp[N]
        t_acc = h_acc = 0.0
        for th, w in mesh:
            o = channel.OracleSystem(N, rho, n2, P, theta=th)
            t = o.energies()[0][:N].sum() / N
            t_acc += w * t
            h_acc += w * (o.eref() / N - t)
        ta[N], ha[N] = t_acc, h_acc
    spread = lambda d: max(d.values()) - min(d.values())
    assert all(abs(ta[N] / t_inf - 1) < 0.012 for N in ta), (ta, t_inf)
    assert spread(ta) < 0.25 * spread(tp)
    big = [38, 54, 66, 114]
    assert all(abs(ha[N] / hf_inf - 1) < 0.006 for N in big), (ha, hf_inf)
    assert spread({N: ha[N] for N in big}) < 0.5 * spread({N: hp[N] for N in big})
