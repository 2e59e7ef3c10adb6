"""Pins of the oracle's Minnesota elements (arXiv:1611.06765 Sec. "Two-body interaction",
Table tab:minnesotatab) against a numerical Fourier transform, the symmetries the paper
states for antisymmetrized elements, and the spin/isospin algebra for two neutrons."""
import math

import numpy as np
import pytest
from scipy import integrate

from conftest import minnesota_params
from oracle import channel, pw


def _ft_numeric(V, kappa, q):
    """V int d^3r exp(-kappa r^2) exp(-i q.r), by radial quadrature."""
    if q == 0.0:
        f = lambda r: 4 * math.pi * r * r * V * math.exp(-kappa * r * r)
    else:
        f = lambda r: 4 * math.pi * r * r * V * math.exp(-kappa * r * r) * math.sin(q * r) / (q * r)
    val, _ = integrate.quad(f, 0, 40.0 / math.sqrt(kappa), limit=400, epsabs=1e-13, epsrel=1e-12)
    return val


def test_fourier_transform_of_gaussian():
    """With only V_R switched on, an opposite-spin element is
    1/2 [G(k_p - k_r) + G(k_p - k_s)] / L^3, G the transform of V_R exp(-kappa_R r^2)."""
    N, rho, n2max = 14, 0.08, 20
    params = (1.0, 1.487, 0.0, 0.639, 0.0, 0.465, 20.721)
    S = channel.OracleSystem(N, rho, n2max, params)
    st = S.states()
    L = S.L
    k = st[:, :3] * (2 * math.pi / L)
    idx = {tuple(s): n for n, s in enumerate(st.tolist())}
    checked = 0
    for (n1, n2, d) in [((0, 0, 0), (1, 0, 0), (0, 1, 0)), ((1, 0, 0), (0, 1, 0), (1, 1, 0)),
                        ((0, 0, 1), (0, 0, -1), (0, 2, 0))]:
        p = idx[n1 + (1,)]
        q = idx[n2 + (-1,)]
        r_n = tuple(np.array(n1) + np.array(d))
        s_n = tuple(np.array(n2) - np.array(d))
        if r_n + (1,) not in idx or s_n + (-1,) not in idx:
            continue
        r = idx[r_n + (1,)]
        s = idx[s_n + (-1,)]
        q1 = np.linalg.norm(k[p] - k[r])
        q2 = np.linalg.norm(k[p] - k[s])
        expect = 0.5 * (_ft_numeric(1.0, 1.487, q1) + _ft_numeric(1.0, 1.487, q2)) / L ** 3
        assert math.isclose(S.v(p, q, r, s), expect, rel_tol=1e-9)
        checked += 1
    assert checked == 3


@pytest.fixture(scope="module")
def small():
    P = minnesota_params()
    S = channel.OracleSystem(14, 0.08, 4, P)
    st = S.states()
    v = pw.v_dense(st, pw.box_length(14, 0.08), P)
    return S, st, v


def test_c_and_numpy_elements_agree(small):
    S, st, v = small
    rng = np.random.default_rng(7)
    idx = rng.integers(0, len(st), (3000, 4))
    # also include conserving tuples so nonzero elements are compared
    cons = np.argwhere(np.abs(v) > 0)[:: max(1, int(np.count_nonzero(v)) // 3000)]
    for p, q, r, s in np.concatenate([idx, cons]):
        assert abs(S.v(p, q, r, s) - v[p, q, r, s]) <= 1e-14 * max(1.0, abs(v[p, q, r, s]))


def test_antisymmetry_hermiticity_zero_repeated(small):
    _, st, v = small
    assert np.allclose(v, -v.transpose(1, 0, 2, 3), atol=0)
    assert np.allclose(v, -v.transpose(0, 1, 3, 2), atol=0)
    assert np.allclose(v, v.transpose(2, 3, 0, 1), atol=1e-15)
    n = len(st)
    for p in range(n):
        assert np.all(v[p, p] == 0) and np.all(v[:, :, p, p] == 0)


def test_momentum_and_spin_conservation(small):
    _, st, v = small
    nz = np.argwhere(v != 0)
    P1 = st[nz[:, 0], :3] + st[nz[:, 1], :3]
    P2 = st[nz[:, 2], :3] + st[nz[:, 3], :3]
    assert np.array_equal(P1, P2)
    S1 = st[nz[:, 0], 3] + st[nz[:, 1], 3]
    S2 = st[nz[:, 2], 3] + st[nz[:, 3], 3]
    assert np.array_equal(S1, S2)


def test_triplet_term_cancels_for_neutrons():
    """(1 + P_s)(1 - P_s P_t) = 0 for P_t = 1, so V_T does not enter any nn element."""
    only_T = (0.0, 1.487, -178.0, 0.639, 0.0, 0.465, 20.721)
    S = channel.OracleSystem(14, 0.08, 4, only_T)
    rng = np.random.default_rng(3)
    st = S.states()
    for _ in range(400):
        p, q, r = rng.integers(0, len(st), 3)
        target = st[p, :3] + st[q, :3] - st[r, :3]
        cand = [s for s in range(len(st)) if np.array_equal(st[s, :3], target)]
        for s in cand:
            assert S.v(p, q, r, s) == 0.0


def test_same_spin_pairs_do_not_interact(small):
    """Spin-triplet nn pairs are spatially odd; the (1 - P_s P_t) form of V makes them
    non-interacting.  So every element with s_p = s_q vanishes."""
    _, st, v = small
    same = st[:, 3][:, None] == st[:, 3][None, :]
    assert np.all(v[same] == 0)
