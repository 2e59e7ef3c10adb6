"""Pins of the oracle's plane-wave basis against arXiv:1611.06765 Table tab:table1, the
magic numbers in the text after it, and the state count of Sec. "Developing a CCD code"."""
import math

import numpy as np
import pytest

from conftest import minnesota_params, read_golden
from oracle import channel, pw


def _golden():
    rows = read_golden("shells.txt")
    magic = [int(x) for x in next(r for r in rows if r[0] == "magic")[1:]]
    count = next(r for r in rows if r[0] == "count")
    shells = {}
    for r in rows:
        if r[0] == "shell":
            shells.setdefault(int(r[1]), set()).add(tuple(int(x) for x in r[2:5]))
    return magic, (int(count[1]), int(count[2])), shells


def test_magic_numbers_are_shell_closures():
    magic, _, _ = _golden()
    st = pw.basis(6)
    n2 = np.sum(st[:, :3] ** 2, axis=1)
    closures = [int(np.sum(n2 <= s)) for s in range(6) if np.any(n2 == s)]
    assert closures == magic


def test_state_count_610():
    _, (n2max, count), _ = _golden()
    assert len(pw.basis(n2max)) == count
    S = channel.OracleSystem(14, 0.08, n2max, minnesota_params())
    assert S.nsp == count


def test_table1_shells():
    _, _, shells = _golden()
    st = pw.basis(3)
    for sh, pts in shells.items():
        got = {tuple(int(v) for v in s[:3]) for s in st if int(np.sum(s[:3] ** 2)) == sh}
        assert got == pts


def test_c_and_numpy_basis_agree_and_order():
    S = channel.OracleSystem(14, 0.08, 20, minnesota_params())
    a = S.states()
    b = pw.basis(20)
    assert np.array_equal(a, b)
    n2 = np.sum(a[:, :3] ** 2, axis=1)
    assert np.all(np.diff(n2) >= 0)                       # shells ascending
    assert np.all(a[0::2, 3] == -1) and np.all(a[1::2, 3] == 1)   # s = -1 before +1


@pytest.mark.parametrize("N,n2max", [(14, 4), (66, 36)])
def test_kinetic_closed_form(N, n2max):
    """T = hbar^2/2m (2 pi / L)^2 sum_holes n^2 with sum n^2 = 12 (N=14) and 156 (N=66),
    counted by hand from the shells: 2*(6*1) and 2*(6*1 + 12*2 + 8*3 + 6*4)."""
    P = minnesota_params()
    rho = 0.08
    S = channel.OracleSystem(N, rho, n2max, P)
    ekin, _ = S.energies()
    L = (N / rho) ** (1 / 3)
    sum_n2 = {14: 12, 66: 156}[N]
    assert abs(S.L - L) < 1e-12 * L
    assert math.isclose(ekin[:N].sum(), P[6] * (2 * math.pi / L) ** 2 * sum_n2, rel_tol=1e-13)


def test_open_shell_rejected():
    with pytest.raises(ValueError):
        channel.OracleSystem(10, 0.08, 4, minnesota_params())
    with pytest.raises(ValueError):
        channel.OracleSystem(14, 0.08, 1, minnesota_params())   # no particle states
