"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer tables (basis, direct and cross channels) must be bit-exact; FP64 energies and
amplitudes agree to 1e-10 relative (the kernels differ from the oracle only in summation
order); the bound required of the FP64 GPU path is 1e-8 relative in E_corr/N.
"""
import math

import numpy as np
import pytest

from conftest import minnesota_params
from oracle import channel, exact2

pytestmark = pytest.mark.gpu

CASES = [(14, 0.08, 4), (14, 0.08, 20), (2, 0.08, 4), (66, 0.16, 36)]


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


_ctx_cache = {}
_orc_cache = {}


def ctx_of(P, N, rho, n2):
    k = (N, rho, n2)
    if k not in _ctx_cache:
        _ctx_cache[k] = P.Context(N, rho, n2, params=minnesota_params())
    return _ctx_cache[k]


def orc_of(N, rho, n2):
    k = (N, rho, n2)
    if k not in _orc_cache:
        _orc_cache[k] = channel.OracleSystem(N, rho, n2, minnesota_params())
    return _orc_cache[k]


@pytest.mark.parametrize("N,rho,n2", CASES)
def test_basis_bit_exact(pkg, N, rho, n2):
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2)
    nv, eps, nh = g.basis()
    assert nh == N
    assert np.array_equal(nv.astype(np.int32), o.states())
    _, eps_o = o.energies()
    assert np.max(np.abs(eps - eps_o)) <= 1e-12 * np.max(np.abs(eps_o))


@pytest.mark.parametrize("N,rho,n2", CASES)
def test_direct_channels_bit_exact(pkg, N, rho, n2):
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2).channel_tables()
    keys, sizes, pairs = g.channels(kind=0)
    assert np.array_equal(keys, o["keys"])
    assert np.array_equal(sizes[:, 0], o["nhh"]) and np.array_equal(sizes[:, 1], o["npp"])
    nh = int(o["nhh"].sum())
    assert np.array_equal(pairs[:nh], o["hh"]) and np.array_equal(pairs[nh:], o["pp"])


@pytest.mark.parametrize("N,rho,n2", CASES)
def test_cross_channels_bit_exact(pkg, N, rho, n2):
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2).cross_tables()
    keys, sizes, pairs = g.channels(kind=1)
    assert np.array_equal(keys, o["keys"])
    assert np.array_equal(sizes[:, 0], o["nph"]) and np.array_equal(sizes[:, 1], o["nhp"])
    n1 = int(o["nph"].sum())
    assert np.array_equal(pairs[:n1], o["ph"]) and np.array_equal(pairs[n1:], o["hp"])


def test_v_elements_sampled(pkg):
    N, rho, n2 = 14, 0.08, 20
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2)
    nv, _, _ = g.basis()
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(300):
        p, q, r = (int(x) for x in rng.integers(0, len(nv), 3))
        target = nv[p, :3].astype(int) + nv[q, :3] - nv[r, :3]
        cand = np.where(np.all(nv[:, :3] == target, axis=1))[0]
        for s in cand[:2]:
            a, b = g.v(p, q, r, int(s)), o.v(p, q, r, int(s))
            assert abs(a - b) <= 1e-13 * max(1.0, abs(b))
            checked += 1
    assert checked > 100


@pytest.mark.parametrize("N,rho,n2", CASES)
def test_eref_and_mbpt2(pkg, N, rho, n2):
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2)
    assert math.isclose(g.eref()[0], o.eref(), rel_tol=1e-12)
    assert math.isclose(g.mbpt2()[0], o.mbpt2(), rel_tol=1e-11)


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 4), (14, 0.08, 20)])
def test_ccd_fp64_history_and_amplitudes(pkg, N, rho, n2):
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2)
    dE_o, it_o, h_o, _ = o.ccd(alpha=0.5, tol=1e-10, maxit=300)
    dE, it, res, rc = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    h = g.history()
    assert it[0] == it_o
    assert np.max(np.abs(h - h_o) / np.abs(h_o)) < 1e-10
    assert abs(dE[0] - dE_o) <= 1e-10 * abs(dE_o)
    labels = g.amplitude_labels()
    t = g.get_amplitudes()
    t_o = o.t_gather(labels)
    assert np.max(np.abs(t - t_o)) <= 1e-10 * np.max(np.abs(t_o))
    assert res[0] < 1e-6


def test_ccd_fp64_large_case(pkg):
    """N = 66, n^2 <= 36, rho = 0.16: E_corr/N within 1e-8 relative of the oracle."""
    N, rho, n2 = 66, 0.16, 36
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2)
    dE_o, it_o, h_o, _ = o.ccd(alpha=0.5, tol=1e-10, maxit=300)
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    assert it[0] == it_o
    assert abs(dE[0] - dE_o) <= 1e-8 * abs(dE_o)
    h = g.history()
    assert np.max(np.abs(h - h_o) / np.abs(h_o)) < 1e-10


def test_first_update_from_zero_is_mbpt2(pkg):
    g = ctx_of(pkg, 14, 0.08, 20)
    _, it, _, rc = g.solve(alpha=1.0, tol=1e-30, max_iter=1, init=pkg.PNM_INIT_ZERO,
                           allow=(pkg.PNM_ENOTCONV,))
    assert rc == pkg.PNM_ENOTCONV and it[0] == 1
    h = g.history()
    assert h[0] == 0.0
    assert math.isclose(h[1], g.mbpt2()[0], rel_tol=1e-12)


def test_two_neutrons_exact(pkg):
    N, rho, n2 = 2, 0.08, 4
    g = ctx_of(pkg, N, rho, n2)
    o = orc_of(N, rho, n2)
    ekin, _ = o.energies()
    E0, Eref, _ = exact2.ground_state(o.states(), ekin, o.v, (0, 1))
    dE, _, _, _ = g.solve(alpha=0.5, tol=1e-13, max_iter=500)
    assert abs(dE[0] - (E0 - Eref)) < 1e-10 * abs(E0)


def test_host_loop_matches_graph_loop(pkg):
    g = ctx_of(pkg, 14, 0.08, 20)
    a = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    ha = g.history()
    b = g.solve(alpha=0.5, tol=1e-10, max_iter=300, host_loop=True)
    hb = g.history()
    assert a[1][0] == b[1][0]
    assert np.array_equal(ha, hb)


def test_keep_start_resumes(pkg):
    """set/get amplitudes round trip; a converged start stops after one update."""
    g = ctx_of(pkg, 14, 0.08, 4)
    g.solve(alpha=0.5, tol=1e-12, max_iter=300)
    t = g.get_amplitudes()
    g.set_amplitudes(t)
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=300, init=pkg.PNM_INIT_KEEP)
    assert it[0] == 1


def test_iteration_cap_reports_notconv(pkg):
    g = ctx_of(pkg, 14, 0.08, 4)
    _, it, _, rc = g.solve(alpha=0.5, tol=1e-14, max_iter=3, allow=(pkg.PNM_ENOTCONV,))
    assert rc == pkg.PNM_ENOTCONV and it[0] == 3


def test_open_shell_rejected(pkg):
    with pytest.raises(pkg.PnmError) as e:
        pkg.Context(10, 0.08, 4, params=minnesota_params())
    assert e.value.code == -1
    with pytest.raises(pkg.PnmError):
        pkg.Context(14, 0.08, 1, params=minnesota_params())


def test_batch_matches_single_systems(pkg):
    """Densities of one batch converge after different numbers of updates; a converged one is
    frozen and its work skipped while the others go on.  Each must still follow the oracle's
    own iteration: same count, history, energy and final amplitudes."""
    rhos = [0.04, 0.08, 0.12]
    g = pkg.Context(14, rhos, 20, params=minnesota_params())
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    assert len(set(int(x) for x in it)) > 1
    for k, rho in enumerate(rhos):
        o = orc_of(14, rho, 20)
        dE_o, it_o, h_o, _ = o.ccd(alpha=0.5, tol=1e-10, maxit=300)
        assert it[k] == it_o
        assert abs(dE[k] - dE_o) <= 1e-10 * abs(dE_o)
        assert np.max(np.abs(g.history(k) - h_o) / np.abs(h_o)) < 1e-10
        t_o = o.t_gather(g.amplitude_labels(k))
        assert np.max(np.abs(g.get_amplitudes(k) - t_o)) <= 1e-10 * np.max(np.abs(t_o))
    g.close()
