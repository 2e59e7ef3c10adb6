"""Global spin-flip symmetry of the oracle (the property the GPU ph term relies on).

F (every state to the one of opposite spin, momentum and species kept) commutes with the
kinetic energy and with the Minnesota interaction (its spin dependence is through the spin
exchange operator only) and maps the spin-saturated reference onto itself.  Checked on the
oracle, independently of the CUDA path:
  - F is an involution on the amplitude labels and maps every direct channel (P, S_z) onto
    (P, -S_z) with the same sizes;
  - the converged CCD amplitudes are flip-symmetric, for neutron matter, a twisted box and
    symmetric nuclear matter;
  - the ph term commutes with F on random (non-symmetric) amplitudes, so the ph term of a
    flip-symmetric t, such as (t + F t)/2, is flip-symmetric.
"""
import numpy as np
import pytest

from conftest import minnesota_params
from inputs import random_amplitudes
from oracle import channel
import spinflip


def _system(N, rho, n2, theta=None, Z=0):
    o = channel.OracleSystem(N, rho, n2, minnesota_params(), theta=theta, Z=Z)
    lab = spinflip.labels_from_tables(o.channel_tables())
    return o, lab, spinflip.flip_permutation(lab, o.states())


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 4), (14, 0.08, 9)])
def test_flip_is_an_involution_on_channels(N, rho, n2):
    o, lab, (idx, sgn) = _system(N, rho, n2)
    assert np.array_equal(idx[idx], np.arange(len(idx)))
    assert np.array_equal(sgn * sgn[idx], np.ones(len(idx)))
    tab = o.channel_tables()
    st = o.states()
    # channel of each amplitude: (P, S_z) of its (a, b) pair
    P = st[lab[:, 0], :3] + st[lab[:, 1], :3]
    Sz = st[lab[:, 0], 3] + st[lab[:, 1], 3]
    assert np.array_equal(P[idx], P) and np.array_equal(Sz[idx], -Sz)
    assert int(np.sum(Sz > 0)) == int(np.sum(Sz < 0)) > 0
    assert len(lab) == int(np.sum(tab["nhh"] * tab["npp"]))


@pytest.mark.parametrize("kw", [dict(N=14, rho=0.08, n2=9), dict(N=14, rho=0.08, n2=9, theta=(0.4, 1.3, 2.6)),
                                dict(N=2, rho=0.16, n2=4, Z=2)])
def test_converged_amplitudes_are_flip_symmetric(kw):
    o, lab, perm = _system(**kw)
    o.ccd(alpha=0.5, tol=1e-12, maxit=400)
    t = o.t_gather(lab)
    scale = np.max(np.abs(t))
    assert scale > 0
    assert np.max(np.abs(t - spinflip.flip(t, perm))) <= 1e-12 * scale


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 4), (14, 0.08, 9)])
def test_ph_term_commutes_with_flip(N, rho, n2):
    o, lab, perm = _system(N, rho, n2)
    t = random_amplitudes(len(lab), seed=21)
    asym = t - spinflip.flip(t, perm)
    assert np.max(np.abs(asym)) > 0.1 * np.max(np.abs(t))  # a non-symmetric input
    r = o.ph_apply(t)
    rf = o.ph_apply(spinflip.flip(t, perm))
    scale = np.max(np.abs(r))
    assert np.max(np.abs(rf - spinflip.flip(r, perm))) <= 1e-12 * scale
    rs = o.ph_apply(spinflip.symmetrise(t, perm))
    assert np.max(np.abs(rs - spinflip.flip(rs, perm))) <= 1e-12 * scale
