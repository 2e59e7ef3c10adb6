"""The simple pairing model of arXiv:1611.06765 (Eqs. sppairing and intpairing, Table
tab:pairingmodelsp): p levels with spin degeneracy two, H0 = delta sum (p-1) n_p and
V = -g/2 sum_pq P_p^+ P_q^-.

TEST INFRASTRUCTURE ONLY.  Provides h0 and the antisymmetrized v for the dense CCD
engine, and a Fock-space full configuration interaction in the space of unbroken pairs.
"""
import itertools

import numpy as np


def states(nlevels=4):
    """Single-particle states in the order of Table tab:pairingmodelsp: level p = 1..,
    2s_z = +1 then -1."""
    return [(p, s) for p in range(1, nlevels + 1) for s in (1, -1)]


def hamiltonian(g, delta=1.0, nlevels=4):
    """h0 (diagonal) and antisymmetrized <pq|v|rs> for the pairing Hamiltonian.

    V = -g/2 sum_{pq} a+_{p+} a+_{p-} a_{q-} a_{q+}.  Its only nonzero antisymmetrized
    elements connect a pair (p+, p-) to a pair (q+, q-):
    <p+ p-|v|q+ q-> = -g/2, with signs from exchanging the two states in bra or ket.
    """
    sp = states(nlevels)
    n = len(sp)
    h0 = np.array([delta * (p - 1) for p, _ in sp], float)
    v = np.zeros((n, n, n, n))
    idx = {st: k for k, st in enumerate(sp)}
    for p in range(1, nlevels + 1):
        for q in range(1, nlevels + 1):
            a, b = idx[(p, 1)], idx[(p, -1)]
            c, d = idx[(q, 1)], idx[(q, -1)]
            val = -0.5 * g
            v[a, b, c, d] = val
            v[b, a, c, d] = -val
            v[a, b, d, c] = -val
            v[b, a, d, c] = val
    return h0, v


def fci_ground(g, delta=1.0, nlevels=4, npairs=2):
    """Lowest eigenvalue of H in the space of unbroken pairs, built directly in second
    quantization (pair occupations), independent of the CCD machinery."""
    confs = list(itertools.combinations(range(1, nlevels + 1), npairs))
    dim = len(confs)
    H = np.zeros((dim, dim))
    for x, cx in enumerate(confs):
        H[x, x] = sum(2 * delta * (p - 1) for p in cx) - 0.5 * g * npairs
        for y, cy in enumerate(confs):
            if x != y and len(set(cx) ^ set(cy)) == 2:
                H[x, y] = -0.5 * g
    return float(np.linalg.eigvalsh(H)[0]), H
