"""Exact diagonalisation for two neutrons (N = 2) in a periodic plane-wave basis.

TEST INFRASTRUCTURE ONLY.  For two particles the CCD wave function exp(T2)|Phi_0> =
(1 + T2)|Phi_0> spans the whole two-body sector of the reference (singles vanish by
momentum conservation), so converged CCD equals the exact ground-state energy.  This
module diagonalises H = sum_p h0_p a+_p a_p + 1/4 sum <pq|v|rs> a+_p a+_q a_s a_r in the
sector of two-particle states |pq>, p < q, with the reference pair's total momentum and
S_z (zero for periodic boundary conditions; a twist can move the lowest pair), where
<pq|H|rs> = (h0_p + h0_q) delta_{pq,rs} + <pq|v|rs>.  The matrix elements come from the
caller (``velem(p, q, r, s)`` and the kinetic energies), so this file holds no force.
"""
import numpy as np


def sector_pairs(states, P=(0, 0, 0), Sz=0):
    """Pairs p<q with n_p + n_q = P and s_p + s_q = Sz."""
    n = len(states)
    P = np.asarray(P)
    out = []
    for p in range(n):
        for q in range(p + 1, n):
            if np.all(states[p, :3] + states[q, :3] == P) and states[p, 3] + states[q, 3] == Sz:
                out.append((p, q))
    return out


def ground_state(states, ekin, velem, ref_pair):
    """Eigenvalue of the state with the largest overlap with the reference pair.

    Returns (E0, E_ref) where E_ref = <ref|H|ref>."""
    i, j = ref_pair
    pairs = sector_pairs(states, states[i, :3] + states[j, :3], states[i, 3] + states[j, 3])
    dim = len(pairs)
    H = np.zeros((dim, dim))
    for x, (p, q) in enumerate(pairs):
        for y, (r, s) in enumerate(pairs):
            H[x, y] = velem(p, q, r, s)
        H[x, x] += ekin[p] + ekin[q]
    w, U = np.linalg.eigh(H)
    ref = pairs.index(tuple(sorted(ref_pair)))
    k = int(np.argmax(np.abs(U[ref, :])))
    return float(w[k]), float(H[ref, ref]), float(w[0])


def rs_third_order(states, ekin, eps, velem, ref_pair):
    """Rayleigh-Schroedinger perturbation theory in the same two-body sector with the
    Moller-Plesset split H = H0 + W, H0 = diag(eps_p + eps_q) (HF energies), reference |ij>:
      E^(2) = sum_k W_0k W_k0 / (E0_0 - E0_k)
      E^(3) = sum_{k,l} W_0k W_kl W_l0 / ((E0_0 - E0_k)(E0_0 - E0_l))
              - W_00 sum_k W_0k W_k0 / (E0_0 - E0_k)^2,   k, l over the other pairs.
    Returns (E^(2), E^(3))."""
    i, j = ref_pair
    pairs = sector_pairs(states, states[i, :3] + states[j, :3], states[i, 3] + states[j, 3])
    dim = len(pairs)
    H = np.zeros((dim, dim))
    for x, (p, q) in enumerate(pairs):
        for y, (r, s) in enumerate(pairs):
            H[x, y] = velem(p, q, r, s)
        H[x, x] += ekin[p] + ekin[q]
    H0 = np.array([eps[p] + eps[q] for p, q in pairs])
    W = H - np.diag(H0)
    k0 = pairs.index(tuple(sorted(ref_pair)))
    rest = [k for k in range(dim) if k != k0]
    d = H0[k0] - H0[rest]
    w = W[k0, rest]
    e2 = float(np.sum(w * w / d))
    e3 = float((w / d) @ W[np.ix_(rest, rest)] @ (w / d) - W[k0, k0] * np.sum(w * w / d ** 2))
    return e2, e3
