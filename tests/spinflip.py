"""The global spin flip F as a permutation of restricted amplitudes (test helper).

F sends every single-particle state (n, s[, t]) to (n, -s[, t]).  On amplitudes labelled
(a, b, i, j) with a < b and i < j it is a signed permutation: (F t)(a, b, i, j) =
sign * t(F a, F b, F i, F j) with the flipped pairs put back in ascending order (one sign per
swapped pair).  Index bookkeeping only: no arithmetic of the method.
"""
import numpy as np


def labels_from_tables(tab):
    """Amplitude labels (a, b, i, j) in the library layout (per channel n_hh x n_pp, hh rows)
    from an oracle channel table."""
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
    return np.array(out, dtype=np.int32).reshape(-1, 4)


def flip_states(states):
    """Index of the flipped state of every state (states: rows n_x, n_y, n_z, s[, t])."""
    key = {tuple(r): k for k, r in enumerate(np.asarray(states).tolist())}
    out = []
    for r in np.asarray(states).tolist():
        f = list(r)
        f[3] = -f[3]
        out.append(key[tuple(f)])
    return np.array(out)


def flip_permutation(labels, states):
    """(idx, sign) with (F t)[e] = sign[e] * t[idx[e]] for amplitudes t in the order of labels."""
    F = flip_states(states)
    pos = {tuple(l): e for e, l in enumerate(np.asarray(labels).tolist())}
    idx = np.zeros(len(labels), dtype=np.int64)
    sgn = np.ones(len(labels))
    for e, (a, b, i, j) in enumerate(np.asarray(labels).tolist()):
        fa, fb, fi, fj = F[a], F[b], F[i], F[j]
        s = 1.0
        if fa > fb:
            fa, fb, s = fb, fa, -s
        if fi > fj:
            fi, fj, s = fj, fi, -s
        idx[e] = pos[(fa, fb, fi, fj)]
        sgn[e] = s
    return idx, sgn


def flip(t, perm):
    idx, sgn = perm
    return sgn * np.asarray(t)[idx]


def symmetrise(t, perm):
    """(t + F t) / 2."""
    return 0.5 * (np.asarray(t) + flip(t, perm))
