"""Dense CCD engine: Eq. (ccd3) of arXiv:1611.06765 ("Developing a CCD code"), every
term written as in the paper on dense 4-index arrays.

TEST INFRASTRUCTURE ONLY.

Index convention: t[a, b, i, j] = t_ij^ab (particles a, b; holes i, j) and
v[p, q, r, s] = <pq|v|rs> (antisymmetrized).  Sums run over unrestricted indices, with
the factors 1/2 and 1/4 of the paper.  Each einsum string spells the indices of the
corresponding term of Eq. (ccd); numpy's contraction-path choice is a library step.

The engine is generic: it takes a one-body diagonal h0, an antisymmetrized v and the
number of holes (the lowest states), so it runs both the pairing model and small
plane-wave systems.
"""
import numpy as np


def _es(sub, *ops):
    return np.einsum(sub, *ops, optimize=True)


def P_ab(X):
    """P(ab) = 1 - P_ab acting on X[a, b, i, j]."""
    return X - X.transpose(1, 0, 2, 3)


def P_ij(X):
    """P(ij) = 1 - P_ij acting on X[a, b, i, j]."""
    return X - X.transpose(0, 1, 3, 2)


class DenseCCD:
    def __init__(self, h0, v, nholes):
        """h0: (n,) one-body diagonal; v: (n,n,n,n) antisymmetrized; holes = [0, nholes)."""
        self.n = len(h0)
        self.nh = nholes
        o, u = slice(0, nholes), slice(nholes, self.n)
        # f_pp = h0_pp + sum_i <pi|v|pi>  (Hartree-Fock energies, Eq. pairingsp / Hnormalorder)
        self.eps = np.asarray(h0, float) + np.einsum("piqi->pq", v[:, o, :, o]).diagonal()
        self.eref = float(np.sum(h0[o]) + 0.5 * np.einsum("ijij->", v[o, o, o, o]))
        self.v_abij = v[u, u, o, o].copy()      # <ab|v|ij>
        self.v_ijab = v[o, o, u, u].copy()      # <ij|v|ab>
        self.v_abcd = v[u, u, u, u].copy()      # <ab|v|cd>
        self.v_klij = v[o, o, o, o].copy()      # <kl|v|ij>
        self.v_kbcj = v[o, u, u, o].copy()      # <kb|v|cj>
        self.v_klcd = v[o, o, u, u].copy()      # <kl|v|cd>
        e_o, e_u = self.eps[o], self.eps[u]
        # eps_ij^ab = e_i + e_j - e_a - e_b
        self.D = (e_o[None, None, :, None] + e_o[None, None, None, :]
                  - e_u[:, None, None, None] - e_u[None, :, None, None])

    def energy(self, t):
        """Eq. (ccdcorr): 1/4 sum_{ijab} <ij|v|ab> t_ij^ab."""
        return 0.25 * float(np.einsum("ijab,abij->", self.v_ijab, t))

    def mbpt2_guess(self):
        """Eq. (ccdGuess): t0 = <ab|v|ij> / eps_ij^ab."""
        return self.v_abij / self.D

    def rhs(self, t, terms="full"):
        """The bracket of Eq. (ccd3): everything except the eps_ij^ab t term.  terms: "full";
        "pp" (Eq. ccd1: v and the pp ladder); "pphh" (Eq. ccd2: and the hh ladder); "linear"
        (every term of Eq. ccd3 linear in t)."""
        v = self
        r = v.v_abij.copy()
        r += 0.5 * _es("abcd,cdij->abij", v.v_abcd, t)
        if terms == "pp":
            return r
        r += 0.5 * _es("klij,abkl->abij", v.v_klij, t)
        if terms == "pphh":
            return r
        r += P_ij(P_ab(_es("kbcj,acik->abij", v.v_kbcj, t)))
        if terms == "linear":
            return r
        r += 0.25 * _es("klcd,cdij,abkl->abij", v.v_klcd, t, t)
        r += P_ij(_es("klcd,acik,bdjl->abij", v.v_klcd, t, t))
        r -= 0.5 * P_ij(_es("klcd,dcik,ablj->abij", v.v_klcd, t, t))
        r -= 0.5 * P_ab(_es("klcd,aclk,dbij->abij", v.v_klcd, t, t))
        return r

    def step(self, t, terms="full"):
        """t^(n+1) of Eq. (ccd3) (or of its truncation), before mixing."""
        return self.rhs(t, terms) / self.D

    def mbpt3(self):
        """Eqs. (diag4), (diag5) and (diag3) written out over the dense arrays, with
        t0_ij^ab = <ij|v|ab> / eps_ij^ab.  Eq. (diag3) is read with <kb|v|cj> where the paper
        prints <bk|v|ic> (= <kb|v|ci>)."""
        t0 = self.mbpt2_guess()                              # [a, b, i, j]
        d4 = 0.125 * _es("cdij,abcd,abij->", t0, self.v_abcd, t0)
        d5 = 0.125 * _es("abkl,klij,abij->", t0, self.v_klij, t0)
        d3 = _es("abij,kbcj,acik->", t0, self.v_kbcj, t0)
        return np.array([d4, d5, d3])

    def solve(self, alpha=1.0, tol=1e-10, maxit=500, init="mbpt2", terms="full"):
        """Iterate with mixing t = alpha t_new + (1 - alpha) t_old until the energy change
        is below tol.  Returns (dE, updates, energy history, t)."""
        t = self.mbpt2_guess() if init == "mbpt2" else np.zeros_like(self.D)
        e_old = self.energy(t)
        hist = [e_old]
        it = 0
        while it < maxit:
            t = alpha * self.step(t, terms) + (1.0 - alpha) * t
            e = self.energy(t)
            it += 1
            hist.append(e)
            diff = abs(e - e_old)
            e_old = e
            if diff < tol:
                break
        return e_old, it, np.array(hist), t
