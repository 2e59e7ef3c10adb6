"""Independent numpy restatement of the plane-wave basis and the antisymmetrized
Minnesota elements for two neutrons (arXiv:1611.06765, Sec. "Single-particle basis for
infinite matter", Sec. "Two-body interaction", Table tab:minnesotatab).

TEST INFRASTRUCTURE ONLY.  Written separately from ``pnm_oracle.c`` so the two can be
compared with each other.  Here the spin algebra is done by hand instead of with
operator matrices: for two neutrons (P_tau = 1) the exchange form
V = 1/2 (V_R + 1/2(1+P_s) V_T + 1/2(1-P_s) V_S)(1 - P_s) reduces, with P_s^2 = 1, to
1/2 (V_R + V_S)(1 - P_s); its antisymmetrized momentum-space element is
<pq|v|rs> = 1/2 [Vt(k_p-k_r) + Vt(k_p-k_s)] (d(s_p,s_r) d(s_q,s_s) - d(s_p,s_s) d(s_q,s_r))
times momentum conservation, with Vt(q) = sum_{a=R,S} (V_a/L^3)(pi/kappa_a)^{3/2} exp(-q^2/4kappa_a).
"""
import math

import numpy as np


def basis(n2max, theta=None, species="n"):
    """States (nx, ny, nz, s) in the shell-ordered loop order, s in units of hbar/2.  With
    protons (species "p" or "np") a fifth column t (+1 neutron, -1 proton) follows, and per
    momentum and spin the protons come before the neutrons.

    With twist angles theta (Sec. "Twist-averaged boundary conditions", k = (2 pi n +
    theta)/L) the same states are reordered by |n + theta/2pi|^2, equal values keeping the
    shell order, so that the lowest N are the holes."""
    r = math.isqrt(n2max)
    ts = {"n": (1,), "p": (-1,), "np": (-1, 1)}[species]
    out = []
    for shell in range(n2max + 1):
        for x in range(-r, r + 1):
            for y in range(-r, r + 1):
                for z in range(-r, r + 1):
                    if x * x + y * y + z * z != shell:
                        continue
                    for s in (-1, 1):
                        for t in ts:
                            out.append((x, y, z, s) if species == "n" else (x, y, z, s, t))
    st = np.array(out, dtype=np.int64)
    if theta is not None:
        st = st[np.argsort(twisted_n2(st, theta), kind="stable")]
    return st


def twisted_n2(states, theta):
    """|n + theta/2pi|^2 per state, the axis terms added smallest first."""
    if theta is None:
        theta = (0.0, 0.0, 0.0)
    phi = np.asarray(theta, float) / (2 * math.pi)
    terms = np.sort((states[:, :3] + phi[None, :]) ** 2, axis=1)
    return (terms[:, 0] + terms[:, 1]) + terms[:, 2]


def box_length(N, rho):
    """L^3 = N / rho."""
    return (N / rho) ** (1.0 / 3.0)


def vtilde(q2, L, params):
    """Sum of the R and S Gaussians in momentum space (the T term cancels for nn)."""
    VR, kR, _VT, _kT, VS, kS, _h = params
    L3 = L ** 3
    return (VR / L3 * (math.pi / kR) ** 1.5 * np.exp(-q2 / (4 * kR))
            + VS / L3 * (math.pi / kS) ** 1.5 * np.exp(-q2 / (4 * kS)))


def v_dense(states, L, params):
    """Full antisymmetrized <pq|v|rs> as an (n, n, n, n) array."""
    n = len(states)
    k = states[:, :3].astype(float) * (2 * math.pi / L)
    s = states[:, 3]
    P = states[:, None, :3] + states[None, :, :3]                       # (p, q)
    cons = np.all(P[:, :, None, None, :] == P[None, None, :, :, :], axis=-1)
    dk_pr = k[:, None, :] - k[None, :, :]                              # k_p - k_r
    q2 = np.sum(dk_pr ** 2, axis=-1)
    Vt = vtilde(q2, L, params)                                          # (p, r)
    sp = s[:, None] == s[None, :]                                       # d(s_p, s_r)
    direct = Vt[:, None, :, None]                                       # Vt(k_p-k_r): (p,_,r,_)
    exch = Vt[:, None, None, :]                                         # Vt(k_p-k_s): (p,_,_,s)
    spin = (sp[:, None, :, None] & sp[None, :, None, :]).astype(float) - \
           (sp[:, None, None, :] & sp[None, :, :, None]).astype(float)
    v = 0.5 * (direct + exch) * spin * cons
    assert v.shape == (n, n, n, n)
    return v


def v_dense_nucleons(states, L, params):
    """Full antisymmetrized <pq|v|rs> for nucleon states (columns nx, ny, nz, s, t), written
    out by hand from V = 1/2 (V_R + 1/2(1+P_s) V_T + 1/2(1-P_s) V_S)(1 - P_s P_t) with P_s^2 =
    P_t^2 = 1:
        O_R = 1/2 (1 - P_s P_t)
        O_T = 1/4 (1 + P_s - P_t - P_s P_t)
        O_S = 1/4 (1 - P_s + P_t - P_s P_t)
    and, in the product basis, <ab|1|cd> = d(a,c) d(b,d) over spin and isospin, P_s exchanging
    the spins of the ket (d(s_a,s_d) d(s_b,s_c) d(t_a,t_c) d(t_b,t_d)), P_t the isospins, P_s P_t
    both.  Antisymmetrized: the direct term at k_p - k_r minus the exchange (r <-> s) at
    k_p - k_s."""
    VR, kR, VT, kT, VS, kS, _ = params
    L3 = L ** 3
    n = len(states)
    k = states[:, :3].astype(float) * (2 * math.pi / L)
    s, t = states[:, 3], states[:, 4]
    P = states[:, None, :3] + states[None, :, :3]
    cons = np.all(P[:, :, None, None, :] == P[None, None, :, :, :], axis=-1)
    q2 = np.sum((k[:, None, :] - k[None, :, :]) ** 2, axis=-1)             # |k_p - k_r|^2
    g = lambda V, kap: V / L3 * (math.pi / kap) ** 1.5 * np.exp(-q2 / (4 * kap))
    GR, GT, GS = g(VR, kR), g(VT, kT), g(VS, kS)
    ss = s[:, None] == s[None, :]
    tt = t[:, None] == t[None, :]

    # index grids p, q, r, s -> axes 0, 1, 2, 3
    sp_r = ss[:, None, :, None]; sq_s = ss[None, :, None, :]
    sp_s = ss[:, None, None, :]; sq_r = ss[None, :, :, None]
    tp_r = tt[:, None, :, None]; tq_s = tt[None, :, None, :]
    tp_s = tt[:, None, None, :]; tq_r = tt[None, :, :, None]

    def structures(spr, sqs, sps, sqr, tpr, tqs, tps, tqr):
        one = (spr & sqs & tpr & tqs).astype(float)
        Ps = (sps & sqr & tpr & tqs).astype(float)
        Pt = (spr & sqs & tps & tqr).astype(float)
        PsPt = (sps & sqr & tps & tqr).astype(float)
        return one, Ps, Pt, PsPt

    # direct <pq|O|rs> and exchange <pq|O|sr> (r and s swapped)
    d1, dPs, dPt, dPsPt = structures(sp_r, sq_s, sp_s, sq_r, tp_r, tq_s, tp_s, tq_r)
    e1, ePs, ePt, ePsPt = structures(sp_s, sq_r, sp_r, sq_s, tp_s, tq_r, tp_r, tq_s)
    oR = lambda a, b, c, d_: 0.5 * (a - d_)
    oT = lambda a, b, c, d_: 0.25 * (a + b - c - d_)
    oS = lambda a, b, c, d_: 0.25 * (a - b + c - d_)
    dirR, dirT, dirS = GR[:, None, :, None], GT[:, None, :, None], GS[:, None, :, None]
    exR, exT, exS = GR[:, None, None, :], GT[:, None, None, :], GS[:, None, None, :]
    v = (dirR * oR(d1, dPs, dPt, dPsPt) + dirT * oT(d1, dPs, dPt, dPsPt) + dirS * oS(d1, dPs, dPt, dPsPt)
         - exR * oR(e1, ePs, ePt, ePsPt) - exT * oT(e1, ePs, ePt, ePsPt) - exS * oS(e1, ePs, ePt, ePsPt))
    v = v * cons
    assert v.shape == (n, n, n, n)
    return v


def kinetic(states, L, hbar2_2m, theta=None):
    """hbar^2/2m |k|^2 with k = (2 pi n + theta)/L."""
    k0 = 2 * math.pi / L
    return hbar2_2m * k0 * k0 * twisted_n2(states, theta)
