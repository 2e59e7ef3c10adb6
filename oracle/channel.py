"""ctypes front end of the C oracle (``pnm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  See ``pnm_oracle.c`` for the passages of arXiv:1611.06765
that each routine follows.
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        L.om_create.restype = vp
        L.om_create.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.om_create_matter.restype = vp
        L.om_create_matter.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.om_isospin.argtypes = [vp, vp]
        L.om_create_twisted.restype = vp
        L.om_create_twisted.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.om_destroy.argtypes = [vp]
        for name in ("om_nsp", "om_nchan", "om_nxchan"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [vp]
        L.om_nt.restype = C.c_size_t
        L.om_nt.argtypes = [vp]
        L.om_L.restype = C.c_double
        L.om_L.argtypes = [vp]
        L.om_states.argtypes = [vp, vp]
        L.om_energies.argtypes = [vp, vp, vp]
        L.om_channel_tables.argtypes = [vp] * 6
        L.om_cross_tables.argtypes = [vp] * 6
        L.om_v.restype = C.c_double
        L.om_v.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.om_eref.restype = C.c_double
        L.om_eref.argtypes = [vp]
        L.om_mbpt2.restype = C.c_double
        L.om_mbpt2.argtypes = [vp]
        L.om_ccd.restype = C.c_int
        L.om_ccd.argtypes = [vp, C.c_double, C.c_double, C.c_int, C.c_int, vp, vp, vp]
        L.om_ccd_terms.restype = C.c_int
        L.om_ccd_terms.argtypes = [vp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, vp, vp, vp]
        L.om_mbpt3.restype = C.c_int
        L.om_mbpt3.argtypes = [vp, vp]
        L.om_t_get.restype = C.c_double
        L.om_t_get.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.om_t_gather.argtypes = [vp, C.c_long, vp, vp]
        L.om_t_dump.argtypes = [vp, vp, vp]
        L.om_vpp_block.restype = C.c_long
        L.om_vpp_block.argtypes = [vp, C.c_int, vp]
        L.om_ph_apply.restype = C.c_int
        L.om_ph_apply.argtypes = [vp, vp, vp, C.c_int]
        L.om_threads.restype = C.c_int
        L.om_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


class OracleSystem:
    """One (N, rho, n2max) pure-neutron-matter system in the C oracle."""

    def __init__(self, N, rho, n2max, params, theta=None, Z=0):
        """N neutrons and Z protons (Z = 0: pure neutron matter; N = Z: symmetric nuclear
        matter; N = 0: pure proton matter) at total density rho.  params: (V_R, kappa_R, V_T,
        kappa_T, V_S, kappa_S, hbar^2/2m); theta: twist angles (radians, one per axis) or None
        for periodic boundary conditions."""
        L = lib()
        p = (C.c_double * 7)(*[float(x) for x in params])
        err = C.c_int(0)
        th = None if theta is None else (C.c_double * 3)(*[float(x) for x in theta])
        if Z == 0 and theta is None:
            h = L.om_create(int(N), float(rho), int(n2max), p, C.byref(err))
        else:
            h = L.om_create_matter(int(N), int(Z), float(rho), int(n2max), p, th, C.byref(err))
        if not h:
            raise ValueError("oracle: invalid system (N=%d is not a closed shell of n2max=%d "
                             "at twist %s?)" % (N, n2max, theta))
        self.theta = None if theta is None else tuple(float(x) for x in theta)
        self._h = C.c_void_p(h)
        self.N, self.rho, self.n2max = int(N) + int(Z), float(rho), int(n2max)
        self.Z = int(Z)
        self.nsp = L.om_nsp(self._h)
        self.L = L.om_L(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.om_destroy(h)
            self._h = None

    # ---- basis and one-body
    def states(self):
        """(nx, ny, nz, s) per state, and a fifth column t (+1 neutron, -1 proton) when the
        system holds protons."""
        out = np.zeros((self.nsp, 4), dtype=np.int32)
        lib().om_states(self._h, _ptr(out))
        if self.Z == 0:
            return out
        t = np.zeros(self.nsp, dtype=np.int32)
        lib().om_isospin(self._h, _ptr(t))
        return np.concatenate([out, t[:, None]], axis=1)

    def energies(self):
        ekin = np.zeros(self.nsp)
        eps = np.zeros(self.nsp)
        lib().om_energies(self._h, _ptr(ekin), _ptr(eps))
        return ekin, eps

    def v(self, p, q, r, s):
        return lib().om_v(self._h, int(p), int(q), int(r), int(s))

    def eref(self):
        return lib().om_eref(self._h)

    def mbpt2(self):
        return lib().om_mbpt2(self._h)

    # ---- channel tables
    def channel_tables(self):
        L = lib()
        nch = L.om_nchan(self._h)
        keys = np.zeros(nch, np.int32)
        nhh = np.zeros(nch, np.int32)
        npp = np.zeros(nch, np.int32)
        L.om_channel_tables(self._h, _ptr(keys), _ptr(nhh), _ptr(npp), None, None)
        hh = np.zeros((int(nhh.sum()), 2), np.int32)
        pp = np.zeros((int(npp.sum()), 2), np.int32)
        L.om_channel_tables(self._h, None, None, None, _ptr(hh), _ptr(pp))
        return dict(keys=keys, nhh=nhh, npp=npp, hh=hh, pp=pp)

    def cross_tables(self):
        L = lib()
        nx = L.om_nxchan(self._h)
        keys = np.zeros(nx, np.int32)
        nph = np.zeros(nx, np.int32)
        nhp = np.zeros(nx, np.int32)
        L.om_cross_tables(self._h, _ptr(keys), _ptr(nph), _ptr(nhp), None, None)
        ph = np.zeros((int(nph.sum()), 2), np.int32)
        hp = np.zeros((int(nhp.sum()), 2), np.int32)
        L.om_cross_tables(self._h, None, None, None, _ptr(ph), _ptr(hp))
        return dict(keys=keys, nph=nph, nhp=nhp, ph=ph, hp=hp)

    # ---- CCD
    TERMS = {"full": 0, "pp": 1, "pphh": 2, "linear": 3}

    def ccd(self, alpha=0.5, tol=1e-10, maxit=200, init="mbpt2", terms="full"):
        """Returns (dE, iterations, energy history, (setup_s, iterate_s)).  terms: "full"
        (Eq. ccd3), "pp" (Eq. ccd1), "pphh" (Eq. ccd2) or "linear" (the terms of Eq. ccd3
        linear in t)."""
        hist = np.zeros(maxit + 1)
        dE = C.c_double(0.0)
        tim = np.zeros(2)
        it = lib().om_ccd_terms(self._h, float(alpha), float(tol), int(maxit),
                                0 if init == "mbpt2" else 1, self.TERMS[terms], C.byref(dE),
                                _ptr(hist), _ptr(tim))
        if it < 0:
            raise ValueError("oracle: zero energy denominator")
        return dE.value, it, hist[: it + 1].copy(), (tim[0], tim[1])

    def mbpt3(self):
        """Third-order diagrams (4) pp ladder, (5) hh ladder, (3) ph ring, from the MBPT2
        amplitudes (see om_mbpt3)."""
        out = np.zeros(3)
        if lib().om_mbpt3(self._h, _ptr(out)) != 0:
            raise ValueError("oracle: zero energy denominator")
        return out

    def amplitudes(self):
        """Restricted amplitudes (a<b, i<j) and their labels, oracle layout."""
        n = int(lib().om_nt(self._h))
        abij = np.zeros((n, 4), np.int32)
        t = np.zeros(n)
        lib().om_t_dump(self._h, _ptr(abij), _ptr(t))
        return abij, t

    def vpp_block(self, c):
        """<ab|v|cd> block of direct channel c (restricted pairs, oracle pair order)."""
        n = lib().om_vpp_block(self._h, int(c), None)
        out = np.zeros(n)
        lib().om_vpp_block(self._h, int(c), _ptr(out))
        m = int(round(np.sqrt(n)))
        return out.reshape(m, m)

    def ph_apply(self, t_lib, absval=False):
        """P(ij)P(ab) sum_kc t_ik^ac chi_kb^cj of Eq. (ccd3) for restricted amplitudes given in
        the library layout (per channel n_hh x n_pp, hh rows); result in the same layout.
        absval: the same with |t|, |v| and + signs (an error bound)."""
        tab = self.channel_tables()
        t_lib = np.asarray(t_lib, dtype=np.float64)
        t_or = np.zeros_like(t_lib)
        off = 0
        for nh, npp in zip(tab["nhh"], tab["npp"]):
            k = int(nh) * int(npp)
            t_or[off:off + k] = t_lib[off:off + k].reshape(int(nh), int(npp)).T.ravel()
            off += k
        out = np.zeros_like(t_or)
        if lib().om_ph_apply(self._h, _ptr(t_or), _ptr(out), int(bool(absval))) != 0:
            raise MemoryError("oracle: out of memory")
        res = np.zeros_like(out)
        off = 0
        for nh, npp in zip(tab["nhh"], tab["npp"]):
            k = int(nh) * int(npp)
            res[off:off + k] = out[off:off + k].reshape(int(npp), int(nh)).T.ravel()
            off += k
        return res

    def t_gather(self, abij):
        abij = np.ascontiguousarray(abij, dtype=np.int32)
        out = np.zeros(abij.shape[0])
        lib().om_t_gather(self._h, abij.shape[0], _ptr(abij), _ptr(out))
        return out


def threads():
    return lib().om_threads()


def set_threads(n):
    lib().om_set_threads(int(n))
