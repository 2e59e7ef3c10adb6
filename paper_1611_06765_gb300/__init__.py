"""GB300-native coupled-cluster doubles for pure neutron matter (arXiv:1611.06765).

``Context`` wraps one ``pnm_ctx`` of the C library: it marshals arguments to the
``pnm_*`` calls of ``include/pnmcc.h`` and returns numpy arrays.  All work happens in the
library's CUDA kernels; importing this package does not need a GPU, calling it does.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import (PNM_EDIVERGED, PNM_ENOTCONV, PNM_INIT_KEEP, PNM_INIT_MBPT2, PNM_INIT_MLP,
                   PNM_INIT_ZERO, PNM_PREC_BF16X3, PNM_PREC_F32PAIR, PNM_PREC_FP64, PNM_TERMS_FULL, PNM_TERMS_LINEAR,
                   PNM_TERMS_PP, PNM_TERMS_PPHH, PnmError)

__all__ = ["Context", "MINNESOTA", "PnmError", "PNM_PREC_FP64", "PNM_PREC_BF16X3", "PNM_PREC_F32PAIR",
           "PNM_INIT_MBPT2", "PNM_INIT_ZERO", "PNM_INIT_KEEP", "PNM_INIT_MLP", "PNM_ENOTCONV",
           "PNM_TERMS_FULL", "PNM_TERMS_PP", "PNM_TERMS_PPHH", "PNM_TERMS_LINEAR", "twist_mesh",
           "PNM_EDIVERGED", "mlp_num_params", "mlp_init", "mlp_train", "mlp_forward", "mlp_loss_grad"]

# V_R, kappa_R, V_T, kappa_T, V_S, kappa_S (Table tab:minnesotatab, attractive T and S) and
# hbar^2/2m in MeV fm^2.
MINNESOTA = (200.0, 1.487, -178.0, 0.639, -91.85, 0.465, 20.721)


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


class Context:
    """One or more (N, rho, n2max) systems built on the GPU by ``pnm_create_batch``."""

    def __init__(self, N, rho, n2max, params=MINNESOTA, stream=None, theta=None, Z=None):
        """N neutrons (per system).  theta: twist angles, shape (3,) or (n, 3) radians
        (``pnm_create_twisted``); None for periodic boundaries.  Z: protons per system
        (``pnm_create_matter``: 0, or equal to N, or with N = 0); None for neutron matter."""
        L = _lib.load()
        Ns = np.atleast_1d(np.asarray(N, dtype=np.int32))
        rhos = np.atleast_1d(np.asarray(rho, dtype=np.float64))
        n2 = np.atleast_1d(np.asarray(n2max, dtype=np.int32))
        th = None if theta is None else np.atleast_2d(np.asarray(theta, dtype=np.float64))
        Zs = None if Z is None else np.atleast_1d(np.asarray(Z, dtype=np.int32))
        n = max(len(Ns), len(rhos), len(n2), 0 if th is None else len(th), 0 if Zs is None else len(Zs))
        Ns, rhos, n2 = (np.ascontiguousarray(np.broadcast_to(a, (n,))) for a in (Ns, rhos, n2))
        self.N, self.rho, self.n2max = Ns.copy(), rhos.copy(), n2.copy()
        p = _lib.pnm_minnesota(*[float(x) for x in params])
        h = C.c_void_p()
        args = (Ns.ctypes.data_as(C.POINTER(C.c_int)), rhos.ctypes.data_as(C.POINTER(C.c_double)),
                n2.ctypes.data_as(C.POINTER(C.c_int)))
        st = C.c_void_p(stream) if stream else None
        self.Z = np.zeros(n, np.int32)
        if Zs is not None:
            Zs = np.ascontiguousarray(np.broadcast_to(Zs, (n,)))
            self.Z = Zs.copy()
            self.theta = None if th is None else np.ascontiguousarray(np.broadcast_to(th, (n, 3))).copy()
            thp = None if th is None else self.theta.ctypes.data_as(C.POINTER(C.c_double))
            _lib.check(L.pnm_create_matter(n, args[0], Zs.ctypes.data_as(C.POINTER(C.c_int)), args[1], args[2],
                                           thp, C.byref(p), st, C.byref(h)))
            self.N = self.N + self.Z
        elif th is None:
            self.theta = None
            _lib.check(L.pnm_create_batch(n, *args, C.byref(p), st, C.byref(h)))
        else:
            th = np.ascontiguousarray(np.broadcast_to(th, (n, 3)))
            self.theta = th.copy()
            _lib.check(L.pnm_create_twisted(n, *args, th.ctypes.data_as(C.POINTER(C.c_double)),
                                            C.byref(p), st, C.byref(h)))
        self._h = h
        self.nsys = n

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().pnm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ queries
    def basis(self, sys=0):
        L = _lib.load()
        nsp, nh = C.c_int(), C.c_int()
        _lib.check(L.pnm_basis(self._h, sys, C.byref(nsp), C.byref(nh), None, None))
        nv = np.zeros((nsp.value, 4), np.int8)
        eps = np.zeros(nsp.value)
        _lib.check(L.pnm_basis(self._h, sys, C.byref(nsp), C.byref(nh), _ptr(nv), _ptr(eps)))
        return nv, eps, nh.value

    def channels(self, sys=0, kind=0):
        L = _lib.load()
        nc, npairs = C.c_int(), C.c_int()
        _lib.check(L.pnm_channels(self._h, sys, kind, C.byref(nc), C.byref(npairs), None, None, None))
        keys = np.zeros(nc.value, np.int32)
        sizes = np.zeros((nc.value, 2), np.int32)
        pairs = np.zeros((npairs.value, 2), np.int32)
        _lib.check(L.pnm_channels(self._h, sys, kind, C.byref(nc), C.byref(npairs), _ptr(keys),
                                  _ptr(sizes), _ptr(pairs)))
        return keys, sizes, pairs

    def v(self, p, q, r, s, sys=0):
        out = C.c_double()
        _lib.check(_lib.load().pnm_v_element(self._h, sys, p, q, r, s, C.byref(out)))
        return out.value

    def eref(self):
        out = np.zeros(self.nsys)
        _lib.check(_lib.load().pnm_eref(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def mbpt2(self):
        out = np.zeros(self.nsys)
        _lib.check(_lib.load().pnm_mbpt2(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def ladder_sizes(self, sys=0):
        """pnm_ladder_sizes: the pp ladder's basis size per direct channel (0: no V_pppp)."""
        L = _lib.load()
        n = C.c_int()
        _lib.check(L.pnm_ladder_sizes(self._h, sys, C.byref(n), None))
        out = np.zeros(n.value, np.int32)
        _lib.check(L.pnm_ladder_sizes(self._h, sys, C.byref(n), out.ctypes.data_as(C.c_void_p)))
        return out

    def mbpt3(self):
        """pnm_mbpt3: (nsys, 3) array of diagrams (4) pp ladder, (5) hh ladder, (3) ph ring."""
        out = np.zeros(3 * self.nsys)
        _lib.check(_lib.load().pnm_mbpt3(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(self.nsys, 3)

    # -------------------------------------------------------------------- solve
    def solve(self, precision=PNM_PREC_FP64, alpha=0.5, tol=1e-10, tol_per_N=0.0, max_iter=500,
              refine_sweeps=0, init=PNM_INIT_MBPT2, host_loop=False, allow=(), terms=PNM_TERMS_FULL,
              refine_kernels=PNM_PREC_FP64):
        """pnm_ccd_solve; returns (dE[nsys], iters[nsys], resid[nsys], rc).  refine_kernels:
        PNM_PREC_FP64 or PNM_PREC_F32PAIR for the contractions of the refinement sweeps."""
        L = _lib.load()
        o = _lib.pnm_solve_opts()
        L.pnm_default_opts(C.byref(o))
        o.precision, o.mix_alpha, o.tol_dE, o.tol_dE_per_N = precision, alpha, tol, tol_per_N
        o.max_iter, o.refine_sweeps, o.init, o.host_loop = max_iter, refine_sweeps, init, int(host_loop)
        o.terms = terms
        o.refine_kernels = refine_kernels
        dE = np.zeros(self.nsys)
        it = np.zeros(self.nsys, np.int32)
        res = np.zeros(self.nsys)
        rc = L.pnm_ccd_solve(self._h, C.byref(o), dE.ctypes.data_as(C.POINTER(C.c_double)),
                             it.ctypes.data_as(C.POINTER(C.c_int)),
                             res.ctypes.data_as(C.POINTER(C.c_double)))
        _lib.check(rc, allow=allow)
        return dE, it, res, rc

    def history(self, sys=0, cap=100000):
        n = C.c_int()
        buf = np.zeros(cap)
        _lib.check(_lib.load().pnm_energy_history(self._h, sys, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                                  cap, C.byref(n)))
        return buf[: n.value].copy()

    def amplitude_labels(self, sys=0):
        L = _lib.load()
        n = C.c_size_t()
        _lib.check(L.pnm_amplitude_labels(self._h, sys, C.byref(n), None))
        out = np.zeros((n.value, 4), np.int32)
        _lib.check(L.pnm_amplitude_labels(self._h, sys, C.byref(n), _ptr(out)))
        return out

    def get_amplitudes(self, sys=0):
        n = C.c_size_t()
        _lib.check(_lib.load().pnm_amplitude_labels(self._h, sys, C.byref(n), None))
        t = np.zeros(n.value)
        _lib.check(_lib.load().pnm_get_amplitudes(self._h, sys, _ptr(t), n.value))
        return t

    def set_amplitudes(self, t, sys=0):
        t = np.ascontiguousarray(t, dtype=np.float64)
        _lib.check(_lib.load().pnm_set_amplitudes(self._h, sys, _ptr(t), t.size))

    def apply_pp_ladder(self, t, precision=PNM_PREC_FP64, sys=0):
        """pnm_apply_pp_ladder: the pp-ladder term alone applied to amplitudes t."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        r = np.zeros_like(t)
        _lib.check(_lib.load().pnm_apply_pp_ladder(self._h, sys, precision, _ptr(t), _ptr(r), t.size))
        return r

    def apply_ph_term(self, t, precision=PNM_PREC_FP64, sys=0):
        """pnm_apply_ph_term: the ph term (linear and quadratic) alone applied to amplitudes t."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        r = np.zeros_like(t)
        _lib.check(_lib.load().pnm_apply_ph_term(self._h, sys, precision, _ptr(t), _ptr(r), t.size))
        return r

    def mlp_features(self, sys=0):
        """(X[n,32], t_MBPT2[n], sigma_sys) of system sys in library order."""
        n = len(self.amplitude_labels(sys))
        X = np.zeros((n, 32), np.float32)
        tm2 = np.zeros(n)
        sig = np.zeros(1)
        _lib.check(_lib.load().pnm_mlp_features(self._h, sys, _ptr(X), _ptr(tm2), _ptr(sig)))
        return X, tm2, float(sig[0])

    def mlp_set_model(self, blob):
        blob = np.ascontiguousarray(blob, dtype=np.float32)
        _lib.check(_lib.load().pnm_mlp_set_model(self._h, blob.ctypes.data_as(C.POINTER(C.c_float))))

    def checkpoint_header(self, sys=0):
        """pnm_checkpoint_header_of: what fixes the system's amplitude layout."""
        h = _lib.pnm_checkpoint_header()
        _lib.check(_lib.load().pnm_checkpoint_header_of(self._h, sys, C.byref(h)))
        return dict(N=h.N, Z=h.Z, n2max=h.n2max, rho=h.rho, twist=tuple(h.twist), n_amplitudes=h.n_amplitudes,
                    channel_hash=h.channel_hash)

    def save_checkpoint(self, path):
        """pnm_checkpoint_save: the held amplitudes of every system with their headers."""
        _lib.check(_lib.load().pnm_checkpoint_save(self._h, str(path).encode()))

    def load_checkpoint(self, path):
        """pnm_checkpoint_load: amplitudes from a checkpoint of the same systems (resume with
        init=PNM_INIT_KEEP); PnmError if a header does not match."""
        _lib.check(_lib.load().pnm_checkpoint_load(self._h, str(path).encode()))

    def mlp_predict(self):
        """Learned start into the held amplitudes (``pnm_mlp_predict``); read with get_amplitudes."""
        _lib.check(_lib.load().pnm_mlp_predict(self._h))

    def tuning(self):
        """Autotuner choices: (k-range splits, ring stages, us per ladder launch, serial mask)."""
        a, b, us, m = C.c_int(), C.c_int(), C.c_float(), C.c_int()
        _lib.check(_lib.load().pnm_get_tuning(self._h, C.byref(a), C.byref(b), C.byref(us), C.byref(m)))
        return a.value, b.value, us.value, m.value

    def set_profiling(self, on=True):
        _lib.check(_lib.load().pnm_set_profiling(self._h, int(on)))

    def kernel_stats(self):
        """{name: (total_ms, launches)} of the last profiled host-loop solves."""
        out = {}
        k = 0
        L = _lib.load()
        while True:
            name, ms, n = C.c_char_p(), C.c_double(), C.c_int()
            if L.pnm_kernel_stats(self._h, k, C.byref(name), C.byref(ms), C.byref(n)) != 0:
                break
            if n.value:
                out[name.value.decode()] = (ms.value, n.value)
            k += 1
        return out

    def timings(self):
        ms = np.zeros(7)
        _lib.check(_lib.load().pnm_get_timings(self._h, ms.ctypes.data_as(C.POINTER(C.c_double)), 7))
        return dict(setup=ms[0], mbpt2=ms[1], solve=ms[2], mixed=ms[3], refine=ms[4], mlp_fallback=int(ms[5]),
                    prepare=ms[6])


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def twist_mesh(nx, ny=None, nz=None):
    """Product Gauss-Legendre twist mesh (``pnm_twist_mesh``): theta (M, 3), weight (M,)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    m = nx * ny * nz
    theta = np.zeros((m, 3))
    w = np.zeros(m)
    _lib.check(_lib.load().pnm_twist_mesh(nx, ny, nz, theta.ctypes.data_as(C.POINTER(C.c_double)),
                                          w.ctypes.data_as(C.POINTER(C.c_double))))
    return theta, w


def measure_fma_peak(fp64=True, stream=None):
    """Measured peak FMA rate of the current device, TFLOP/s (FP64 or FP32)."""
    out = C.c_double()
    _lib.check(_lib.load().pnm_measure_fma_peak(int(fp64), C.c_void_p(stream) if stream else None,
                                                C.byref(out)))
    return out.value


def mlp_num_params():
    n = C.c_int()
    _lib.check(_lib.load().pnm_mlp_num_params(C.byref(n)))
    return n.value


def mlp_init(seed=0):
    blob = np.zeros(mlp_num_params(), np.float32)
    _lib.check(_lib.load().pnm_mlp_init(_fptr(blob), seed))
    return blob


def mlp_train(contexts, blob, epochs=20, batch=4096, lr=1e-3, seed=0, lr_final=None):
    """pnm_mlp_train on the amplitudes held by the contexts; returns (blob, loss history).
    lr_final: the learning rate decays from lr to lr_final along a half cosine (None: constant)."""
    blob = np.ascontiguousarray(blob, dtype=np.float32).copy()
    o = _lib.pnm_mlp_opts(epochs, batch, lr, seed, lr if lr_final is None else lr_final)
    handles = (C.c_void_p * len(contexts))(*[c._h.value for c in contexts])
    hist = np.zeros(max(1, epochs), np.float32)
    nh = C.c_int()
    _lib.check(_lib.load().pnm_mlp_train(handles, len(contexts), C.byref(o), _fptr(blob), _fptr(hist),
                                         hist.size, C.byref(nh)))
    return blob, hist[: nh.value].copy()


def mlp_forward(blob, X, tensor_cores=True, fp32=False):
    """pnm_mlp_forward: the tcgen05 inference kernel (tensor_cores=True), the SIMT forward, or
    the SIMT forward without BF16 rounding (fp32=True, the debug mode)."""
    blob = np.ascontiguousarray(blob, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.zeros(X.shape[0], np.float32)
    mode = _lib.PNM_MLP_SIMT_FP32 if fp32 else (_lib.PNM_MLP_TENSOR_CORES if tensor_cores else _lib.PNM_MLP_SIMT)
    _lib.check(_lib.load().pnm_mlp_forward(_fptr(blob), _fptr(X), X.shape[0], _fptr(Y), mode, None))
    return Y


def mlp_loss_grad(blob, X, T, fp32=False, tensor_cores=True):
    """pnm_mlp_loss_grad: (mean squared error, gradient blob); fp32=True is the debug mode
    without BF16 rounding (SIMT products); in the BF16 mode tensor_cores selects the tcgen05
    products that training uses (else the SIMT ones)."""
    blob = np.ascontiguousarray(blob, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    g = np.zeros_like(blob)
    loss = C.c_float()
    _lib.check(_lib.load().pnm_mlp_loss_grad(_fptr(blob), _fptr(X), _fptr(T), X.shape[0], C.byref(loss),
                                             _fptr(g), 1 if fp32 else (0 if tensor_cores else 2), None))
    return float(loss.value), g
