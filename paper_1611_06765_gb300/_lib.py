"""ctypes binding of ``libpnmcc.so`` (C ABI in ``include/pnmcc.h``).

Argument marshalling only: every computation runs in the library's CUDA kernels.  Loading
fails loudly when the library has not been built; there is no CPU fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpnmcc.so")

PNM_OK = 0
PNM_EINVAL = -1
PNM_ENOMEM = -2
PNM_ECUDA = -3
PNM_ENOTCONV = -4
PNM_EDIVERGED = -5
PNM_ETIMEOUT = -6

PNM_PREC_FP64 = 0
PNM_PREC_BF16X3 = 2
PNM_PREC_F32PAIR = 3
PNM_INIT_MBPT2 = 0
PNM_INIT_ZERO = 1
PNM_INIT_KEEP = 2
PNM_INIT_MLP = 3

PNM_TERMS_FULL = 0
PNM_TERMS_PP = 1
PNM_TERMS_PPHH = 2
PNM_TERMS_LINEAR = 3

PNM_MLP_SIMT = 0
PNM_MLP_TENSOR_CORES = 1
PNM_MLP_SIMT_FP32 = 2

# Every symbol include/pnmcc.h declares.
EXPORTS = (
    "pnm_default_opts", "pnm_create", "pnm_create_batch", "pnm_create_twisted", "pnm_create_matter",
    "pnm_twist_mesh",
    "pnm_destroy", "pnm_num_systems",
    "pnm_basis", "pnm_channels", "pnm_v_element", "pnm_eref", "pnm_mbpt2", "pnm_mbpt2_noalloc", "pnm_mbpt3", "pnm_ladder_sizes",
    "pnm_ccd_solve",
    "pnm_energy_history", "pnm_amplitude_labels", "pnm_get_amplitudes", "pnm_set_amplitudes",
    "pnm_get_timings", "pnm_apply_pp_ladder", "pnm_apply_ph_term", "pnm_mlp_num_params", "pnm_mlp_init",
    "pnm_mlp_features", "pnm_mlp_train", "pnm_mlp_set_model", "pnm_mlp_predict", "pnm_checkpoint_header_of", "pnm_checkpoint_save", "pnm_checkpoint_load", "pnm_mlp_forward", "pnm_mlp_loss_grad", "pnm_set_profiling", "pnm_kernel_stats", "pnm_get_tuning", "pnm_selftest_timeout",
    "pnm_measure_fma_peak", "pnm_last_error",
)


class pnm_minnesota(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("VR", "kR", "VT", "kT", "VS", "kS", "hbar2_2m")]


class pnm_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("mix_alpha", C.c_double), ("tol_dE", C.c_double),
                ("tol_dE_per_N", C.c_double), ("max_iter", C.c_int), ("refine_sweeps", C.c_int),
                ("init", C.c_int), ("host_loop", C.c_int), ("terms", C.c_int), ("refine_kernels", C.c_int)]


class pnm_checkpoint_header(C.Structure):
    _fields_ = [("N", C.c_int32), ("Z", C.c_int32), ("n2max", C.c_int32), ("reserved", C.c_int32),
                ("rho", C.c_double), ("twist", C.c_double * 3), ("n_amplitudes", C.c_int64),
                ("channel_hash", C.c_uint64)]


class pnm_mlp_opts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("seed", C.c_ulonglong),
                ("lr_final", C.c_double)]


class PnmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


_lib = None


def load(path=None):
    """Load libpnmcc.so (built by ``paper_1611_06765_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError("libpnmcc.so is not built (%s); run paper_1611_06765_gb300.build.build()" % path)
    L = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    L.pnm_default_opts.restype = None
    L.pnm_default_opts.argtypes = [C.POINTER(pnm_solve_opts)]
    L.pnm_create.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(pnm_minnesota), vp, C.POINTER(vp)]
    L.pnm_create_batch.argtypes = [C.c_int, ip, dp, ip, C.POINTER(pnm_minnesota), vp, C.POINTER(vp)]
    L.pnm_create_twisted.argtypes = [C.c_int, ip, dp, ip, dp, C.POINTER(pnm_minnesota), vp,
                                     C.POINTER(vp)]
    L.pnm_twist_mesh.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
    L.pnm_create_matter.argtypes = [C.c_int, ip, ip, dp, ip, dp, C.POINTER(pnm_minnesota), vp,
                                    C.POINTER(vp)]
    L.pnm_destroy.argtypes = [vp]
    L.pnm_num_systems.argtypes = [vp, ip]
    L.pnm_basis.argtypes = [vp, C.c_int, ip, ip, vp, vp]
    L.pnm_channels.argtypes = [vp, C.c_int, C.c_int, ip, ip, vp, vp, vp]
    L.pnm_v_element.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp]
    L.pnm_eref.argtypes = [vp, dp]
    L.pnm_mbpt2.argtypes = [vp, dp]
    L.pnm_mbpt2_noalloc.argtypes = [vp, dp]
    L.pnm_mbpt3.argtypes = [vp, dp]
    L.pnm_ladder_sizes.argtypes = [vp, C.c_int, ip, vp]
    L.pnm_ccd_solve.argtypes = [vp, C.POINTER(pnm_solve_opts), dp, ip, dp]
    L.pnm_energy_history.argtypes = [vp, C.c_int, dp, C.c_int, ip]
    L.pnm_amplitude_labels.argtypes = [vp, C.c_int, C.POINTER(C.c_size_t), vp]
    L.pnm_get_amplitudes.argtypes = [vp, C.c_int, vp, C.c_size_t]
    L.pnm_set_amplitudes.argtypes = [vp, C.c_int, vp, C.c_size_t]
    L.pnm_get_timings.argtypes = [vp, dp, C.c_int]
    L.pnm_apply_pp_ladder.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.c_size_t]
    L.pnm_apply_ph_term.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.c_size_t]
    fp = C.POINTER(C.c_float)
    L.pnm_mlp_num_params.argtypes = [ip]
    L.pnm_mlp_init.argtypes = [fp, C.c_ulonglong]
    L.pnm_mlp_features.argtypes = [vp, C.c_int, vp, vp, vp]
    L.pnm_mlp_train.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(pnm_mlp_opts), fp, fp, C.c_int, ip]
    L.pnm_mlp_set_model.argtypes = [vp, fp]
    L.pnm_mlp_predict.argtypes = [vp]
    L.pnm_checkpoint_header_of.argtypes = [vp, C.c_int, C.POINTER(pnm_checkpoint_header)]
    L.pnm_checkpoint_save.argtypes = [vp, C.c_char_p]
    L.pnm_checkpoint_load.argtypes = [vp, C.c_char_p]
    L.pnm_mlp_forward.argtypes = [fp, fp, C.c_long, fp, C.c_int, vp]
    L.pnm_mlp_loss_grad.argtypes = [fp, fp, fp, C.c_int, fp, fp, C.c_int, vp]
    L.pnm_get_tuning.argtypes = [vp, ip, ip, C.POINTER(C.c_float), ip]
    L.pnm_selftest_timeout.argtypes = [vp]
    L.pnm_measure_fma_peak.argtypes = [C.c_int, vp, dp]
    L.pnm_set_profiling.argtypes = [vp, C.c_int]
    L.pnm_kernel_stats.argtypes = [vp, C.c_int, C.POINTER(C.c_char_p), dp, ip]
    L.pnm_last_error.restype = C.c_char_p
    L.pnm_last_error.argtypes = []
    for name in EXPORTS:
        if name not in ("pnm_default_opts", "pnm_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(rc, allow=()):
    """Raise PnmError for a negative return code not listed in ``allow``."""
    if rc != PNM_OK and rc not in allow:
        raise PnmError(rc, load().pnm_last_error().decode())
    return rc
