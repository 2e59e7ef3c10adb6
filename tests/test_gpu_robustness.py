"""Failure handling and tuning on the GPU, without faulting it: the bounded device wait,
the learned-start fallback, option validation, the autotuners, and a mixed-precision batch."""
import numpy as np
import pytest

from conftest import minnesota_params
from oracle import channel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


def test_bounded_wait_reports_timeout_and_context_survives(pkg):
    from paper_1611_06765_gb300 import _lib
    g = pkg.Context(14, 0.08, 4, params=minnesota_params())
    assert _lib.load().pnm_selftest_timeout(g._h) == _lib.PNM_ETIMEOUT
    dE, it, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    o = channel.OracleSystem(14, 0.08, 4, minnesota_params())
    dE_o, it_o, _, _ = o.ccd(alpha=0.5, tol=1e-10, maxit=300)
    assert it[0] == it_o and abs(dE[0] - dE_o) <= 1e-10 * abs(dE_o)
    g.close()


def test_learned_start_falls_back_to_mbpt2(pkg):
    """A model whose predictions are far off: the CCD iteration from it fails, the solver
    restarts from the MBPT2 guess and returns that result."""
    g = pkg.Context(14, 0.08, 20, params=minnesota_params())
    blob = pkg.mlp_init(seed=3)
    blob[64] = 1e6  # y_scale: predictions a million times too large
    g.mlp_set_model(blob)
    ref, it_ref, _, _ = g.solve(alpha=0.5, tol=1e-10, max_iter=60)
    dE, it, _, rc = g.solve(alpha=0.5, tol=1e-10, max_iter=60, init=pkg.PNM_INIT_MLP)
    assert rc == 0
    assert dE[0] == ref[0] and it[0] == it_ref[0]
    g.close()


def test_option_validation(pkg):
    g = pkg.Context(14, 0.08, 4, params=minnesota_params())
    for kw in (dict(alpha=0.0), dict(alpha=1.5), dict(precision=7), dict(max_iter=0), dict(init=9),
               dict(tol=0.0, tol_per_N=0.0), dict(refine_sweeps=-1)):
        with pytest.raises(pkg.PnmError) as e:
            g.solve(**kw)
        assert e.value.code == -1
    bad = pkg.mlp_init(seed=0)
    bad[100] = np.inf
    with pytest.raises(pkg.PnmError):
        g.mlp_set_model(bad)
    g.close()


def test_autotuner_choices_are_valid(pkg):
    g = pkg.Context(14, 0.08, 20, params=minnesota_params())
    g.solve(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-6, max_iter=300,
            refine_sweeps=2, allow=(pkg.PNM_ENOTCONV,))
    ksplit, stages, us, mask = g.tuning()
    assert ksplit in (1, 2, 4) and stages in (2, 3, 4) and us > 0
    assert mask & 12 == 0  # both precision modes tuned
    g.close()


def test_mixed_precision_batch(pkg):
    rhos = [0.05, 0.1, 0.2]
    g = pkg.Context(14, rhos, 20, params=minnesota_params())
    dE, it, _, _ = g.solve(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-8,
                           max_iter=300, refine_sweeps=3, allow=(pkg.PNM_ENOTCONV,))
    for k, rho in enumerate(rhos):
        o = channel.OracleSystem(14, rho, 20, minnesota_params())
        dE_o, _, _, _ = o.ccd(alpha=0.5, tol=1e-10 * 14, maxit=300)
        assert abs(dE[k] - dE_o) / 14 < 1e-6
    g.close()


def test_fma_peak_measurement(pkg):
    """The FMA-rate microbenchmark returns a finite rate, FP32 above FP64."""
    fp64 = pkg.measure_fma_peak(True)
    fp32 = pkg.measure_fma_peak(False)
    assert 0.1 < fp64 < 1000.0 and 1.0 < fp32 < 1000.0
    assert fp32 > fp64


def test_refinement_runs_exactly_the_requested_sweeps(pkg):
    """refine_sweeps FP64 updates always follow the converged mixed phase (the FP64 stopping
    test only counts from the last of them on)."""
    g = pkg.Context(14, 0.08, 20, params=minnesota_params())
    kw = dict(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-6, max_iter=300)
    _, it0, _, _ = g.solve(refine_sweeps=0, **kw)
    for k in (1, 2, 3):
        _, itk, _, rc = g.solve(refine_sweeps=k, **kw)
        assert rc == 0
        assert itk[0] >= it0[0] + k, (k, it0, itk)
    g.close()
