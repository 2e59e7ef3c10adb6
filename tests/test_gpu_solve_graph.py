"""The whole-solve graph (one launch per solve: start, iteration loop, refinement gate and loop,
settling, read-back) against the host-driven path (one update per host step), and its run-time
parameters and invalidation."""
import numpy as np
import pytest

from conftest import minnesota_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


def _both(g, **kw):
    """The same solve through the graph and host-driven: (dE, iters, resid, amplitudes) each."""
    out = []
    for host in (False, True):
        dE, it, res, rc = g.solve(host_loop=host, **kw)
        amps = [g.get_amplitudes(s) for s in range(g.nsys)]
        out.append((dE.copy(), it.copy(), res.copy(), rc, amps))
    return out


@pytest.mark.parametrize("kind", ["mixed_pair", "mixed_fp64refine", "fp64", "ccd2"])
def test_graph_solve_equals_host_driven_solve(pkg, kind):
    """Every configuration ends bit for bit where the host-driven loop ends: the same kernels
    in the same order, only the control (loop parameters, refinement gate, settling) moved onto
    the device."""
    P = minnesota_params()
    g = pkg.Context(14, [0.06, 0.12], 20, params=P)
    kw = dict(alpha=0.5, tol=1e-30, tol_per_N=1e-6, max_iter=300)
    if kind == "mixed_pair":
        kw.update(precision=pkg.PNM_PREC_BF16X3, refine_sweeps=2, refine_kernels=pkg.PNM_PREC_F32PAIR)
    elif kind == "mixed_fp64refine":
        kw.update(precision=pkg.PNM_PREC_BF16X3, refine_sweeps=2, refine_kernels=pkg.PNM_PREC_FP64)
    elif kind == "ccd2":
        kw.update(terms=pkg.PNM_TERMS_PPHH, tol_per_N=1e-8)
    else:
        kw.update(tol_per_N=1e-8)
    (dg, ig, rg, cg, ag), (dh, ih, rh, ch, ah) = _both(g, **kw)
    assert cg == ch == 0
    assert np.array_equal(ig, ih), (ig, ih)
    assert np.array_equal(dg, dh), (dg, dh)
    assert np.array_equal(rg, rh)
    for a, b in zip(ag, ah):
        assert np.array_equal(a, b)
    g.close()


def test_unconverged_mixed_phase_skips_refinement(pkg):
    """A mixed loop stopped by its cap returns PNM_ENOTCONV after exactly max_iter updates: the
    device-side gate runs no refinement sweep."""
    g = pkg.Context(14, 0.08, 20, params=minnesota_params())
    kw = dict(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-9, max_iter=3,
              refine_sweeps=2, allow=(pkg.PNM_ENOTCONV,))
    for host in (False, True):
        _, it, _, rc = g.solve(host_loop=host, **kw)
        assert rc == pkg.PNM_ENOTCONV
        assert it[0] == 3, it
    g.close()


def test_run_time_parameters_reach_the_graph(pkg):
    """alpha, the iteration caps and the tolerances are run-time inputs of the cached graph:
    solving with other values and back again reproduces a fresh context's results."""
    P = minnesota_params()
    kw = dict(precision=pkg.PNM_PREC_BF16X3, tol=1e-30, max_iter=300, refine_sweeps=2,
              refine_kernels=pkg.PNM_PREC_F32PAIR)
    g = pkg.Context(14, 0.08, 20, params=P)
    first = g.solve(alpha=0.5, tol_per_N=1e-6, **kw)
    other = g.solve(alpha=0.6, tol_per_N=1e-7, **kw)
    again = g.solve(alpha=0.5, tol_per_N=1e-6, **kw)
    g.close()
    fresh = pkg.Context(14, 0.08, 20, params=P)
    ref_other = fresh.solve(alpha=0.6, tol_per_N=1e-7, **kw)
    fresh.close()
    assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])
    assert np.array_equal(other[0], ref_other[0]) and np.array_equal(other[1], ref_other[1])
    assert not np.array_equal(first[1], other[1]) or not np.array_equal(first[0], other[0])


def test_new_model_invalidates_the_graph(pkg):
    """The learned start's kernels hold the model's output scale as an argument: after
    pnm_mlp_set_model the next solve starts from the new model (as a fresh context would)."""
    P = minnesota_params()
    kw = dict(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-6, max_iter=300,
              refine_sweeps=2, refine_kernels=pkg.PNM_PREC_F32PAIR, init=pkg.PNM_INIT_MLP)
    a = pkg.mlp_init(seed=4)
    a[64] = 1e-3  # y_scale: starts close to the MBPT2 guess, so both converge without fallback
    b = a.copy()
    b[64] = 2e-3  # another output scale
    g = pkg.Context(14, 0.08, 20, params=P)
    g.mlp_set_model(a)
    with_a = g.solve(**kw)
    g.mlp_set_model(b)
    got = g.solve(**kw)
    assert g.timings()["mlp_fallback"] == 0
    g.close()
    fresh = pkg.Context(14, 0.08, 20, params=P)
    fresh.mlp_set_model(b)
    ref = fresh.solve(**kw)
    fresh.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert not np.array_equal(with_a[0], got[0])  # the two models start differently
