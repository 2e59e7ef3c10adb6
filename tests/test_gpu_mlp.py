"""Learned warm start: GPU training kernels against the FP64 reference network, the fused
tensor-core inference against the SIMT forward, the feature kernel against a numpy
restatement, and the gain of the trained network over the MBPT2 start at held-out densities.
"""
import math

import numpy as np
import pytest

from conftest import minnesota_params
from inputs import random_mlp
from oracle import channel, mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


def test_param_count(pkg):
    assert pkg.mlp_num_params() == mlp.NPARAM


def test_loss_and_gradient_match_reference(pkg):
    """BF16 activations make single elements jump where a rounding decision flips between
    FP32 and FP64, so the gradient is compared as a whole: relative L2 error <= 1e-2."""
    blob, X, T = random_mlp(n=256, seed=11, nparam=mlp.NPARAM)
    loss_g, g_g = pkg.mlp_loss_grad(blob, X, T)
    loss_r, g_r = mlp.loss_and_grad(blob, X, T, round_bf16=True)
    assert abs(loss_g - loss_r) <= 1e-3 * abs(loss_r)
    for name, (o, k) in mlp.offsets().items():
        a, b = g_g[o:o + k].astype(np.float64), g_r[o:o + k]
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b), name
    assert np.all(g_g[:mlp.HEADER] == 0)


def test_tensor_core_forward_matches_simt_and_reference(pkg):
    blob, X, _ = random_mlp(n=1000, seed=12, nparam=mlp.NPARAM)
    y_tc = pkg.mlp_forward(blob, X, tensor_cores=True)
    y_simt = pkg.mlp_forward(blob, X, tensor_cores=False)
    y_ref, _ = mlp.forward(blob, X, round_bf16=True)
    scale = np.linalg.norm(y_ref)
    assert np.linalg.norm(y_tc - y_simt) <= 1e-2 * scale
    assert np.linalg.norm(y_tc - y_ref) <= 1e-2 * scale
    assert np.linalg.norm(y_simt - y_ref) <= 1e-2 * scale


def test_features_match_numpy(pkg):
    N, rho, n2 = 14, 0.08, 4
    P = minnesota_params()
    g = pkg.Context(N, rho, n2, params=P)
    o = channel.OracleSystem(N, rho, n2, P)
    X, tm2, sigma = g.mlp_features()
    labels = g.amplitude_labels()
    st = o.states()
    _, eps = o.energies()
    kF = (3 * math.pi ** 2 * rho) ** (1 / 3)
    epsF = P[6] * kF * kF
    ks = (2 * math.pi / o.L) / kF
    a, b, i, j = labels.T
    v = np.array([o.v(*row) for row in labels])
    D = eps[i] + eps[j] - eps[a] - eps[b]
    t2 = v / D
    sig = math.sqrt(np.mean(t2 * t2))
    assert np.allclose(tm2, t2, rtol=1e-12, atol=0)
    assert abs(sigma - sig) <= 1e-12 * sig
    ref = np.zeros_like(X, dtype=np.float64)
    for c, p in enumerate((a, b, i, j)):
        ref[:, 3 * c:3 * c + 3] = ks * st[p, :3]
        ref[:, 12 + c] = st[p, 3]
    ref[:, 16] = D / epsF
    ref[:, 17] = v * N / epsF
    ref[:, 18] = t2 / sig
    ref[:, 19] = rho / 0.16
    ref[:, 20] = kF
    ref[:, 21] = N / 66
    assert np.allclose(X, ref, rtol=2e-7, atol=1e-7)
    g.close()


def test_warm_start_gain_at_held_out_densities(pkg):
    """Train on solver amplitudes of N=14 (n^2<=20, 16 densities 0.02..0.32) and N=66
    (n^2<=36, rho=0.16); start N=66 at held-out rho in {0.05, 0.11, 0.17}.  The learned start
    must reach the same fixed point (|dE/N| difference < 1e-6 MeV) in fewer updates."""
    P = minnesota_params()
    kw = dict(alpha=0.5, tol=1e-30, tol_per_N=1e-8, max_iter=300)
    train14 = pkg.Context(14, [0.02 * k for k in range(1, 17)], 20, params=P)
    train14.solve(**kw)
    train66 = pkg.Context(66, 0.16, 36, params=P)
    train66.solve(**kw)
    blob, hist = pkg.mlp_train([train14, train66], pkg.mlp_init(seed=1), epochs=12, batch=4096, lr=1e-3, seed=2)
    assert hist[-1] < hist[0]
    test = pkg.Context(66, [0.05, 0.11, 0.17], 36, params=P)
    test.mlp_set_model(blob)
    dE_m, it_m, _, _ = test.solve(init=pkg.PNM_INIT_MBPT2, **kw)
    dE_l, it_l, _, _ = test.solve(init=pkg.PNM_INIT_MLP, **kw)
    assert np.all(np.abs(dE_l - dE_m) / 66 < 1e-6)
    assert it_l.sum() < it_m.sum(), (it_l, it_m)
    for c in (train14, train66, test):
        c.close()
