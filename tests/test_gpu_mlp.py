"""Learned warm start: GPU training kernels against the FP64 reference network element by
element (an FP32 debug mode without BF16 rounding, and the BF16 mode against rounding-aware
scales), the fused tensor-core inference per output, the feature kernel against a numpy
restatement, and the solve the metric is defined on (learned start, BF16x3 ladders, two FP64
refinement sweeps; N = 66, n^2 <= 36, held-out densities) against the oracle's fixed point.
"""
import math

import numpy as np
import pytest

from conftest import minnesota_params
from inputs import random_mlp
from oracle import channel, mlp

pytestmark = pytest.mark.gpu

HELDOUT = [0.05, 0.11, 0.17]
# One BF16 unit relative to a value (8 significant bits: 2^-7 at most): the size of the
# difference a rounding decision taken in FP32 on the GPU and in FP64 in the reference can make.
BF16_UNIT = 2.0 ** -7


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


def _per_tensor(g):
    for name, (o, k) in mlp.offsets().items():
        yield name, slice(o, o + k)


def test_param_count(pkg):
    assert pkg.mlp_num_params() == mlp.NPARAM


def test_fp32_gradient_matches_reference_elementwise(pkg):
    """FP32 debug mode (the training kernels with the BF16 rounding switched off) against the
    FP64 reference without rounding: every gradient element within 1e-6 of its tensor's
    largest element, the loss within 1e-6 relative, every output within 1e-6 of the largest."""
    blob, X, T = random_mlp(n=256, seed=11, nparam=mlp.NPARAM)
    loss_g, g_g = pkg.mlp_loss_grad(blob, X, T, fp32=True)
    loss_r, g_r = mlp.loss_and_grad(blob, X, T, round_bf16=False)
    assert abs(loss_g - loss_r) <= 1e-6 * abs(loss_r)
    worst = 0.0
    for name, sl in _per_tensor(g_r):
        a, b = g_g[sl].astype(np.float64), g_r[sl]
        scale = np.max(np.abs(b))
        worst = max(worst, np.max(np.abs(a - b)) / scale)
        assert np.all(np.abs(a - b) <= 1e-6 * scale), name
    print("FP32 gradient: max |error| / tensor max = %.3g" % worst)
    assert np.all(g_g[:mlp.HEADER] == 0)
    y_g = pkg.mlp_forward(blob, X, tensor_cores=False, fp32=True)
    y_r, _ = mlp.forward(blob, X, round_bf16=False)
    assert np.all(np.abs(y_g - y_r) <= 1e-6 * np.max(np.abs(y_r)))


@pytest.mark.parametrize("tensor_cores", [True, False])
@pytest.mark.parametrize("n", [256, 300])
def test_bf16_gradient_within_rounding_scale_elementwise(pkg, n, tensor_cores):
    """BF16 mode: the GPU rounds activations after FP32 arithmetic, the reference after FP64,
    so a rounding decision can differ by one BF16 unit.  Every gradient element stays within
    one BF16 unit of its absolute-value scale (oracle.mlp.abs_bounds), every element within
    1e-4 of its tensor's largest, and the whole gradient within 1e-3 in L2.  Both the tcgen05
    products training uses (operands split into BF16 hi + lo, exact for the BF16 weights and
    layer inputs, 2^-18 for the FP32 error signals) and the SIMT ones; n = 300 leaves a partial
    128-row tile, a partial 64-wide k stage and a k range split over several CTAs."""
    blob, X, T = random_mlp(n=n, seed=11, nparam=mlp.NPARAM)
    loss_g, g_g = pkg.mlp_loss_grad(blob, X, T, tensor_cores=tensor_cores)
    loss_r, g_r = mlp.loss_and_grad(blob, X, T, round_bf16=True)
    _, B_g = mlp.abs_bounds(blob, X, T, round_bf16=True)
    assert abs(loss_g - loss_r) <= 1e-4 * abs(loss_r)
    for name, sl in _per_tensor(g_r):
        a, b = g_g[sl].astype(np.float64), g_r[sl]
        assert np.all(np.abs(a - b) <= BF16_UNIT * B_g[sl]), name
        assert np.all(np.abs(a - b) <= 1e-4 * np.max(np.abs(b))), name
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), name
    assert np.all(g_g[:mlp.HEADER] == 0)


def test_tensor_core_forward_per_output(pkg):
    """The fused tcgen05 inference (BF16 operands, FP32 accumulation in tensor memory, hardware
    tanh in GELU) per output against the reference and against the SIMT forward: within two
    BF16 units of the output's absolute-value scale B_y = sum_k |h3_k w4_k| + |b4|, and the SIMT
    BF16 forward within one unit.  A misplaced row or column gives errors of the order of |y|,
    about B_y / 10 for these random networks."""
    blob, X, T = random_mlp(n=1000, seed=12, nparam=mlp.NPARAM)
    y_tc = pkg.mlp_forward(blob, X, tensor_cores=True).astype(np.float64)
    y_simt = pkg.mlp_forward(blob, X, tensor_cores=False).astype(np.float64)
    y_ref, _ = mlp.forward(blob, X, round_bf16=True)
    B_y, _ = mlp.abs_bounds(blob, X, T, round_bf16=True)
    print("max |tc - ref| / B_y = %.3g, max |simt - ref| / B_y = %.3g"
          % (np.max(np.abs(y_tc - y_ref) / B_y), np.max(np.abs(y_simt - y_ref) / B_y)))
    assert np.all(np.abs(y_simt - y_ref) <= BF16_UNIT * B_y)
    assert np.all(np.abs(y_tc - y_ref) <= 2 * BF16_UNIT * B_y)
    assert np.all(np.abs(y_tc - y_simt) <= 2 * BF16_UNIT * B_y)
    assert np.median(np.abs(y_tc - y_ref) / B_y) <= 2.0 ** -12


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


@pytest.fixture(scope="module")
def trained(pkg):
    """The warm-start network as the benchmark trains it: the library's kernels (matrix
    products on the tensor cores) on the amplitudes the FP64 solver converges (|dE/N| < 1e-8 MeV) for N = 14 (n^2 <= 20, 16
    densities 0.02 ... 0.32) and N = 66 (n^2 <= 36, rho = 0.04, 0.06, ..., 0.20, none of them
    held out); 40 epochs, batch 1024, Adam with the learning rate decaying from 1e-3 to 1e-5
    along a half cosine, seeds 1 (initial weights) and 3 (shuffling)."""
    P = minnesota_params()
    kw = dict(alpha=0.5, tol=1e-30, tol_per_N=1e-8, max_iter=300)
    train14 = pkg.Context(14, [0.02 * k for k in range(1, 17)], 20, params=P)
    train14.solve(**kw)
    train66 = pkg.Context(66, [0.04, 0.06, 0.08, 0.10, 0.12, 0.14, 0.16, 0.18, 0.20], 36, params=P)
    train66.solve(**kw)
    blob, hist = pkg.mlp_train([train14, train66], pkg.mlp_init(seed=1), epochs=40, batch=1024, lr=1e-3, seed=3,
                               lr_final=1e-5)
    for c in (train14, train66):
        c.close()
    assert hist[-1] < hist[0]
    return blob


def test_learned_start_matches_network_on_features(pkg, trained):
    """The learned start forms its features inside the inference kernel.  Every amplitude it
    writes is the network applied to the feature row pnm_mlp_features returns (checked above
    against a numpy restatement), t_MBPT2 + sigma_sys y_scale y.  Rows the updates compute get
    their own prediction, the other rows the prediction of their spin-flip partner (sign of
    the reordering of the restricted pairs).  Two densities in one context, to cover the
    per-system constants.  The only allowed difference is the rounding of the fused
    multiply-add the kernel may form: 2^-50 of |t_MBPT2| + |sigma y_scale y|."""
    P = minnesota_params()
    g = pkg.Context(14, [0.06, 0.12], 20, params=P)
    g.mlp_set_model(trained)
    g.mlp_predict()
    y_scale = float(trained[2 * 32])  # the blob header: mu[32], inv_std[32], y_scale, pad[3]
    for sys in range(2):
        t0 = g.get_amplitudes(sys)
        X, tm2, sigma = g.mlp_features(sys)
        y = pkg.mlp_forward(trained, X, tensor_cores=True).astype(np.float64)
        pred = tm2 + sigma * y_scale * y
        tol = 2.0 ** -50 * (np.abs(tm2) + np.abs(sigma * y_scale * y))
        nv, _, _ = g.basis(sys)
        where = {tuple(int(u) for u in nv[p]): p for p in range(len(nv))}
        flip = np.array([where[(int(q[0]), int(q[1]), int(q[2]), -int(q[3]))] for q in nv])
        labels = g.amplitude_labels(sys)
        index = {tuple(int(u) for u in lab): z for z, lab in enumerate(labels)}
        own = np.abs(t0 - pred) <= tol
        partner_ok = np.zeros(len(t0), bool)
        for z in np.nonzero(~own)[0]:
            a, b, i, j = (int(flip[p]) for p in labels[z])
            sign = 1.0
            if (a, b, i, j) not in index:
                if (b, a, i, j) in index:
                    a, b, sign = b, a, -1.0
                elif (a, b, j, i) in index:
                    i, j, sign = j, i, -1.0
                else:
                    a, b, i, j = b, a, j, i
            zp = index[(a, b, i, j)]
            partner_ok[z] = abs(t0[z] - sign * pred[zp]) <= tol[zp]
        frac_own = own.mean()
        print("sys %d: %d amplitudes, %.3f own predictions" % (sys, len(t0), frac_own))
        assert np.all(own | partner_ok)
        assert 0.4 <= frac_own
    g.close()


@pytest.fixture(scope="module")
def heldout_oracle():
    """The oracle's CCD energy per neutron at the held-out densities (mixing 0.5, MBPT2 start):
    stopped by the metric's rule |dE^(n+1) - dE^(n)| / N < 1e-6 MeV, and converged to its fixed
    point (1e-10 MeV)."""
    P = minnesota_params()
    rule, fixed = [], []
    for rho in HELDOUT:
        o = channel.OracleSystem(66, rho, 36, P)
        dE, _, _, _ = o.ccd(alpha=0.5, tol=1e-6 * 66, maxit=400)
        rule.append(dE / 66)
        dE, _, _, _ = o.ccd(alpha=0.5, tol=1e-10 * 66, maxit=400)
        fixed.append(dE / 66)
    return np.array(rule), np.array(fixed)


def test_metric_configuration_against_oracle(pkg, trained, heldout_oracle):
    """The configuration the time-to-converge metric is quoted on: N = 66, n^2 <= 36, held-out
    rho = 0.05, 0.11, 0.17 in one batched context, learned start, BF16x3 tensor-core ladders
    with FP32 contractions, stopping rule |dE^(n+1) - dE^(n)| / N < 1e-6 MeV, then two FP64
    refinement sweeps (FP32-pair contractions, FP64 update), without the MBPT2 fallback, in at
    least 25% fewer updates than the same solve from the MBPT2 start (Eq. ccdGuess).
    The stopping rule (Sec. "Developing a CCD code") ends an iteration somewhere in a band
    around the fixed point: the FP64 oracle stopped by it sits 1.1e-6 to 1.4e-6 MeV per neutron
    above its fixed point.  From the MBPT2 start the GPU follows the oracle's own trajectory and
    matches the oracle at the rule within 1e-6 MeV per neutron.  From the learned start it
    follows another one and stops at another point of the band, so it is held to the fixed
    point: at every density it ends at least as close to the oracle's fixed point as the oracle
    stopped by the same rule (and within 1.5e-6 MeV per neutron)."""
    rule, fixed = heldout_oracle
    test = pkg.Context(66, HELDOUT, 36, params=minnesota_params())
    test.mlp_set_model(trained)
    kw = dict(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-6, max_iter=500,
              refine_sweeps=2, refine_kernels=pkg.PNM_PREC_F32PAIR)
    dE_m, it_m, _, _ = test.solve(init=pkg.PNM_INIT_MBPT2, **kw)
    dE_l, it_l, _, _ = test.solve(init=pkg.PNM_INIT_MLP, **kw)
    assert test.timings()["mlp_fallback"] == 0
    for k in range(3):
        print("rho %.2f learned-start energies per neutron:" % HELDOUT[k], np.round(test.history(k) / 66, 8))
    print("learned start: updates %s, dE/N - oracle at the rule %s, - fixed point %s"
          % (it_l, dE_l / 66 - rule, dE_l / 66 - fixed))
    print("MBPT2 start:   updates %s, dE/N - oracle at the rule %s, - fixed point %s"
          % (it_m, dE_m / 66 - rule, dE_m / 66 - fixed))
    assert np.all(np.abs(dE_m / 66 - rule) < 1e-6)
    assert np.all(np.abs(dE_l / 66 - fixed) <= np.abs(rule - fixed)), (dE_l / 66 - fixed, rule - fixed)
    assert np.all(np.abs(dE_l / 66 - fixed) < 1.5e-6)
    assert np.all(np.abs(dE_m / 66 - fixed) < 1.5e-6)
    assert np.all(it_l <= 0.75 * it_m), (it_l, it_m)
    test.close()


def test_warm_start_gain_fp64(pkg, trained):
    """In FP64 the learned start reaches the same fixed point as the MBPT2 start
    (|dE/N| difference < 1e-6 MeV at a 1e-8 MeV rule) in fewer updates."""
    test = pkg.Context(66, HELDOUT, 36, params=minnesota_params())
    test.mlp_set_model(trained)
    kw = dict(alpha=0.5, tol=1e-30, tol_per_N=1e-8, max_iter=300)
    dE_m, it_m, _, _ = test.solve(init=pkg.PNM_INIT_MBPT2, **kw)
    dE_l, it_l, _, _ = test.solve(init=pkg.PNM_INIT_MLP, **kw)
    assert np.all(np.abs(dE_l - dE_m) / 66 < 1e-6)
    assert it_l.sum() < it_m.sum(), (it_l, it_m)
    test.close()
