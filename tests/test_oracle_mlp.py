"""Pins of the FP64 warm-start network reference: analytic gradient vs central finite
differences (without BF16 rounding, where the loss is smooth), the BF16 rounding against
known values, and GELU against its textbook values."""
import numpy as np

from inputs import random_mlp
from oracle import mlp


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.140625, 65504.0, 1e-3], np.float32)
    got = mlp.bf16(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1.0); 1.005859375 rounds up
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0078125
    assert got[3] == -3.140625
    assert got[4] == 65536.0
    assert abs(got[5] - 1e-3) <= 2 ** -9 * 1e-3


def test_gelu_values():
    """The tanh form of GELU stays within 5e-4 of x Phi(x) (its known maximum deviation is
    4.7e-4; a dropped cubic term gives 3.4e-2), at the tabulated normal CDF values
    Phi(1) = 0.8413447460685429, Phi(3) = 0.9986501019683699 and on a grid against the
    library erf; gelu(x) - gelu(-x) = x exactly; the derivative matches central differences."""
    from scipy.special import erf
    z = np.array([0.0, 1.0, -1.0, 3.0])
    expect = np.array([0.0, 0.8413447460685429, -0.15865525393145707, 3 * 0.9986501019683699])
    assert np.max(np.abs(mlp.gelu(z) - expect)) < 5e-4
    assert mlp.gelu(0.0) == 0.0
    x = np.linspace(-8.0, 8.0, 4001)
    assert np.max(np.abs(mlp.gelu(x) - 0.5 * x * (1.0 + erf(x / np.sqrt(2.0))))) < 5e-4
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, rtol=1e-13, atol=1e-13)
    h = 1e-6
    zz = np.array([-3.0, -1.0, -0.3, 0.0, 0.5, 1.0, 3.0])
    assert np.allclose(mlp.gelu_prime(zz), (mlp.gelu(zz + h) - mlp.gelu(zz - h)) / (2 * h), rtol=1e-8, atol=1e-10)


def test_analytic_gradient_matches_finite_differences():
    blob, X, T = random_mlp(n=16, seed=3)
    loss, g = mlp.loss_and_grad(blob, X, T, round_bf16=False)
    rng = np.random.default_rng(5)
    off = mlp.offsets()
    picks = []
    for name, (o, k) in off.items():
        picks += list(o + rng.choice(k, size=min(k, 6), replace=False))
    b64 = blob.astype(np.float64)
    for idx in picks:
        h = 1e-5 * max(1.0, abs(b64[idx]))
        bp = b64.copy(); bp[idx] += h
        bm = b64.copy(); bm[idx] -= h
        lp, _ = mlp.loss_and_grad(bp, X, T, round_bf16=False)
        lm, _ = mlp.loss_and_grad(bm, X, T, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * abs(fd) + 1e-10, (idx, fd, g[idx])


def test_abs_bounds_dominate_and_are_tight_without_cancellation():
    """abs_bounds: B_y >= |y| and B_g >= |grad| element by element on random parameters;
    with nonnegative inputs, weights and biases (so z >= 0 and gelu'(z) > 0) and targets
    below every output (so y - T > 0) no sum has terms of both signs and the scales equal the
    absolute values of the output and of the gradient."""
    blob, X, T = random_mlp(n=64, seed=13)
    y, _ = mlp.forward(blob, X, round_bf16=True)
    _, g = mlp.loss_and_grad(blob, X, T, round_bf16=True)
    By, Bg = mlp.abs_bounds(blob, X, T, round_bf16=True)
    assert np.all(By >= np.abs(y) * (1 - 1e-12))
    assert np.all(Bg >= np.abs(g) * (1 - 1e-12))
    assert np.all(Bg[:mlp.HEADER] == 0)
    pos = np.abs(blob).astype(np.float32)
    pos[:mlp.F] = 0.0                      # mu
    pos[mlp.F:2 * mlp.F] = 1.0             # inv_std
    Xp = np.abs(X)
    Tn = -np.ones(len(T), np.float32)
    for rnd in (False, True):
        y, _ = mlp.forward(pos, Xp, round_bf16=rnd)
        _, g = mlp.loss_and_grad(pos, Xp, Tn, round_bf16=rnd)
        By, Bg = mlp.abs_bounds(pos, Xp, Tn, round_bf16=rnd)
        assert np.allclose(By, np.abs(y), rtol=1e-13, atol=0)
        assert np.allclose(Bg, np.abs(g), rtol=1e-13, atol=0)
