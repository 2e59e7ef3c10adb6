"""FP64 reference of the learned warm-start network (not part of the paper: the warm start of the CCD iteration).

TEST INFRASTRUCTURE ONLY.

Model (the definition the CUDA kernels implement):
  x_n = (x - mu) * inv_std                            feature normalisation (F = 32 inputs)
  h_0 = bf16(x_n)
  z_l = h_{l-1} W_l^T + b_l,  h_l = bf16(gelu(z_l))   l = 1, 2, 3 (width 128)
  y   = h_3 w_4 + b_4                                  scalar output
  loss = mean((y - target)^2)
with gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (the tanh form of GELU),
weights used through their BF16 rounding, and the
rounding of activations treated as the identity in the backward pass (straight-through).
bf16() is round-to-nearest-even on float32, as __float2bfloat16_rn.

Parameter blob (float32), the layout shared with include/pnmcc.h:
  mu[32], inv_std[32], y_scale, pad[3], W1[128][32], b1[128], W2[128][128], b2[128],
  W3[128][128], b3[128], w4[128], b4
"""
import numpy as np

F = 32
H = 128
HEADER = 2 * F + 4
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
         ("w4", (H,)), ("b4", (1,))]
NPARAM = HEADER + sum(int(np.prod(s)) for _, s in SIZES)


def unpack(blob):
    blob = np.asarray(blob)
    if blob.dtype != np.float64:
        blob = blob.astype(np.float32)
    assert blob.size == NPARAM
    out = {"mu": blob[:F], "inv_std": blob[F:2 * F], "y_scale": blob[2 * F]}
    o = HEADER
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = blob[o:o + n].reshape(shape)
        o += n
    return out


def offsets():
    o = HEADER
    res = {}
    for name, shape in SIZES:
        n = int(np.prod(shape))
        res[name] = (o, n)
        o += n
    return res


def bf16(x):
    """Round float32 values to bfloat16 (round to nearest even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


GELU_C = np.sqrt(2.0 / np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + 0.044715 * z ** 3)))


def gelu_prime(z):
    th = np.tanh(GELU_C * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * GELU_C * (1.0 + 3 * 0.044715 * z * z)


def forward(blob, X, round_bf16=True):
    """Returns (y, cache).  X: (n, 32) raw features."""
    p = unpack(blob)
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, np.float64))
    W = [rnd(p["W1"]), rnd(p["W2"]), rnd(p["W3"])]
    w4 = rnd(p["w4"])
    b = [p["b1"].astype(np.float64), p["b2"].astype(np.float64), p["b3"].astype(np.float64)]
    xn = (np.asarray(X, np.float64) - p["mu"]) * p["inv_std"]
    h = [rnd(xn)]
    z = []
    for l in range(3):
        zl = h[-1] @ W[l].T + b[l]
        z.append(zl)
        h.append(rnd(gelu(zl)))
    y = h[3] @ w4 + float(p["b4"][0])
    return y, dict(h=h, z=z, W=W, w4=w4)


def loss_and_grad(blob, X, T, round_bf16=True):
    """Mean squared error and its gradient with respect to the parameter blob (header
    entries get zero gradient)."""
    y, c = forward(blob, X, round_bf16)
    n = len(T)
    r = y - np.asarray(T, np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = np.zeros(NPARAM)
    off = offsets()
    h, z, W = c["h"], c["z"], c["W"]

    def put(name, val):
        o, k = off[name]
        g[o:o + k] = np.ravel(val)

    put("w4", dy @ h[3])
    put("b4", [dy.sum()])
    dh = np.outer(dy, c["w4"])
    for l in (2, 1, 0):
        dz = dh * gelu_prime(z[l])
        put("W%d" % (l + 1), dz.T @ h[l])
        put("b%d" % (l + 1), dz.sum(axis=0))
        dh = dz @ W[l]
    return loss, g


def abs_bounds(blob, X, T, round_bf16=True):
    """Absolute-value scales of the network's output and gradient, for rounding-aware
    tolerances: the forward pass of forward() and the backward pass of loss_and_grad() with
    every factor replaced by its absolute value (|h|, |W|, |b|, |dy|, |gelu'(z)|), at the same
    activations.  Returns (B_y per sample, B_g per parameter); B_y >= |y| and B_g >= |grad|
    element by element (triangle inequality), with equality when no sum has terms of both
    signs.  A rounding error of relative size u in any one factor moves y or a gradient
    element by at most about u times its scale."""
    y, c = forward(blob, X, round_bf16)
    p = unpack(blob)
    h, z, W = c["h"], c["z"], c["W"]
    aw4 = np.abs(c["w4"])
    By = np.abs(h[3]) @ aw4 + abs(float(p["b4"][0]))
    n = len(T)
    ady = 2.0 * np.abs(y - np.asarray(T, np.float64)) / n
    g = np.zeros(NPARAM)
    off = offsets()

    def put(name, val):
        o, k = off[name]
        g[o:o + k] = np.ravel(val)

    put("w4", ady @ np.abs(h[3]))
    put("b4", [ady.sum()])
    dh = np.outer(ady, aw4)
    for l in (2, 1, 0):
        dz = dh * np.abs(gelu_prime(z[l]))
        put("W%d" % (l + 1), dz.T @ np.abs(h[l]))
        put("b%d" % (l + 1), dz.sum(axis=0))
        dh = dz @ np.abs(W[l])
    return By, g
