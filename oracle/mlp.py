"""CPU oracle of the learned radiance cache's network (numpy, fp64).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU legs; the product path never imports it.

The cache is a small MLP R(x, d) over a frequency encoding of a position x in
[0,1]^3 (grid space over the domain extent) and a unit direction d:

  e(x, d)  = [x, d, sin/cos(2^l pi x_a) for l < 12, sin/cos(2^l pi d_a) for l < 4, 0...]  (128 wide)
  h1 = relu(W1 e + b1),  h2 = relu(W2 h1 + b2),  h3 = relu(W3 h2 + b3)  (3 hidden layers of 64)
  R  = w4 . h3 + b4

trained with the L2 loss (R - target)^2 on path vertices and Adam.  Parameters
are one flat fp32 vector: W1[64][128], b1[64], W2[64][64], b2[64], W3[64][64],
b3[64], w4[64], b4.

`bf16=True` evaluates the network the way a BF16 tensor-core implementation
with FP32 accumulation does: the operands of the three matrix products (the
encoding, h1, h2, the weight matrices, and in the backward pass the
pre-activation gradients) are rounded to bf16 (round to nearest even) and the
products are exact sums (fp64 here); biases, h3, the output layer and the
bias gradients stay unrounded.  bf16=False is the plain fp64 network, pinned
by finite differences.
"""
from __future__ import annotations

import numpy as np

WIDTH = 64
ENC = 128
POS_FREQS = 12
DIR_FREQS = 4

# flat parameter layout
O_W1 = 0
O_B1 = O_W1 + WIDTH * ENC
O_W2 = O_B1 + WIDTH
O_B2 = O_W2 + WIDTH * WIDTH
O_W3 = O_B2 + WIDTH
O_B3 = O_W3 + WIDTH * WIDTH
O_W4 = O_B3 + WIDTH
O_B4 = O_W4 + WIDTH
NUM_PARAMS = O_B4 + 1


def unpack(p):
    p = np.asarray(p, np.float64)
    return dict(W1=p[O_W1:O_B1].reshape(WIDTH, ENC), b1=p[O_B1:O_W2], W2=p[O_W2:O_B2].reshape(WIDTH, WIDTH),
                b2=p[O_B2:O_W3], W3=p[O_W3:O_B3].reshape(WIDTH, WIDTH), b3=p[O_B3:O_W4], w4=p[O_W4:O_B4],
                b4=p[O_B4])


def pack(W1, b1, W2, b2, W3, b3, w4, b4):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3, w4, [b4]]).astype(np.float64)


def bf16(a):
    """Round to the nearest bfloat16 (ties to even) via float32, as a float64 array."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def encode(x, d):
    """Frequency encoding of positions x (n,3) in [0,1] and directions d (n,3): (n, 128)."""
    x = np.asarray(x, np.float64)
    d = np.asarray(d, np.float64)
    n = len(x)
    e = np.zeros((n, ENC))
    e[:, 0:3] = x
    e[:, 3:6] = d
    for a in range(3):
        for l in range(POS_FREQS):
            arg = np.pi * (2.0 ** l) * x[:, a]
            e[:, 6 + a * 2 * POS_FREQS + 2 * l] = np.sin(arg)
            e[:, 7 + a * 2 * POS_FREQS + 2 * l] = np.cos(arg)
    base = 6 + 6 * POS_FREQS
    for a in range(3):
        for l in range(DIR_FREQS):
            arg = np.pi * (2.0 ** l) * d[:, a]
            e[:, base + a * 2 * DIR_FREQS + 2 * l] = np.sin(arg)
            e[:, base + 1 + a * 2 * DIR_FREQS + 2 * l] = np.cos(arg)
    return e


def forward(p, x, d, bf16_ops=False):
    """R(x, d) for every row, with the intermediate values (for backward)."""
    P = unpack(p)
    r = bf16 if bf16_ops else (lambda a: np.asarray(a, np.float64))
    e = r(encode(x, d))
    z1 = e @ r(P["W1"]).T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    a1 = r(h1)
    z2 = a1 @ r(P["W2"]).T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    a2 = r(h2)
    z3 = a2 @ r(P["W3"]).T + P["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ P["w4"] + P["b4"]
    return y, dict(e=e, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, h3=h3)


def loss_grad(p, x, d, target, valid, bf16_ops=False):
    """Sum over rows of valid * (R - target)^2, the sum of valid, and the gradient
    of the first with respect to the parameters (not divided by the count)."""
    P = unpack(p)
    r = bf16 if bf16_ops else (lambda a: np.asarray(a, np.float64))
    y, c = forward(p, x, d, bf16_ops)
    w = np.asarray(valid, np.float64)
    res = y - np.asarray(target, np.float64)
    loss = float(np.sum(w * res * res))
    dy = w * 2.0 * res                                   # d loss / d R per row
    g_w4 = c["h3"].T @ dy
    g_b4 = dy.sum()
    dz3 = np.outer(dy, P["w4"]) * (c["z3"] > 0)
    g_b3 = dz3.sum(0)
    dz3r = r(dz3)
    g_W3 = dz3r.T @ c["a2"]
    dz2 = (dz3r @ r(P["W3"])) * (c["z2"] > 0)
    g_b2 = dz2.sum(0)
    dz2r = r(dz2)
    g_W2 = dz2r.T @ c["a1"]
    dz1 = (dz2r @ r(P["W2"])) * (c["z1"] > 0)
    g_b1 = dz1.sum(0)
    g_W1 = r(dz1).T @ c["e"]
    return loss, float(w.sum()), pack(g_W1, g_b1, g_W2, g_b2, g_W3, g_b3, g_w4, g_b4)


def adam(p, m, v, grad, count, step, lr, beta1=0.9, beta2=0.99, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) on the mean gradient
    grad / max(count, 1); step counts from 1.  Returns new (p, m, v)."""
    g = np.asarray(grad, np.float64) / max(float(count), 1.0)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p = np.asarray(p, np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v
