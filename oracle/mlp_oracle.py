"""FP64 CPU oracle for the learned per-frame correction MLP.

TEST INFRASTRUCTURE ONLY (same rule as ``melt_oracle``: only tests, the smoke
check and the bench's CPU-baseline leg may use it; it imports nothing from
the product package).

The paper does not evaluate a correction layer (Sec. VI-C, "Model-capacity
dependence", names a calibration layer as untested; Sec. IV-H and Sec. V
describe the MelT-to-STFT+Mel gap as mostly a per-band affine map).  The
correction here is this project's reading of that remark:

    xh = (x - mu) / sd                          per-band standardisation
    h  = xh W1^T + b1        W1 [Hd x M]
    a  = GELU(h)             exact erf form: 0.5 h (1 + erf(h / sqrt 2))
    y  = x + a W2^T + b2     W2 [M x Hd]        residual output
    L  = mean((y - target)^2)                   MSE in nats over all entries

AdamW (Loshchilov & Hutter, decoupled weight decay) on every parameter:
    m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
    p = p (1 - lr wd) - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(h):
    h = np.asarray(h, np.float64)
    return 0.5 * h * (1.0 + erf(h / SQRT2))


def gelu_grad(h):
    """d GELU / dh = Phi(h) + h phi(h)."""
    h = np.asarray(h, np.float64)
    return 0.5 * (1.0 + erf(h / SQRT2)) + h * INV_SQRT_2PI * np.exp(-0.5 * h * h)


def band_stats(x):
    """Per-band mean and standard deviation (population) of training inputs."""
    x = np.asarray(x, np.float64)
    mu = x.mean(axis=0)
    sd = np.sqrt(np.mean((x - mu) ** 2, axis=0))
    return mu, np.maximum(sd, 1e-6)


def forward(params, x, mu, sd):
    """Returns (y, cache)."""
    W1, b1, W2, b2 = (np.asarray(p, np.float64) for p in params)
    x = np.asarray(x, np.float64)
    xh = (x - mu) / sd
    h = xh @ W1.T + b1
    a = gelu(h)
    y = x + a @ W2.T + b2
    return y, (x, xh, h, a)


def forward_bf16(params, x, mu, sd):
    """The model with the operand rounding of a BF16 tensor-core evaluation.

    x-hat, W1, GELU(h) and W2 are rounded to bfloat16 (nearest-even) before
    they enter a product; the products, the sums and everything else are exact
    (FP64).  Returns (y, (xh_b, h, a_b, W1_b, W2_b)).  A BF16 evaluation
    with FP32 accumulation differs from this only by its summation order and
    by where FP32 rounding moves a value across a bfloat16 rounding boundary.
    """
    from oracle.melt_oracle import round_bf16
    W1, b1, W2, b2 = (np.asarray(p, np.float64) for p in params)
    x = np.asarray(x, np.float64)
    xh_b = round_bf16((x - mu) / sd)
    W1_b, W2_b = round_bf16(W1), round_bf16(W2)
    h = xh_b @ W1_b.T + b1
    a_b = round_bf16(gelu(h))
    y = x + a_b @ W2_b.T + b2
    return y, (xh_b, h, a_b, W1_b, W2_b)


def loss(y, target) -> float:
    d = np.asarray(y, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d))


def backward(params, cache, y, target, sd):
    """Gradients of the MSE loss: (dW1, db1, dW2, db2, dx)."""
    W1, b1, W2, b2 = (np.asarray(p, np.float64) for p in params)
    x, xh, h, a = cache
    dy = 2.0 * (y - np.asarray(target, np.float64)) / y.size
    dW2 = dy.T @ a
    db2 = dy.sum(axis=0)
    da = dy @ W2
    dh = da * gelu_grad(h)
    dW1 = dh.T @ xh
    db1 = dh.sum(axis=0)
    dx = dy + (dh @ W1) / sd
    return dW1, db1, dW2, db2, dx


def adamw_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01):
    """One AdamW update of parameter ``p`` (returns new p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    p = p * (1.0 - lr * wd) - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v
