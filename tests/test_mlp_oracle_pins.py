"""Pins of the FP64 correction-MLP oracle: textbook values, finite
differences, the closed form of AdamW's first step, and learnability of the
per-band affine map the paper says separates MelT from STFT+Mel."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as P


def test_gelu_textbook_values():
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429, Phi(-1) = 1 - Phi(1)
    assert P.gelu(1.0) == pytest.approx(0.8413447460685429, rel=1e-14)
    assert P.gelu(-1.0) == pytest.approx(-(1 - 0.8413447460685429), rel=1e-13)
    assert P.gelu(0.0) == 0.0
    h = np.linspace(-6, 6, 241)
    fd = (P.gelu(h + 1e-6) - P.gelu(h - 1e-6)) / 2e-6
    np.testing.assert_allclose(P.gelu_grad(h), fd, atol=1e-8)


def _setup(seed=0, n=37, m=6, hd=11):
    g = np.random.default_rng(seed)
    x = g.standard_normal((n, m)) * 3 - 5
    tgt = x * g.uniform(0.5, 1.5, m) + g.uniform(-2, 2, m)
    params = [g.standard_normal((hd, m)) * 0.3, g.standard_normal(hd) * 0.1,
              g.standard_normal((m, hd)) * 0.3, g.standard_normal(m) * 0.1]
    mu, sd = P.band_stats(x)
    return x, tgt, params, mu, sd


def test_backward_matches_central_differences():
    x, tgt, params, mu, sd = _setup()
    y, cache = P.forward(params, x, mu, sd)
    grads = P.backward(params, cache, y, tgt, sd)
    h = 1e-6
    for pi in range(4):
        p = params[pi]
        flat = p.reshape(-1)
        for idx in np.random.default_rng(pi).choice(flat.size, min(flat.size, 12), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = P.loss(P.forward(params, x, mu, sd)[0], tgt)
            flat[idx] = old - h
            lm = P.loss(P.forward(params, x, mu, sd)[0], tgt)
            flat[idx] = old
            assert grads[pi].reshape(-1)[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
    # dx too
    dx = grads[4]
    for (i, j) in [(0, 0), (5, 3), (36, 5)]:
        xp = x.copy(); xp[i, j] += h
        xm = x.copy(); xm[i, j] -= h
        fd = (P.loss(P.forward(params, xp, mu, sd)[0], tgt) - P.loss(P.forward(params, xm, mu, sd)[0], tgt)) / (2 * h)
        assert dx[i, j] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adamw_first_step_closed_form():
    # t = 1: mhat = g, vhat = g^2, so p1 = p0 (1 - lr wd) - lr g / (|g| + eps)
    p0 = np.array([0.5, -1.0, 2.0, 0.0])
    g = np.array([0.1, -3.0, 1e-12, 2.0])
    p1, m, v = P.adamw_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=1e-3, wd=0.01, eps=1e-8)
    np.testing.assert_allclose(p1, p0 * (1 - 1e-5) - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_training_learns_per_band_affine_map():
    x, tgt, params, mu, sd = _setup(n=512, m=6, hd=32)
    params = [p.copy() for p in params]
    state = [(np.zeros_like(p), np.zeros_like(p)) for p in params]
    l0 = P.loss(P.forward(params, x, mu, sd)[0], tgt)
    for t in range(1, 1501):
        y, cache = P.forward(params, x, mu, sd)
        grads = P.backward(params, cache, y, tgt, sd)
        for i in range(4):
            params[i], m, v = P.adamw_step(params[i], grads[i], state[i][0], state[i][1], t, lr=1e-2)
            state[i] = (m, v)
    l1 = P.loss(P.forward(params, x, mu, sd)[0], tgt)
    assert l1 < 0.05 * l0
