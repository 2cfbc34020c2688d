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


def test_forward_bf16_hand_example():
    """Which values the BF16 evaluation rounds, worked by hand.  mu = (0, 1),
    sd = (1, 0.5); x = (1 + 2^-8, 2).  x-hat = (1 + 2^-8, 2) rounds to
    (1, 2) (a tie goes to the even neighbour 1).  W1 = [[1.5 + 2^-8, 0],
    [0, -0.75]] rounds to [[1.5, 0], [0, -0.75]] (tie, even), b1 = (0, 0.25):
    h = (1.5, -1.25), not rounded.  GELU(1.5) = 1.5 Phi(1.5) = 1.39978920
    rounds to 1.3984375 (179 steps of 2^-7), GELU(-1.25) = -1.25 Phi(-1.25)
    = -0.13206222 rounds to -0.1318359375 (135 steps of 2^-10).  W2 =
    [[2 + 2^-7, 0.5], [0, 1]] rounds to [[2, 0.5], [0, 1]] (tie, even); b2 =
    (0, 0.5) and the residual x are not rounded."""
    phi_15, phi_m125 = 0.9331927987311419, 0.10564977366685535   # standard normal table
    assert P.gelu(1.5) == pytest.approx(1.5 * phi_15, rel=1e-14)
    assert P.gelu(-1.25) == pytest.approx(-1.25 * phi_m125, rel=1e-13)
    W1 = np.array([[1.5 + 2 ** -8, 0.0], [0.0, -0.75]])
    b1 = np.array([0.0, 0.25])
    W2 = np.array([[2.0 + 2 ** -7, 0.5], [0.0, 1.0]])
    b2 = np.array([0.0, 0.5])
    x = np.array([[1.0 + 2 ** -8, 2.0]])
    y, (xh_b, h, a_b, W1_b, W2_b) = P.forward_bf16([W1, b1, W2, b2], x, np.array([0.0, 1.0]), np.array([1.0, 0.5]))
    np.testing.assert_array_equal(xh_b, [[1.0, 2.0]])
    np.testing.assert_array_equal(h, [[1.5, -1.25]])
    np.testing.assert_array_equal(a_b, [[1.3984375, -0.1318359375]])
    np.testing.assert_array_equal(W1_b, [[1.5, 0.0], [0.0, -0.75]])
    np.testing.assert_array_equal(W2_b, [[2.0, 0.5], [0.0, 1.0]])
    y0 = (1.0 + 2 ** -8) + 2.0 * 1.3984375 + 0.5 * -0.1318359375
    y1 = 2.0 + 1.0 * -0.1318359375 + 0.5
    np.testing.assert_array_equal(y, [[y0, y1]])
    assert y0 == 3.73486328125 and y1 == 2.3681640625
