"""Host-side check of the fused epilogue's GELU constants (no GPU needed).

The CTA-pair kernel's fused correction MLP evaluates GELU(h) = h Phi(h) as
max(h, 0) - |h| Q(|h|), the normal tail Q(t) = 2^(S(t) - t^2 log2(e) / 2),
with S a polynomial in u = 0.4 min(t, 5) - 1.  This test reads the
polynomial's coefficients and the exponent constant out of the kernel source,
replays the evaluation in float32 (each fused multiply-add as one float64
operation rounded to float32; the base-2 exponential exact, then rounded),
and holds the result to the bound the kernel's comment and include/melt_diag.h
state against the exact function: relative error <= 2e-5 for |h| <= 5,
absolute error <= 3e-6 everywhere.  The GPU test
(tests/test_gpu_mlp.py::test_fused_gelu_error_bound) checks the device's own
evaluation against the same bound.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNEL = os.path.join(ROOT, "paper_2606_01009_gb300", "csrc", "melt_tc2_kernel.cuh")
_NUM = r"(-?\d+(?:\.\d*)?(?:e[-+]?\d+)?)f"


def _gelu_constants():
    src = open(KERNEL).read()
    m = re.search(r"float gelu_poly\(float h\) \{(.*?)\n\}", src, re.S)
    assert m, "gelu_poly not found"
    body = m.group(1)
    first = re.search(r"float r = " + _NUM + ";", body)
    rest = re.findall(r"r = fmaf\(r, u, " + _NUM + r"\);", body)
    expo = re.search(r"t \* " + _NUM + r", t, r\)", body)
    clamp = re.search(r"fmaf\(" + _NUM + r", fminf\(t, " + r"(\d+(?:\.\d*)?)f\), " + _NUM + r"\)", body)
    assert first and rest and expo and clamp, "unexpected gelu_poly form"
    coeffs = [float(first.group(1))] + [float(x) for x in rest]
    return (np.float32(clamp.group(1)), np.float32(clamp.group(2)), np.float32(clamp.group(3)),
            [np.float32(c) for c in coeffs], np.float32(expo.group(1)))


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + np.float64(c) if np.isscalar(c)
            else a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _gelu_replay(h):
    scale, tmax, shift, coeffs, expo = _gelu_constants()
    h = h.astype(np.float32)
    t = np.abs(h)
    u = _fma32(np.full_like(t, scale), np.minimum(t, tmax), shift)
    r = np.full_like(u, coeffs[0])
    for c in coeffs[1:]:
        r = _fma32(r, u, c)
    p = _fma32((t * expo).astype(np.float32), t, r)
    q = np.exp2(p.astype(np.float64)).astype(np.float32)
    return _fma32(-t, q, np.maximum(h, np.float32(0))).astype(np.float64)


def test_gelu_polynomial_meets_its_stated_bound():
    from scipy.special import ndtr
    g = np.random.default_rng(5)
    h = np.concatenate([np.linspace(-12, 12, 1_200_001), g.standard_normal(100000) * 3,
                        np.array([0.0, 1e-30, -1e-30, 5.0, -5.0, 4.9999, -5.0001, 30.0, -30.0])]).astype(np.float32)
    got = _gelu_replay(h)
    hd = h.astype(np.float64)
    exact = hd * ndtr(hd)
    err = np.abs(got - exact)
    assert err.max() <= 3e-6, float(err.max())
    inner = (np.abs(hd) <= 5) & (exact != 0)
    rel = err[inner] / np.abs(exact[inner])
    assert rel.max() <= 2e-5, float(rel.max())


def test_gelu_polynomial_is_degree_six():
    """The stated operation count (about a dozen) rests on a degree-6 S."""
    _, _, _, coeffs, _ = _gelu_constants()
    assert len(coeffs) == 7


@pytest.mark.parametrize("h", [-3.0, -1.0, -0.25, 0.25, 1.0, 3.0])
def test_gelu_special_values(h):
    """Spot values of h Phi(h), and the odd-part identity GELU(h) - GELU(-h) = h."""
    from scipy.special import ndtr
    a = _gelu_replay(np.array([h], np.float32))[0]
    b = _gelu_replay(np.array([-h], np.float32))[0]
    assert a == pytest.approx(h * ndtr(h), rel=2e-5, abs=3e-6)
    assert a - b == pytest.approx(h, rel=1e-6, abs=1e-6)
