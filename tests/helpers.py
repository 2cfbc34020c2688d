"""Shared helpers for the GPU parity tests (oracle side + CUDA side)."""
from __future__ import annotations

import math

import numpy as np

from oracle import melt_oracle as O

U32 = 2.0 ** -24      # unit roundoff of float32
LOGF_ABS = 2.0 ** -21  # __logf: absolute error <= 2^-21.41 on [0.5, 2]
LOGF_REL = 4 * 2.0 ** -23  # ... and <= 3 ulp of the result elsewhere


def gpu_features(fe, clips, offsets=None, stream=None):
    """Run a Frontend on host clips (packed at 4-float alignment) -> float64 [sum T, n_out]."""
    import torch
    from paper_2606_01009_gb300 import inputs as G
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    out = fe(wave, pk.offsets if offsets is None else offsets, pk.lengths, stream=stream)
    fe.sync(stream)
    return out.cpu().numpy().astype(np.float64)


def oracle_features(spec, clips, rounded=None):
    outs = []
    for c in clips:
        outs.append(O.melt_clip(c, spec) if rounded is None else O.melt_clip_rounded(c, spec, rounded))
    return np.concatenate(outs) if outs else np.zeros((0, spec.n_out))


def frame_abs_sums(spec, clips):
    """Per frame: sum_n |w[n] x_t[n]|, the scale of the projection's rounding error."""
    rows = []
    for c in clips:
        X = O.frame_signal(c, spec.n_fft, spec.hop)
        rows.append(np.abs(X) @ np.abs(spec.window))
    return np.concatenate(rows) if rows else np.zeros(0)


def log_error_bound(spec, clips, rel_sum_err):
    """Elementwise bound on |GPU log(S+eps) - oracle| given |dR|,|dI| <= rel_sum_err * sum|w x|.

    With E = rel_sum_err * sum_n |w x_t[n]| and S = R^2 + I^2:
        |dS| <= 2 (|R| + |I|) E + 2 E^2 + float32 rounding of S itself,
        |d log(S + eps)| <= |dS| / (S + eps - |dS|)  (or unbounded when |dS| >= S + eps),
    plus the log's own error.
    """
    Rs, Is = [], []
    for c in clips:
        R, I = O.melt_components(c, spec)
        Rs.append(R)
        Is.append(I)
    R = np.concatenate(Rs)
    I = np.concatenate(Is)
    E = rel_sum_err * frame_abs_sums(spec, clips)[:, None]
    S = R * R + I * I
    dS = 2 * (np.abs(R) + np.abs(I)) * E + 2 * E * E + 4 * U32 * S
    den = S + spec.eps - dS
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.where(den > 0, dS / np.maximum(den, 1e-300), np.inf)
    return b + LOGF_ABS + LOGF_REL * np.abs(np.log(S + spec.eps))


def fp32_sum_error(n_terms: int) -> float:
    """Worst-case relative error of an n-term FP32 dot product with FP32-rounded weights."""
    g = (n_terms + 2) * U32
    return g / (1 - g)


def db_report(got, ref, depths=(60.0, 100.0)):
    out = {}
    mx, rms = O.err_db(got, ref)
    out["all"] = (mx, rms)
    for d in depths:
        m = O.within_db_of_frame_max(ref, d)
        out[f"within_{int(d)}dB"] = O.err_db(got, ref, m)
    return out


def rounded_components(spec, clips, precision):
    """(R, I, ER, EI) of the rounded-operand form: the exact (float64) projection of the
    operands each reduced-precision kernel multiplies, plus the sum of |products| per
    output (the scale of any FP32 accumulation error)."""
    Rs, Is, ERs, EIs = [], [], [], []
    W = np.concatenate([spec.Wr, spec.Wi])
    M = spec.n_mels
    for c in clips:
        X = O.frame_signal(c, spec.n_fft, spec.hop)
        if precision == "bf16":
            Xq, Wq = O.round_bf16(X), O.round_bf16(W)
            Y = Xq @ Wq.T
            E = np.abs(Xq) @ np.abs(Wq).T
        elif precision == "bf16x3":
            xh, xl = O.split_bf16(X)
            wh, wl = O.split_bf16(W)
            Y = xh @ wh.T + xh @ wl.T + xl @ wh.T
            E = np.abs(xh) @ np.abs(wh).T + np.abs(xh) @ np.abs(wl).T + np.abs(xl) @ np.abs(wh).T
        elif precision == "fp8":
            Xs = X.astype(np.float32)
            amax = np.max(np.abs(Xs), axis=1) if Xs.size else np.zeros(0, np.float32)
            pos = amax > 0
            inv = np.ones_like(amax)
            inv[pos] = (np.float32(448.0) / amax[pos]).astype(np.float32)
            st = np.ones_like(amax)
            st[pos] = (amax[pos] / np.float32(448.0)).astype(np.float32)
            Aq = O.round_e4m3((Xs * inv[:, None]).astype(np.float32))
            Bq = O.round_e4m3(W * 448.0)
            sc = (st.astype(np.float64) / 448.0)[:, None]
            Y = (Aq @ Bq.T) * sc
            E = (np.abs(Aq) @ np.abs(Bq).T) * sc
        else:
            raise ValueError(precision)
        Rs.append(Y[:, :M]); Is.append(Y[:, M:])
        ERs.append(E[:, :M]); EIs.append(E[:, M:])
    cat = lambda L: np.concatenate(L) if L else np.zeros((0, M))
    return cat(Rs), cat(Is), cat(ERs), cat(EIs)


def rounded_log_bound(spec, clips, precision, rel):
    """Elementwise bound on |GPU - rounded-operand oracle| for log(S + eps) when each
    accumulated sum carries at most rel * (sum of |products|) of error."""
    R, I, ER, EI = rounded_components(spec, clips, precision)
    dR, dI = rel * ER, rel * EI
    S = R * R + I * I
    dS = 2 * np.abs(R) * dR + 2 * np.abs(I) * dI + dR * dR + dI * dI + 4 * U32 * S
    den = S + spec.eps - dS
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.where(den > 0, dS / np.maximum(den, 1e-300), np.inf)
    return b + LOGF_ABS + LOGF_REL * np.abs(np.log(S + spec.eps))
