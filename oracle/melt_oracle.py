"""FP64 CPU oracle for the MelT / MFCCT frontend.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA product
path never imports, links or calls it, and this module imports nothing from
the product package: the two share no code.

Everything here is the paper's plain definition written out in float64 with
numpy (a dense matmul serves as the summation step of the projection; there
is no blocking, fusion or reordering beyond the equations).  Citations are to
the paper's Sec. III-A "Matmul-Native Mel Frontends":

    Eq. 1  Mel map            mu(f) = 2595 log10(1 + f/700)
    Eq. 2  inverse Mel map    f_m = 700 (10^(mu_m/2595) - 1)
    Eq. 3  R, I projections   R = sum_n w[n]x_t[n] cos(2 pi f_m n / f_s), I = ... sin
    Eq. 4  energy             S = R^2 + I^2
    Eq. 5  folded basis       W_r = w[n] cos(.), W_i = w[n] sin(.)
    Eq. 6  projection GEMMs   R = X W_r^T, I = X W_i^T
    Eq. 7  matrix energy      S = R o R + I o I
    Eq. 8  MelT               log(S + eps)
    Eq. 9  MFCCT              log(S + eps) D^T, D orthonormal DCT-II [K x M]

Readings where the paper is silent or ambiguous:

* Frequencies: the M analysis frequencies are the M interior points of M+2
  Mel-uniform points on [f_min, f_max] (the centres of an HTK triangular
  filterbank, whose two edge points are not centres).
* Window: Hann of length N, periodic (denominator N) by default, symmetric
  (denominator N-1) on request (Sec. III-A calls it symmetric; the workloads
  use periodic).
* Framing: no centring or padding; T = floor((L - N)/H) + 1 frames, 0 if
  L < N; frame t holds samples tH .. tH+N-1; the phase origin n = 0 is the
  frame start.
* Centred framing (an option beyond the paper, as in frontends built on a
  centred STFT): the clip is first padded with N/2 samples of reflection at
  both ends (no repeated edge sample), then framed as above, so frame t is
  centred on sample tH and there are floor(L/H) + 1 frames for even N.
* eps is additive (Eq. 8 as written), natural log.
* No normalisation of the basis (Eq. 5 has none).
* DCT-II: D[k, m] = sqrt((2 - [k = 0]) / M) cos(pi k (2m + 1) / (2M)).
"""
from __future__ import annotations

import math

import numpy as np

NAT_TO_DB = 10.0 / math.log(10.0)


# --------------------------------------------------------------------------
# Eq. 1, Eq. 2: Mel map and analysis frequencies
# --------------------------------------------------------------------------
def mel_htk(f):
    """Eq. 1: mu(f) = 2595 log10(1 + f/700)."""
    return 2595.0 * np.log10(1.0 + np.asarray(f, dtype=np.float64) / 700.0)


def mel_htk_inv(mu):
    """Eq. 2: f = 700 (10^(mu/2595) - 1)."""
    return 700.0 * (10.0 ** (np.asarray(mu, dtype=np.float64) / 2595.0) - 1.0)


def melt_frequencies(n_mels: int, fmin: float, fmax: float) -> np.ndarray:
    """The M analysis frequencies f_m (Sec. III-A, Eq. 1-2).

    M+2 points uniform on the Mel scale from mu(fmin) to mu(fmax); the M
    interior ones are the triangle centres and become the analysis bins.
    """
    lo, hi = mel_htk(fmin), mel_htk(fmax)
    mu = lo + (hi - lo) * np.arange(1, n_mels + 1, dtype=np.float64) / (n_mels + 1)
    return mel_htk_inv(mu)


# --------------------------------------------------------------------------
# Window and framing
# --------------------------------------------------------------------------
def hann(n: int, periodic: bool = True) -> np.ndarray:
    """Hann window w[n] = 0.5 - 0.5 cos(2 pi n / D), D = N (periodic) or N-1."""
    d = float(n if periodic else n - 1)
    k = np.arange(n, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * math.pi * k / d)


def num_frames(length: int, n_fft: int, hop: int) -> int:
    """Frames of a clip: floor((L - N)/H) + 1, or 0 when L < N."""
    if length < n_fft:
        return 0
    return (length - n_fft) // hop + 1


def frame_signal(x: np.ndarray, n_fft: int, hop: int, frames=None) -> np.ndarray:
    """Stack frames X[t, n] = x[tH + n] (Sec. III-A, the matrix X of Eq. 6)."""
    x = np.asarray(x, dtype=np.float64)
    T = num_frames(x.shape[0], n_fft, hop)
    idx = np.arange(T) if frames is None else np.asarray(frames, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= T):
        raise IndexError("frame index out of range")
    return x[idx[:, None] * hop + np.arange(n_fft)[None, :]] if idx.size else np.zeros((0, n_fft))


def reflect_pad(x: np.ndarray, pad: int) -> np.ndarray:
    """x padded with ``pad`` samples of reflection at both ends: y[i] = x[|i - pad|]
    on the left, mirrored about the last sample on the right (no repeated edge
    sample).  Needs pad < len(x)."""
    x = np.asarray(x, dtype=np.float64)
    if pad >= x.shape[0]:
        raise ValueError("reflection needs pad < len(x)")
    return np.pad(x, (pad, pad), mode="reflect")


# --------------------------------------------------------------------------
# Eq. 5: window-folded basis; Eq. 6-8: projection, energy, log
# --------------------------------------------------------------------------
def dmp_weights(freqs, n_fft: int, sr: float, window: np.ndarray):
    """Eq. 5: W_r[m, n] = w[n] cos(2 pi f_m n / f_s), W_i[m, n] = w[n] sin(...)."""
    f = np.asarray(freqs, dtype=np.float64)[:, None]
    n = np.arange(n_fft, dtype=np.float64)[None, :]
    theta = 2.0 * math.pi * f * n / sr
    w = np.asarray(window, dtype=np.float64)[None, :]
    return w * np.cos(theta), w * np.sin(theta)


def dmp_projection(X: np.ndarray, Wr: np.ndarray, Wi: np.ndarray):
    """Eq. 6: R = X W_r^T, I = X W_i^T."""
    return X @ Wr.T, X @ Wi.T


def dmp_energy(R: np.ndarray, I: np.ndarray) -> np.ndarray:
    """Eq. 4 / Eq. 7: S = R o R + I o I."""
    return R * R + I * I


def melt_log(S: np.ndarray, eps: float) -> np.ndarray:
    """Eq. 8: log(S + eps), natural log, additive eps."""
    return np.log(S + eps)


def dct2_ortho(n_out: int, n_in: int) -> np.ndarray:
    """Orthonormal DCT-II matrix D [K x M] (Eq. 9): first K rows."""
    k = np.arange(n_out, dtype=np.float64)[:, None]
    m = np.arange(n_in, dtype=np.float64)[None, :]
    D = np.cos(math.pi * k * (2.0 * m + 1.0) / (2.0 * n_in)) * math.sqrt(2.0 / n_in)
    D[0, :] *= math.sqrt(0.5)
    return D


def mfcct(logmel: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Eq. 9: C = log(S + eps) D^T."""
    return logmel @ D.T


class MelTSpec:
    """Parameters of one MelT configuration (same meaning as the C ABI)."""

    def __init__(self, sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0,
                 periodic=True, eps=1e-10, n_mfcc=0, freqs=None):
        self.sr, self.n_fft, self.hop, self.n_mels = float(sr), int(n_fft), int(hop), int(n_mels)
        self.fmin, self.fmax, self.periodic = float(fmin), float(fmax), bool(periodic)
        self.eps, self.n_mfcc = float(eps), int(n_mfcc)
        self.freqs = (melt_frequencies(self.n_mels, self.fmin, self.fmax) if freqs is None
                      else np.asarray(freqs, dtype=np.float64))
        self.n_mels = int(self.freqs.shape[0])
        self.window = hann(self.n_fft, self.periodic)
        self.Wr, self.Wi = dmp_weights(self.freqs, self.n_fft, self.sr, self.window)
        self.D = dct2_ortho(self.n_mfcc, self.n_mels) if self.n_mfcc else None

    @property
    def n_out(self) -> int:
        return self.n_mfcc if self.n_mfcc else self.n_mels


def melt_components(x, spec: MelTSpec, frames=None):
    """(R, I) of every (or the selected) frame of one clip (Eq. 3 via Eq. 6)."""
    X = frame_signal(x, spec.n_fft, spec.hop, frames)
    return dmp_projection(X, spec.Wr, spec.Wi)


def melt_clip(x, spec: MelTSpec, frames=None) -> np.ndarray:
    """MelT (Eq. 8) or MFCCT (Eq. 9) features of one clip, float64 [T, n_out]."""
    R, I = melt_components(x, spec, frames)
    out = melt_log(dmp_energy(R, I), spec.eps)
    return mfcct(out, spec.D) if spec.D is not None else out


def melt_clip_centred(x, spec: MelTSpec) -> np.ndarray:
    """The features of one clip with centred framing: reflection padding of N/2
    samples at both ends, then Eq. 8 / Eq. 9 on the padded clip."""
    return melt_clip(reflect_pad(x, spec.n_fft // 2), spec)


def melt_batch(clips, spec: MelTSpec) -> np.ndarray:
    """Clip after clip, frame-major: [sum_b T_b, n_out]."""
    outs = [melt_clip(c, spec) for c in clips]
    return np.concatenate(outs, axis=0) if outs else np.zeros((0, spec.n_out))


# --------------------------------------------------------------------------
# Operand rounding (reading of the reduced-precision forms; the paper itself
# runs FP32/TF32 only).  Each function returns the exact float64 value of the
# rounded number, so the products below are computed without further error.
# --------------------------------------------------------------------------
def round_bf16(a) -> np.ndarray:
    """Round to bfloat16, nearest-even, from the exact input value.

    bfloat16 keeps 8 significant bits and float32's exponent range; values
    below the normal range round on the same absolute grid (2^-133 step).
    """
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros_like(a)
    nz = (a != 0) & np.isfinite(a)
    m, e = np.frexp(a[nz])            # a = m 2^e, 0.5 <= |m| < 1
    e = np.maximum(e, -125)           # subnormal grid below 2^-126
    q = np.ldexp(a[nz], 8 - e)        # scale so the kept bits are integral
    out[nz] = np.ldexp(np.round(q), e - 8)   # np.round: half to even
    return out


def split_bf16(a):
    """Two-term bfloat16 split: hi = bf16(a), lo = bf16(a - hi)."""
    a = np.asarray(a, dtype=np.float64)
    hi = round_bf16(a)
    return hi, round_bf16(a - hi)


E4M3_MAX = 448.0


def round_e4m3(a) -> np.ndarray:
    """Round to FP8 e4m3 (OCP 'fn' variant), nearest-even, saturating to +-448.

    e4m3: 4 exponent bits (bias 7), 3 mantissa bits; normals from 2^-6,
    subnormals on a 2^-9 grid; no infinities.
    """
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros_like(a)
    nz = (a != 0) & np.isfinite(a)
    m, e = np.frexp(a[nz])
    e = np.maximum(e, -5)             # 2^-6 = 0.5 * 2^-5 : subnormal grid below it
    q = np.ldexp(a[nz], 4 - e)        # 4 significant bits integral
    out[nz] = np.ldexp(np.round(q), e - 4)
    return np.clip(out, -E4M3_MAX, E4M3_MAX)


def f32(a) -> np.ndarray:
    """Round to float32 and return as float64 (exact)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def fp8_row_exponents(amax) -> np.ndarray:
    """Exponent e_u of each FP8 row scale 2^e_u: the least integer e with
    amax_u * 2^-e <= 448 (the largest e4m3 value), so that the scaled row
    fills (224, 448]; at least -127 (the smallest UE8M0 scale), and -127 for
    an all-zero row.  amax_u is a float32 magnitude."""
    a = np.asarray(amax, dtype=np.float64)
    e = np.full(a.shape, -127, dtype=np.int64)
    pos = a > 0
    _, E = np.frexp(a[pos])                       # a = m 2^E, 0.5 <= m < 1
    cand = E.astype(np.int64) - 9                 # a 2^-cand = m 2^9 in [256, 512)
    cand += (np.ldexp(a[pos], -cand) > E4M3_MAX).astype(np.int64)
    e[pos] = np.maximum(cand, -127)
    return e


def fp8_row_quantised(x, hop: int) -> np.ndarray:
    """The sample values the FP8 form multiplies, for one clip.

    The clip is cut into polyphase rows of H samples from its first sample
    (row u = samples uH .. uH+H-1, the last one cut at the clip end); row u
    gets the scale 2^e_u of ``fp8_row_exponents`` from max |x| over its
    samples, its samples are rounded to e4m3 after division by 2^e_u, and
    the result is multiplied back.  Returned as float64 (exact values)."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    L = x.shape[0]
    U = -(-L // hop)
    rows = np.zeros(U * hop)
    rows[:L] = x
    rows = rows.reshape(U, hop)
    e = fp8_row_exponents(np.max(np.abs(rows), axis=1) if U else np.zeros(0))
    q = np.ldexp(round_e4m3(np.ldexp(rows, -e[:, None])), e[:, None])
    return q.reshape(-1)[:L]


def fp8_frame_quantised(X) -> np.ndarray:
    """Per-frame alternative of the FP8 operand rounding (the frame-level
    amax scaling named with the precision sweep): each frame row of X gets
    the power-of-two scale of ``fp8_row_exponents`` from max |x| over the
    whole frame.  Kept to compare the two scalings; the FP8 form itself
    scales polyphase rows (``fp8_row_quantised``)."""
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    e = fp8_row_exponents(np.max(np.abs(X), axis=1) if X.size else np.zeros(X.shape[0]))
    return np.ldexp(round_e4m3(np.ldexp(X, -e[:, None])), e[:, None])


FP8_BASIS_EXP = 8   # the e4m3 basis holds W * 2^8 (|W| <= 1, so at most 256 <= 448)


def fp8_basis_quantised(W) -> np.ndarray:
    """The basis values the FP8 form multiplies: e4m3(W 2^8) 2^-8 (exact)."""
    return np.ldexp(round_e4m3(np.ldexp(np.asarray(W, np.float64), FP8_BASIS_EXP)), -FP8_BASIS_EXP)


def melt_clip_rounded(x, spec: MelTSpec, precision: str, frames=None) -> np.ndarray:
    """MelT with the GEMM operands rounded as each reduced-precision form does.

    The products and sums are then exact (float64); only operand rounding
    differs from ``melt_clip``.  Forms:

    * ``bf16``:   A = bf16(x), B = bf16(W).
    * ``bf16x3``: x = xh + xl, W = Wh + Wl (two-term bf16 splits), and the
      three products xh Wh + xh Wl + xl Wh (the xl Wl term is dropped).
    * ``fp8``:    every polyphase row of H samples (from the clip's first
      sample) has its own power-of-two scale 2^e_u from its max |x|
      (``fp8_row_quantised``); the basis is e4m3(W 2^8) 2^-8
      (``fp8_basis_quantised``).  A frame's samples thus carry the scales of
      the J rows they come from.
    * ``fp32``:   B = float32(W) (A is already float32).
    """
    W = np.concatenate([spec.Wr, spec.Wi], axis=0)
    M = spec.n_mels
    if precision == "fp8":
        X = frame_signal(fp8_row_quantised(x, spec.hop), spec.n_fft, spec.hop, frames)
        Y = X @ fp8_basis_quantised(W).T
    elif precision == "fp8_frame":
        X = fp8_frame_quantised(frame_signal(x, spec.n_fft, spec.hop, frames))
        Y = X @ fp8_basis_quantised(W).T
    else:
        X = frame_signal(x, spec.n_fft, spec.hop, frames)
        if precision == "fp32":
            Y = X @ f32(W).T
        elif precision == "bf16":
            Y = round_bf16(X) @ round_bf16(W).T
        elif precision == "bf16x3":
            xh, xl = split_bf16(X)
            wh, wl = split_bf16(W)
            Y = xh @ wh.T + xh @ wl.T + xl @ wh.T
        else:
            raise ValueError(precision)
    S = dmp_energy(Y[:, :M], Y[:, M:])
    out = melt_log(S, spec.eps)
    return mfcct(out, spec.D) if spec.D is not None else out


# --------------------------------------------------------------------------
# Conventional comparator: STFT (direct DFT) + triangular Mel filterbank
# (Sec. IV-A "Comparators and Controls": matched STFT+Mel pipeline).
# --------------------------------------------------------------------------
def dft_power(Xw: np.ndarray, n_fft: int) -> np.ndarray:
    """|DFT|^2 of windowed frames at f_k = k sr / N, k = 0..N/2 (direct sums)."""
    k = np.arange(n_fft // 2 + 1, dtype=np.float64)[:, None]
    n = np.arange(n_fft, dtype=np.float64)[None, :]
    ang = 2.0 * math.pi * k * n / n_fft
    re = Xw @ np.cos(ang).T
    im = Xw @ np.sin(ang).T
    return re * re + im * im


def mel_slaney(f):
    """Slaney Mel scale: linear (200/3 Hz per mel) below 1 kHz, log above."""
    f = np.asarray(f, dtype=np.float64)
    lin = f / (200.0 / 3.0)
    logstep = math.log(6.4) / 27.0
    with np.errstate(divide="ignore"):
        lg = 15.0 + np.log(np.maximum(f, 1e-300) / 1000.0) / logstep
    return np.where(f >= 1000.0, lg, lin)


def mel_slaney_inv(m):
    m = np.asarray(m, dtype=np.float64)
    logstep = math.log(6.4) / 27.0
    return np.where(m >= 15.0, 1000.0 * np.exp(logstep * (m - 15.0)), m * (200.0 / 3.0))


def triangular_filterbank(n_mels: int, n_fft: int, sr: float, fmin: float, fmax: float,
                          scale: str = "htk") -> np.ndarray:
    """Triangular Mel filterbank [M x (N/2+1)] on the FFT bin frequencies.

    Edges are M+2 points uniform on the chosen Mel scale; filter m rises from
    edge m to edge m+1 and falls to edge m+2.  ``htk``: HTK scale (Eq. 1),
    peak-1 triangles.  ``slaney``: Slaney scale with area normalisation
    2 / (f_{m+2} - f_m).
    """
    fk = np.arange(n_fft // 2 + 1, dtype=np.float64) * sr / n_fft
    if scale == "htk":
        edges = mel_htk_inv(np.linspace(mel_htk(fmin), mel_htk(fmax), n_mels + 2))
    elif scale == "slaney":
        edges = mel_slaney_inv(np.linspace(mel_slaney(fmin), mel_slaney(fmax), n_mels + 2))
    else:
        raise ValueError(scale)
    F = np.zeros((n_mels, fk.shape[0]))
    for m in range(n_mels):
        lo, c, hi = edges[m], edges[m + 1], edges[m + 2]
        rise = (fk - lo) / (c - lo)
        fall = (hi - fk) / (hi - c)
        F[m] = np.maximum(0.0, np.minimum(rise, fall))
        if scale == "slaney":
            F[m] *= 2.0 / (hi - lo)
    return F


def stft_mel_clip(x, spec: MelTSpec, scale: str = "htk", frames=None) -> np.ndarray:
    """Conventional log-Mel: window, |DFT|^2, triangular Mel, log(. + eps)."""
    X = frame_signal(x, spec.n_fft, spec.hop, frames) * spec.window[None, :]
    P = dft_power(X, spec.n_fft)
    F = triangular_filterbank(spec.n_mels, spec.n_fft, spec.sr, spec.fmin, spec.fmax, scale)
    return np.log(P @ F.T + spec.eps)


def stft_mel_clip_rounded(x, spec: MelTSpec, scale: str = "htk", precision: str = "fp64") -> np.ndarray:
    """The conventional pipeline with the GEMM operands rounded as the fused
    STFT+Mel comparator does: the DFT is the projection of the frames onto the
    window-folded cos/sin rows (Eq. 5) at the uniform frequencies f_k = k sr/N,
    k = 0..N/2, with the operand rounding of ``melt_clip_rounded``; then
    |X_k|^2, the triangular Mel filterbank and log(. + eps), exactly.  With
    precision "fp64" this is ``stft_mel_clip``."""
    fk = np.arange(spec.n_fft // 2 + 1, dtype=np.float64) * spec.sr / spec.n_fft
    Wr, Wi = dmp_weights(fk, spec.n_fft, spec.sr, spec.window)
    W = np.concatenate([Wr, Wi], axis=0)
    K = fk.shape[0]
    X = frame_signal(x, spec.n_fft, spec.hop)
    if precision == "fp64":
        Y = X @ W.T
    elif precision == "fp32":
        Y = X @ f32(W).T
    elif precision == "bf16":
        Y = round_bf16(X) @ round_bf16(W).T
    elif precision == "bf16x3":
        xh, xl = split_bf16(X)
        wh, wl = split_bf16(W)
        Y = xh @ wh.T + xh @ wl.T + xl @ wh.T
    else:
        raise ValueError(precision)
    P = dmp_energy(Y[:, :K], Y[:, K:])
    F = triangular_filterbank(spec.n_mels, spec.n_fft, spec.sr, spec.fmin, spec.fmax, scale)
    return np.log(P @ F.T + spec.eps)


# --------------------------------------------------------------------------
# Metrics (Sec. IV-F, Table "equiv_features"): cosine, Lin's CCC, RMSE in dB
# --------------------------------------------------------------------------
def nat_to_db(v):
    """Log-power difference in nats -> dB: 10/ln(10) per nat."""
    return np.asarray(v, dtype=np.float64) * NAT_TO_DB


def err_db(test, ref, mask=None):
    """(max, rms) of |test - ref| in dB over the (masked) entries."""
    d = np.abs(np.asarray(test, np.float64) - np.asarray(ref, np.float64))
    if mask is not None:
        d = d[mask]
    if d.size == 0:
        return 0.0, 0.0
    return float(nat_to_db(d.max())), float(nat_to_db(math.sqrt(float(np.mean(d * d)))))


def within_db_of_frame_max(logmel, depth_db: float) -> np.ndarray:
    """Mask of bins no more than ``depth_db`` below their frame's largest bin."""
    lm = np.asarray(logmel, np.float64)
    top = lm.max(axis=1, keepdims=True)
    return nat_to_db(top - lm) <= depth_db


def mean_row_cosine(A, B) -> float:
    """Mean over frames of the cosine between the two frames' M log values."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    num = np.sum(A * B, axis=1)
    den = np.linalg.norm(A, axis=1) * np.linalg.norm(B, axis=1)
    return float(np.mean(num / den))


def lin_ccc(a, b) -> float:
    """Lin's concordance correlation 2 cov / (var_a + var_b + (mu_a - mu_b)^2)."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    ma, mb = a.mean(), b.mean()
    cov = np.mean((a - ma) * (b - mb))
    return float(2.0 * cov / (a.var() + b.var() + (ma - mb) ** 2))


def rmse_db(A, B) -> float:
    d = np.asarray(A, np.float64) - np.asarray(B, np.float64)
    return float(nat_to_db(math.sqrt(float(np.mean(d * d)))))


def fidelity(pairs):
    """Per-clip means over (test, ref) log-Mel pairs: cosine, CCC, RMSE dB."""
    cos = [mean_row_cosine(a, b) for a, b in pairs]
    ccc = [lin_ccc(a, b) for a, b in pairs]
    rm = [rmse_db(a, b) for a, b in pairs]
    return {"cosine": float(np.mean(cos)), "ccc": float(np.mean(ccc)), "rmse_db": float(np.mean(rm))}


# --------------------------------------------------------------------------
# Roofline convention used with the paper's arithmetic-intensity figure
# (Sec. V, Fig. "roofline": MelT ~57 FLOP/B).
# --------------------------------------------------------------------------
def gemm_flops_per_frame(n_fft: int, n_mels: int) -> int:
    """2 N (2M): one multiply-add per sample per basis row."""
    return 2 * n_fft * 2 * n_mels


def materialised_bytes_per_frame(n_fft: int, n_mels: int) -> int:
    """FP32 frame read (4N) + FP32 R|I write (4 * 2M) when X is materialised."""
    return 4 * n_fft + 4 * 2 * n_mels
