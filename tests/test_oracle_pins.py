"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, a library routine that
computes the same quantity by another route, an invariant of the
mathematics, or a number printed in the paper.  A dropped term, wrong sign,
wrong index or transposed operand anywhere in the oracle fails at least one.
"""
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.signal
import torch

from oracle import melt_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Mel map
def test_mel_map_textbook_points():
    # Eq. 1 at f = 700 Hz is 2595 log10(2); HTK maps 1000 Hz to ~1000 mel.
    assert O.mel_htk(700.0) == pytest.approx(2595.0 * math.log10(2.0), rel=1e-15)
    assert O.mel_htk(1000.0) == pytest.approx(1000.0, abs=0.05)
    assert O.mel_htk(0.0) == 0.0
    f = np.linspace(0.0, 11025.0, 257)
    np.testing.assert_allclose(O.mel_htk_inv(O.mel_htk(f)), f, rtol=1e-12, atol=1e-9)


def test_analysis_frequencies_interior_and_mel_uniform():
    f = O.melt_frequencies(80, 0.0, 8000.0)
    assert f.shape == (80,)
    assert 0.0 < f[0] and f[-1] < 8000.0           # interior points only
    step = (O.mel_htk(8000.0) - O.mel_htk(0.0)) / 81.0
    mu = O.mel_htk(f)
    np.testing.assert_allclose(np.diff(mu), step, rtol=1e-10)
    assert mu[0] == pytest.approx(step, rel=1e-10)


# ------------------------------------------------------------------ window
@pytest.mark.parametrize("n", [8, 400, 1024, 1200])
def test_hann_matches_scipy(n):
    np.testing.assert_allclose(O.hann(n, periodic=True),
                               scipy.signal.get_window("hann", n, fftbins=True), atol=1e-15)
    np.testing.assert_allclose(O.hann(n, periodic=False),
                               scipy.signal.windows.hann(n, sym=True), atol=1e-15)


def test_frame_count_rule():
    # 1 s at 16 kHz with N=400, H=160 gives 98 frames (the 8 x 1 s workload's count)
    assert O.num_frames(16000, 400, 160) == 98
    assert O.num_frames(399, 400, 160) == 0
    assert O.num_frames(400, 400, 160) == 1
    assert O.num_frames(559, 400, 160) == 1
    assert O.num_frames(560, 400, 160) == 2
    assert O.num_frames(480000, 400, 160) == 2998


# ------------------------------------------------------- tone closed form
def _geom(omega, n):
    """G(omega) = sum_{k<n} e^{-i omega k} in closed form."""
    omega = np.asarray(omega, np.float64)
    z = np.exp(-1j * omega)
    near = np.abs(np.angle(z)) < 1e-12
    out = np.where(near, n + 0j, (1 - z ** n) / np.where(near, 1, 1 - z))
    return out


def _hann_dtft(omega, n, periodic):
    d = n if periodic else n - 1
    s = 2 * math.pi / d
    return 0.5 * _geom(omega, n) - 0.25 * _geom(omega - s, n) - 0.25 * _geom(omega + s, n)


@pytest.mark.parametrize("periodic", [True, False])
def test_tone_closed_form_all_bins(periodic):
    sr, N, M = 16000.0, 400, 80
    spec = O.MelTSpec(sr=sr, n_fft=N, hop=160, n_mels=M, periodic=periodic)
    rng = np.random.default_rng(7)
    for m0 in [10, 33, 57, 70]:
        A, phi = 0.37, rng.uniform(0, 2 * math.pi)
        th0 = 2 * math.pi * spec.freqs[m0] / sr
        x = A * np.cos(th0 * np.arange(N) + phi)
        R, I = O.melt_components(x, spec)
        S = O.dmp_energy(R, I)[0]
        th = 2 * math.pi * spec.freqs / sr
        Z = 0.5 * A * (np.exp(1j * phi) * _hann_dtft(th - th0, N, periodic)
                       + np.exp(-1j * phi) * _hann_dtft(th + th0, N, periodic))
        np.testing.assert_allclose(R[0] - 1j * I[0], Z, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(S, np.abs(Z) ** 2, rtol=1e-9, atol=1e-12)
        assert int(np.argmax(S)) == m0


def test_tone_peak_magnitude_at_own_bin():
    # away from DC, |R - iI| at the tone's own bin is ~A/2 * sum(w) = A N / 4
    sr, N = 16000.0, 400
    spec = O.MelTSpec(sr=sr, n_fft=N, hop=160, n_mels=80)
    m0 = 40
    th0 = 2 * math.pi * spec.freqs[m0] / sr
    x = 0.5 * np.cos(th0 * np.arange(N))
    S = O.dmp_energy(*O.melt_components(x, spec))[0]
    assert math.sqrt(S[m0]) == pytest.approx(0.5 * N / 4.0, rel=2e-3)


# ------------------------------------------- uniform-frequency special case
@pytest.mark.parametrize("periodic", [True, False])
def test_uniform_frequencies_equal_rfft(periodic):
    sr, N, H = 16000.0, 400, 160
    freqs = np.arange(N // 2 + 1) * sr / N
    spec = O.MelTSpec(sr=sr, n_fft=N, hop=H, periodic=periodic, freqs=freqs)
    x = np.random.default_rng(3).standard_normal(N + 3 * H)
    R, I = O.melt_components(x, spec)
    X = O.frame_signal(x, N, H) * O.hann(N, periodic)[None, :]
    F = np.fft.rfft(X, axis=1)
    np.testing.assert_allclose(R, F.real, atol=1e-10)
    np.testing.assert_allclose(I, -F.imag, atol=1e-10)
    np.testing.assert_allclose(O.dft_power(X, N), np.abs(F) ** 2, rtol=1e-10, atol=1e-9)


def test_parseval_full_uniform_set():
    sr, N = 16000.0, 256
    spec = O.MelTSpec(sr=sr, n_fft=N, hop=64, freqs=np.arange(N) * sr / N)
    x = np.random.default_rng(5).standard_normal(N + 64)
    S = O.dmp_energy(*O.melt_components(x, spec))
    Xw = O.frame_signal(x, N, 64) * spec.window[None, :]
    np.testing.assert_allclose(S.sum(axis=1), N * np.sum(Xw * Xw, axis=1), rtol=1e-11)


# -------------------------------------------------------------- invariants
def test_linearity_and_scale_law():
    spec = O.MelTSpec()
    g = np.random.default_rng(11)
    x1, x2 = g.standard_normal(4000), g.standard_normal(4000)
    a, b = 0.7, -1.9
    R1, I1 = O.melt_components(x1, spec)
    R2, I2 = O.melt_components(x2, spec)
    R, I = O.melt_components(a * x1 + b * x2, spec)
    np.testing.assert_allclose(R, a * R1 + b * R2, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(I, a * I1 + b * I2, rtol=1e-10, atol=1e-10)
    S1 = O.dmp_energy(R1, I1)
    S = O.dmp_energy(*O.melt_components(3.0 * x1, spec))
    np.testing.assert_allclose(S, 9.0 * S1, rtol=1e-11)


def test_hop_shift():
    spec = O.MelTSpec()
    x = np.random.default_rng(2).standard_normal(6000)
    out = O.melt_clip(x, spec)
    out2 = O.melt_clip(x[spec.hop:], spec)
    np.testing.assert_allclose(out2, out[1:1 + out2.shape[0]], rtol=1e-12, atol=1e-12)
    pre = np.concatenate([np.random.default_rng(3).standard_normal(spec.hop), x])
    out3 = O.melt_clip(pre, spec)
    np.testing.assert_allclose(out3[1:], out[:out3.shape[0] - 1], rtol=1e-12, atol=1e-12)


def test_brute_force_tiny():
    # tiny case summed with Python loops straight from Eq. 3
    sr, N, H = 100.0, 8, 3
    freqs = np.array([7.0, 19.0, 31.5])
    spec = O.MelTSpec(sr=sr, n_fft=N, hop=H, freqs=freqs, periodic=False)
    x = [math.sin(0.3 * k) + 0.1 * k for k in range(N + 2 * H + 1)]
    R, I = O.melt_components(np.array(x), spec)
    assert R.shape == (3, 3)
    for t in range(3):
        for m, f in enumerate(freqs):
            r = i = 0.0
            for n in range(N):
                w = 0.5 - 0.5 * math.cos(2 * math.pi * n / (N - 1))
                r += w * x[t * H + n] * math.cos(2 * math.pi * f * n / sr)
                i += w * x[t * H + n] * math.sin(2 * math.pi * f * n / sr)
            assert R[t, m] == pytest.approx(r, abs=1e-12)
            assert I[t, m] == pytest.approx(i, abs=1e-12)


# -------------------------------------------------------------------- DCT
@pytest.mark.parametrize("K,M", [(40, 80), (40, 128), (13, 40)])
def test_dct_matches_scipy(K, M):
    D = O.dct2_ortho(K, M)
    v = np.random.default_rng(1).standard_normal((5, M))
    np.testing.assert_allclose(v @ D.T, scipy.fft.dct(v, type=2, norm="ortho", axis=1)[:, :K],
                               atol=1e-12)


def test_dct_orthonormal():
    D = O.dct2_ortho(80, 80)
    np.testing.assert_allclose(D @ D.T, np.eye(80), atol=1e-12)


# ----------------------------------------------------- conventional pipeline
def test_slaney_scale_textbook_points():
    assert O.mel_slaney(1000.0) == pytest.approx(15.0)
    assert O.mel_slaney(6400.0) == pytest.approx(42.0)
    assert O.mel_slaney(200.0 / 3.0) == pytest.approx(1.0)
    f = np.linspace(0, 8000, 101)
    np.testing.assert_allclose(O.mel_slaney_inv(O.mel_slaney(f)), f, atol=1e-9)


def test_htk_triangles_partition_of_unity():
    N, sr = 1024, 16000.0
    F = O.triangular_filterbank(40, N, sr, 0.0, 8000.0, "htk")
    edges = O.mel_htk_inv(np.linspace(O.mel_htk(0.0), O.mel_htk(8000.0), 42))
    fk = np.arange(N // 2 + 1) * sr / N
    inside = (fk >= edges[1]) & (fk <= edges[-2])
    np.testing.assert_allclose(F[:, inside].sum(axis=0), 1.0, atol=1e-12)
    assert F.max() <= 1.0 + 1e-12


def test_slaney_triangle_area_is_one():
    N, sr = 4096, 16000.0
    F = O.triangular_filterbank(40, N, sr, 0.0, 8000.0, "slaney")
    # Riemann sum over bin spacing of a unit-area triangle spanning many bins
    np.testing.assert_allclose(F.sum(axis=1) * sr / N, 1.0, rtol=2e-2)


# ----------------------------------------------------------------- metrics
def test_metrics_closed_forms():
    a = np.array([1.0, 2.0, 3.0])
    assert O.lin_ccc(a, a + 1.0) == pytest.approx(4.0 / 7.0)
    A = np.random.default_rng(0).standard_normal((6, 9))
    assert O.mean_row_cosine(A, A) == pytest.approx(1.0)
    assert O.lin_ccc(A, A) == pytest.approx(1.0)
    assert O.rmse_db(A, A) == 0.0


def test_paper_delta_nat_to_db():
    # Sec. IV-F: a 1% f_max retuning gives delta = 0.244 nat = 1.06 dB
    assert O.rmse_db(np.full((3, 4), 0.244), np.zeros((3, 4))) == pytest.approx(1.06, abs=0.005)


def test_paper_arithmetic_intensity():
    # Sec. V, Fig. "roofline": MelT at ~57 FLOP/B for N=400, M=80
    ai = O.gemm_flops_per_frame(400, 80) / O.materialised_bytes_per_frame(400, 80)
    assert round(ai) == 57


# ------------------------------------------------------- operand rounding
def test_bf16_rounding_matches_torch():
    g = np.random.default_rng(4)
    v = np.concatenate([(g.standard_normal(20000) * 10.0 ** g.integers(-30, 30, 20000)).astype(np.float32),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 3e-39, -7e-40],
                                 np.float32)])
    assert v.dtype == np.float32
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_bf16(v.astype(np.float64)), ref)


def test_e4m3_rounding_matches_torch():
    g = np.random.default_rng(5)
    v = (g.uniform(-460, 460, 20000) * 2.0 ** g.integers(-12, 1, 20000)).astype(np.float32)
    v = np.concatenate([v, np.array([0.0, 2 ** -9, 1.5 * 2 ** -9, 2.5 * 2 ** -9, 448.0, -448.0, 17.0,
                                     9.0, 11.0, 2 ** -10], np.float32)])
    v = v[np.abs(v) <= 448.0]
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_e4m3(v.astype(np.float64)), ref)
    assert O.round_e4m3(np.array([1000.0, -470.0]))[0] == 448.0
    assert O.round_e4m3(np.array([1000.0, -470.0]))[1] == -448.0


def test_rounded_forms_reduce_to_library_products():
    spec = O.MelTSpec()
    x = np.random.default_rng(9).standard_normal(3000).astype(np.float32)
    X = O.frame_signal(x, 400, 160)
    W = np.concatenate([spec.Wr, spec.Wi])
    tb = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).to(torch.float64)
    Y = (tb(X) @ tb(W).T).numpy()
    ref = np.log(Y[:, :80] ** 2 + Y[:, 80:] ** 2 + spec.eps)
    np.testing.assert_allclose(O.melt_clip_rounded(x, spec, "bf16"), ref, rtol=1e-12, atol=1e-12)
    # the split form is far closer to FP64 than plain bf16
    exact = O.melt_clip(x, spec)
    e_bf16 = np.abs(O.melt_clip_rounded(x, spec, "bf16") - exact).max()
    e_x3 = np.abs(O.melt_clip_rounded(x, spec, "bf16x3") - exact).max()
    assert e_x3 < e_bf16 / 50.0


def test_fp8_form_power_of_two_scale_invariance():
    # per-frame amax scaling makes x -> 2^k x change the output by exactly 2k ln 2
    spec = O.MelTSpec(eps=0.0)
    x = np.random.default_rng(8).standard_normal(2400).astype(np.float32)
    a = O.melt_clip_rounded(x, spec, "fp8")
    b = O.melt_clip_rounded(x * np.float32(8.0), spec, "fp8")
    np.testing.assert_allclose(b - a, 2 * 3 * math.log(2.0), atol=1e-9)


def test_zero_frame_is_log_eps():
    spec = O.MelTSpec()
    out = O.melt_clip(np.zeros(800), spec)
    np.testing.assert_allclose(out, math.log(spec.eps))
    np.testing.assert_allclose(O.melt_clip_rounded(np.zeros(800, np.float32), spec, "fp8"),
                               math.log(spec.eps))


# -------------------------------------------------------- golden fixtures
def test_golden_paper_figures():
    import json
    with open(os.path.join(GOLDEN, "paper_figures.json")) as f:
        g = json.load(f)
    assert round(O.gemm_flops_per_frame(g["n_fft"], g["n_mels"])
                 / O.materialised_bytes_per_frame(g["n_fft"], g["n_mels"])) == g["ai_melt_flop_per_byte"]
    assert O.rmse_db(np.full(4, g["delta_nat"]), np.zeros(4)) == pytest.approx(g["delta_db"], abs=0.005)


# ------------------------------------------------- centred framing (option)
def test_reflect_pad_hand_example():
    # reflection about the first and the last sample, which are not repeated
    np.testing.assert_array_equal(O.reflect_pad(np.array([1.0, 2, 3, 4, 5]), 2),
                                  [3.0, 2, 1, 2, 3, 4, 5, 4, 3])
    np.testing.assert_array_equal(O.reflect_pad(np.array([7.0, 8]), 1), [8.0, 7, 8, 7])
    with pytest.raises(ValueError):
        O.reflect_pad(np.array([1.0, 2]), 2)


def test_centred_frame_count():
    # floor(L/H) + 1 frames for even N: a centred 30 s clip at 16 kHz, hop 160,
    # has 3001 frames (frontends that keep 3000 drop the last one)
    spec = O.MelTSpec()
    assert O.melt_clip_centred(np.zeros(480000), spec).shape == (3001, 80)
    for L in (201, 400, 1000, 16000, 16159):
        assert O.melt_clip_centred(np.ones(L), spec).shape[0] == L // 160 + 1


def test_centred_impulse_closed_form():
    # an impulse at sample tH sits at the centre n = N/2 of centred frame t,
    # where the periodic Hann window is exactly 1: S = 1 in every band; frames
    # t -+ 1 see it at n = N/2 +- H, so S = w[N/2 +- H]^2 exactly
    spec = O.MelTSpec(eps=0.0)
    t, H, N = 20, 160, 400
    x = np.zeros(8000)
    x[t * H] = 1.0
    with np.errstate(divide="ignore"):  # frames that miss the impulse have S = 0 and eps = 0
        out = O.melt_clip_centred(x, spec)
    np.testing.assert_allclose(out[t], 0.0, atol=1e-12)
    w = O.hann(N, True)
    np.testing.assert_allclose(out[t - 1], 2 * math.log(w[N // 2 + H]), atol=1e-12)
    np.testing.assert_allclose(out[t + 1], 2 * math.log(w[N // 2 - H]), atol=1e-12)


def test_centring_is_a_shift_when_half_frame_is_a_hop():
    # with N = 2H the padding is exactly one hop: centred frame t + 1 is
    # uncentred frame t wherever both are defined
    spec = O.MelTSpec(n_fft=320, hop=160)
    x = np.random.default_rng(12).standard_normal(5000)
    c, u = O.melt_clip_centred(x, spec), O.melt_clip(x, spec)
    np.testing.assert_allclose(c[1:1 + u.shape[0]], u, atol=1e-12)


def test_melt_vs_matched_stft_mel_on_synthetic_audio():
    """MelT against the conventional pipeline with the same DSP specification
    (HTK scale, peak-1 triangles on the same points, n_fft = N; Sec. IV-F
    metrics).  The paper reports cosine 0.9840, CCC 0.9541 and RMSE 6.03 dB on
    LibriSpeech; synthetic audio is a different signal, so the figures are
    printed beside those, held only to loose bounds (parity unpinned)."""
    from paper_2606_01009_gb300 import inputs as G
    spec = O.MelTSpec(fmin=80.0, fmax=7600.0, periodic=False)
    cos, ccc, rms = [], [], []
    for i in range(4):
        x = G.rich_clip(2026, i, 160000)
        a, b = O.melt_clip(x, spec), O.stft_mel_clip(x, spec, "htk")
        cos.append(O.mean_row_cosine(a, b))
        ccc.append(O.lin_ccc(a, b))
        rms.append(O.rmse_db(a, b))
    print(f"MelT vs matched STFT-Mel, synthetic: cosine {np.mean(cos):.4f} CCC {np.mean(ccc):.4f} "
          f"RMSE {np.mean(rms):.2f} dB (paper, LibriSpeech: 0.9840 / 0.9541 / 6.03 dB)")
    assert np.mean(cos) > 0.85 and np.mean(ccc) > 0.7 and np.mean(rms) < 10.0


# ------------------------------------------- conventional pipeline, whole
@pytest.mark.parametrize("scale", ["htk", "slaney"])
def test_stft_mel_matches_rfft_composition(scale):
    """The whole conventional pipeline against the same steps built from
    numpy.fft.rfft: window, |rfft|^2, the (separately pinned) triangular
    filterbank, log(. + eps)."""
    spec = O.MelTSpec(n_mels=40)
    x = np.random.default_rng(21).standard_normal(400 + 7 * 160 + 33)
    X = O.frame_signal(x, 400, 160) * O.hann(400, True)[None, :]
    P = np.abs(np.fft.rfft(X, axis=1)) ** 2
    F = O.triangular_filterbank(40, 400, 16000.0, 0.0, 8000.0, scale)
    np.testing.assert_allclose(O.stft_mel_clip(x, spec, scale), np.log(P @ F.T + spec.eps),
                               rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("scale", ["htk", "slaney"])
def test_stft_mel_bin_centred_tone_closed_form(scale):
    """A cosine at FFT bin k0 through the periodic Hann window: |X[k0]|^2 =
    (A N / 4)^2, |X[k0 +- 1]|^2 = (A N / 8)^2, every other bin 0.  So band m
    holds exactly F[m, k0-1] (AN/8)^2 + F[m, k0] (AN/4)^2 + F[m, k0+1] (AN/8)^2.
    A dropped window, magnitude instead of power, or a shifted bin grid fails."""
    N, H, sr, A, k0 = 400, 160, 16000.0, 0.3, 50          # 2000 Hz
    spec = O.MelTSpec(n_fft=N, hop=H, n_mels=40)
    n = np.arange(N + 2 * H)
    x = A * np.cos(2 * math.pi * k0 * n / N)
    F = O.triangular_filterbank(40, N, sr, 0.0, 8000.0, scale)
    band = (F[:, k0 - 1] + F[:, k0 + 1]) * (A * N / 8) ** 2 + F[:, k0] * (A * N / 4) ** 2
    out = O.stft_mel_clip(x, spec, scale)
    assert out.shape == (3, 40)
    for t in range(3):   # the tone's phase moves with t; its power does not
        np.testing.assert_allclose(out[t], np.log(band + spec.eps), atol=1e-8)
    assert np.count_nonzero(band) >= 1


# ----------------------------------------------------------- FP8 form
def test_fp8_row_exponent_is_least_power_of_two():
    """e_u is the least integer e with amax 2^-e <= 448 (brute force), clamped
    at -127, on random float32 magnitudes and the edges of the rule."""
    g = np.random.default_rng(31)
    a = (g.uniform(0.5, 2.0, 4000) * 2.0 ** g.integers(-140, 120, 4000)).astype(np.float32)
    edge = np.array([1.75, np.nextafter(np.float32(1.75), np.float32(2)), 1.0, 448.0, 449.0, 3.5,
                     2.0 ** -126, 2.0 ** -130, 1e-45, 3.0e38], np.float32)
    a = np.concatenate([a, edge]).astype(np.float64)
    e = O.fp8_row_exponents(a)
    for v, ev in zip(a, e):
        best = next(k for k in range(-200, 200) if math.ldexp(v, -k) <= 448.0)
        assert ev == max(best, -127), (v, ev, best)
    assert O.fp8_row_exponents(np.array([0.0]))[0] == -127
    assert O.fp8_row_exponents(np.array([1.75]))[0] == -8          # 1.75 * 2^8 = 448
    assert O.fp8_row_exponents(np.array([1.7500001]))[0] == -7


def test_fp8_rows_match_torch_e4m3_cast():
    """Per-row scaling, then torch's float8_e4m3fn cast of float32(x 2^-e_u),
    then 2^e_u back, equals the oracle's quantised samples."""
    g = np.random.default_rng(32)
    H = 160
    x = (g.standard_normal(37 * H + 55) * 10.0 ** g.uniform(-4, 1)).astype(np.float32)
    x[5 * H:6 * H] = 0.0                                  # an all-zero row
    x[9 * H:10 * H] *= np.float32(1e-30)                   # a row of float32 subnormal / tiny values
    q = O.fp8_row_quantised(x, H)
    rows = np.zeros(38 * H, np.float64)
    rows[:x.size] = x
    rows = rows.reshape(38, H)
    e = O.fp8_row_exponents(np.max(np.abs(rows), axis=1))
    scaled = torch.from_numpy(np.ldexp(rows, -e[:, None]).astype(np.float32))
    ref = np.ldexp(scaled.to(torch.float8_e4m3fn).to(torch.float64).numpy(), e[:, None]).reshape(-1)[:x.size]
    np.testing.assert_array_equal(q, ref)


def test_fp8_form_hand_example():
    """Two rows of H = 4 samples worked by hand.  Row [1, 2, 3, 4]: amax 4,
    e = -6 (4 * 64 = 256 <= 448, 512 is not), every value exact in e4m3.
    Row [0.1, 0.2, 0.3, 0.45]: amax 0.45, e = -9 (0.45 * 512 = 230.4; 460.8
    is too large); scaled 51.2, 102.4, 153.6, 230.4 round to 52, 104, 160,
    224 (e4m3 steps 4, 8, 16, 16), i.e. 0.1015625, 0.203125, 0.3125, 0.4375."""
    x = np.array([1, 2, 3, 4, 0.1, 0.2, 0.3, 0.45], np.float32)
    q = O.fp8_row_quantised(x, 4)
    np.testing.assert_array_equal(q, [1, 2, 3, 4, 0.1015625, 0.203125, 0.3125, 0.4375])
    # the basis: W 2^8 in e4m3, then 2^-8: 0.3 -> 76.8 -> 80 (step 8 in [64, 128)) -> 0.3125
    np.testing.assert_array_equal(O.fp8_basis_quantised(np.array([0.3, -1.0, 0.0])), [0.3125, -1.0, 0.0])


def test_fp8_row_and_frame_scaling_agree_in_the_normal_range():
    """With power-of-two scales, e4m3 rounding commutes with the scale for
    values in e4m3's normal range, so the per-row form equals the per-frame
    form wherever no sample is subnormal under either scale (a signal with
    no sample near zero relative to its frame's amax)."""
    spec = O.MelTSpec()
    n = np.arange(400 + 5 * 160)
    x = (0.6 + 0.3 * np.sin(2 * math.pi * 440 * n / 16000.0)).astype(np.float32)   # all in [0.3, 0.9]
    np.testing.assert_allclose(O.melt_clip_rounded(x, spec, "fp8"), O.melt_clip_rounded(x, spec, "fp8_frame"),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("scale", ["htk", "slaney"])
def test_rounded_stft_mel_reduces_to_the_pipeline_and_library_products(scale):
    """The comparator's rounded-operand form: with no rounding it is the
    conventional pipeline itself (window, |DFT|^2, filterbank, log); with BF16
    it is torch's bfloat16 operands multiplied in float64."""
    spec = O.MelTSpec(n_mels=40)
    x = np.random.default_rng(23).standard_normal(400 + 5 * 160 + 7).astype(np.float32)
    np.testing.assert_allclose(O.stft_mel_clip_rounded(x, spec, scale, "fp64"), O.stft_mel_clip(x, spec, scale),
                               rtol=1e-11, atol=1e-10)
    fk = np.arange(201) * 16000.0 / 400
    Wr, Wi = O.dmp_weights(fk, 400, 16000.0, O.hann(400, True))
    tb = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).to(torch.float64)
    X = O.frame_signal(x, 400, 160)
    Y = (tb(X) @ tb(np.concatenate([Wr, Wi])).T).numpy()
    F = O.triangular_filterbank(40, 400, 16000.0, 0.0, 8000.0, scale)
    ref = np.log((Y[:, :201] ** 2 + Y[:, 201:] ** 2) @ F.T + spec.eps)
    np.testing.assert_allclose(O.stft_mel_clip_rounded(x, spec, scale, "bf16"), ref, rtol=1e-12, atol=1e-12)
