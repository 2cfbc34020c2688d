"""The fused STFT + triangular Mel comparator (melt_stft_create) against the
oracle's conventional pipeline (GPU).

The comparator projects each frame onto the window-folded cos/sin rows at the
N/2 + 1 uniform DFT frequencies on the tensor cores and fuses |X_k|^2, the
triangular filterbank and the log into the epilogue.  Element by element it
must match the oracle evaluated on the same rounded GEMM operands
(stft_mel_clip_rounded) within a bound built like the MelT one: each bin's
power carries at most the FP32 accumulation error of its two sums, carried
through the non-negative filterbank, plus the FP32 filterbank sum itself.
"""
import numpy as np
import pytest

from oracle import melt_oracle as O
from paper_2606_01009_gb300 import inputs as G
from tests.helpers import LOGF_ABS, LOGF_REL, U32, acc_rel, gpu_features, rounded_components

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def melt():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt as m
    return m


def _bound(spec, clips, prec, scale):
    """Elementwise bound on |GPU - stft_mel_clip_rounded| (natural log)."""
    K = spec.n_fft // 2 + 1
    uni = O.MelTSpec(sr=spec.sr, n_fft=spec.n_fft, hop=spec.hop, periodic=spec.periodic,
                     freqs=np.arange(K) * spec.sr / spec.n_fft)
    R, I, ER, EI = rounded_components(uni, clips, prec)
    rel = acc_rel(prec, spec.n_fft, spec.hop)
    dR, dI = rel * ER, rel * EI
    S = R * R + I * I
    dS = 2 * np.abs(R) * dR + 2 * np.abs(I) * dI + dR * dR + dI * dI + 4 * U32 * S
    F = O.triangular_filterbank(spec.n_mels, spec.n_fft, spec.sr, spec.fmin, spec.fmax, scale)
    E = S @ F.T
    nnz = (F > 0).sum(axis=1)
    dE = dS @ F.T + ((nnz + 3) * U32)[None, :] * E  # + FP32 filterbank sum and FP32 weights
    den = E + spec.eps - dE
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.where(den > 0, dE / np.maximum(den, 1e-300), np.inf)
    return b + LOGF_ABS + LOGF_REL * np.abs(np.log(E + spec.eps))


@pytest.mark.parametrize("scale", ["htk", "slaney"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_fused_stft_mel_matches_rounded_pipeline(melt, prec, scale):
    lens = [0, 399, 400, 30000, 128 * 160 + 240, 129 * 160 + 240, 16000]
    clips = [G.rich_clip(81, i, L) if L >= 16 else np.zeros(L, np.float32) for i, L in enumerate(lens)]
    spec = O.MelTSpec(n_mels=80)
    fe = melt.StftMelFrontend(precision=prec, scale=scale)
    assert fe.n_out == 80
    got = gpu_features(fe, clips)
    fe.close()
    ref = np.concatenate([O.stft_mel_clip_rounded(c, spec, scale, prec) for c in clips])
    assert got.shape == ref.shape
    bound = _bound(spec, clips, prec, scale)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (prec, scale, int(bad.sum()), np.argwhere(bad)[:5])
    exact = np.concatenate([O.stft_mel_clip(c, spec, scale) for c in clips])
    d = O.nat_to_db(np.abs(got - exact))
    print(f"fused STFT+Mel {prec} {scale}: max {d.max():.3g} dB, rms {np.sqrt(np.mean(d * d)):.3g} dB vs FP64")


def test_fused_stft_mel_other_geometry_and_refusals(melt):
    """22.05 kHz, N = 1024, H = 256 (513 DFT bins, five accumulator blocks), 40
    Slaney bands over 50-8000 Hz; FP32 and FP8 are refused."""
    clips = [G.rich_clip(82, i, L, sr=22050.0) for i, L in enumerate((22050 * 2 + 3, 5000))]
    spec = O.MelTSpec(sr=22050.0, n_fft=1024, hop=256, n_mels=40, fmin=50.0, fmax=8000.0)
    fe = melt.StftMelFrontend(sr=22050.0, n_fft=1024, hop=256, n_mels=40, fmin=50.0, fmax=8000.0, precision="bf16",
                              scale="slaney")
    got = gpu_features(fe, clips)
    fe.close()
    ref = np.concatenate([O.stft_mel_clip_rounded(c, spec, "slaney", "bf16") for c in clips])
    bad = np.abs(got - ref) > _bound(spec, clips, "bf16", "slaney")
    assert not bad.any(), int(bad.sum())
    for prec in ("fp32", "fp8"):
        with pytest.raises(melt.MeltError) as ei:
            melt.StftMelFrontend(precision=prec)
        assert ei.value.status == melt.MELT_ERR_UNSUPPORTED
