"""Parity of the plain FP32 CUDA path (SIMT FFMA kernel) with the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import melt_oracle as O
from paper_2606_01009_gb300 import inputs as G
from tests.helpers import (db_report, fp32_sum_error, gpu_features, log_error_bound,
                           oracle_features)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def melt():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt as m
    return m


def _spec(**kw):
    base = dict(sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0)
    base.update(kw)
    return O.MelTSpec(**base)


def test_basis_builder_matches_oracle_basis(melt):
    for kw in [dict(), dict(n_mels=128), dict(sr=22050.0, n_fft=1024, hop=256),
               dict(fmin=80.0, fmax=7600.0, periodic=False)]:
        spec = _spec(**kw)
        h = melt.melt_basis_create_ex(spec.sr, spec.n_fft, spec.hop, spec.n_mels, spec.fmin, spec.fmax,
                                      0 if spec.periodic else 1)
        freqs, w = melt.melt_basis_get_fp64(h)
        melt.melt_destroy(h)
        np.testing.assert_allclose(freqs, spec.freqs, rtol=1e-13)
        np.testing.assert_allclose(w, np.concatenate([spec.Wr, spec.Wi]), atol=1e-12)


def test_tones_8x1s_elementwise(melt):
    clips, sr = G.workload("tones_8x1s")
    spec = _spec()
    fe = melt.Frontend(sr=sr, precision="fp32")
    got = gpu_features(fe, clips)
    ref = oracle_features(spec, clips)
    assert got.shape == ref.shape == (8 * 98, 80)
    bound = log_error_bound(spec, clips, fp32_sum_error(spec.n_fft))
    viol = np.abs(got - ref) > bound
    assert not viol.any(), f"{viol.sum()} elements outside the FP32 error bound"
    rep = db_report(got, ref)
    print("fp32 tones_8x1s", rep)
    assert rep["within_60dB"][0] < 1e-3


def test_components_match_oracle(melt):
    clips = [G.rich_clip(5, i, 9000) for i in range(3)]
    spec = _spec()
    fe = melt.Frontend(precision="fp32")
    import torch
    pk = G.pack_clips(clips)
    T = fe.total_frames(pk.lengths)
    out = torch.empty((T, 160), device="cuda")
    melt.melt_forward_components(fe.handle, torch.from_numpy(pk.wave).cuda(), pk.offsets, pk.lengths, out)
    fe.sync()
    got = out.cpu().numpy().astype(np.float64)
    R = np.concatenate([O.melt_components(c, spec)[0] for c in clips])
    I = np.concatenate([O.melt_components(c, spec)[1] for c in clips])
    E = fp32_sum_error(400) * np.concatenate([np.abs(O.frame_signal(c, 400, 160)) @ spec.window for c in clips])
    assert np.all(np.abs(got[:, :80] - R) <= E[:, None])
    assert np.all(np.abs(got[:, 80:] - I) <= E[:, None])


def test_ragged_lengths_offsets_and_tiles(melt):
    spec = _spec()
    lens = [0, 399, 400, 401, 559, 560, 16000, 128 * 160 + 240, 129 * 160 + 240, 300 * 160 + 397, 3]
    clips = [G.rich_clip(11, i, L) if L >= 16 else np.random.default_rng(i).standard_normal(L).astype(np.float32)
             for i, L in enumerate(lens)]
    fe = melt.Frontend(precision="fp32")
    got = gpu_features(fe, clips)
    ref = oracle_features(spec, clips)
    assert got.shape == ref.shape
    bound = log_error_bound(spec, clips, fp32_sum_error(400))
    assert np.all(np.abs(got - ref) <= bound)
    # explicit, non-packed offsets (each a multiple of 4, with gaps of garbage)
    import torch
    offs = []
    pos = 12
    for L in lens:
        offs.append(pos)
        pos += (L + 3) // 4 * 4 + 8
    buf = np.full(pos + 16, np.nan, np.float32)
    for o, c in zip(offs, clips):
        buf[o:o + len(c)] = c
        buf[o + len(c):o + (len(c) + 3) // 4 * 4] = 0.0
    out = fe(torch.from_numpy(buf).cuda(), np.array(offs, np.int64), np.array(lens, np.int64))
    fe.sync()
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), got)


def test_uniform_frequencies_are_a_dft(melt):
    N, H, sr = 192, 48, 8000.0          # N/2 + 1 = 97 analysis bins (cap is 128)
    freqs = np.arange(N // 2 + 1) * sr / N
    fe = melt.Frontend(sr=sr, n_fft=N, hop=H, precision="fp32", freqs=freqs)
    clips = [np.random.default_rng(4).standard_normal(N + 40 * H).astype(np.float32)]
    got = gpu_features(fe, clips)
    X = O.frame_signal(clips[0], N, H) * O.hann(N)[None, :]
    ref = np.log(np.abs(np.fft.rfft(X, axis=1)) ** 2 + 1e-10)
    spec = O.MelTSpec(sr=sr, n_fft=N, hop=H, freqs=freqs)
    bound = log_error_bound(spec, clips, fp32_sum_error(N))
    assert np.all(np.abs(got - ref) <= bound + 1e-9)


@pytest.mark.parametrize("n_mels", [80, 128, 40, 13])
def test_mfcc_and_mel_counts(melt, n_mels):
    clips = [G.rich_clip(3, i, 20000) for i in range(2)]
    K = min(40, n_mels)
    spec = _spec(n_mels=n_mels, n_mfcc=K)
    fe = melt.Frontend(n_mels=n_mels, n_mfcc=K, precision="fp32")
    got = gpu_features(fe, clips)
    spec_l = _spec(n_mels=n_mels)
    lb = log_error_bound(spec_l, clips, fp32_sum_error(400))
    ref = oracle_features(spec, clips)
    D = O.dct2_ortho(K, n_mels)
    logmel = oracle_features(spec_l, clips)
    bound = lb @ np.abs(D).T + (n_mels + 2) * 2 ** -24 * (np.abs(logmel) @ np.abs(D).T)
    assert np.all(np.abs(got - ref) <= bound)


def test_22k_group_config(melt):
    clips = [G.rich_clip(9, i, 22050 * 2 + 77, sr=22050.0) for i in range(3)]
    spec = _spec(sr=22050.0, n_fft=1024, hop=256)
    fe = melt.Frontend(sr=22050.0, n_fft=1024, hop=256, precision="fp32")
    got = gpu_features(fe, clips)
    ref = oracle_features(spec, clips)
    assert np.all(np.abs(got - ref) <= log_error_bound(spec, clips, fp32_sum_error(1024)))


@pytest.mark.slow
def test_full_rich_64x30s_sampled(melt):
    """Full 64 x 30 s workload in one launch; sampled frames against the oracle."""
    clips, sr = G.workload("rich_64x30s")
    spec = _spec()
    fe = melt.Frontend(sr=sr, precision="fp32")
    got = gpu_features(fe, clips)
    assert got.shape == (64 * 2998, 80)
    rng = np.random.default_rng(0)
    for b in rng.choice(64, 6, replace=False):
        frames = np.sort(rng.choice(2998, 40, replace=False))
        frames[-1] = 2997
        ref = O.melt_clip(clips[b], spec, frames)
        R, I = O.melt_components(clips[b], spec, frames)
        E = fp32_sum_error(400) * (np.abs(O.frame_signal(clips[b], 400, 160, frames)) @ spec.window)[:, None]
        S = R * R + I * I
        dS = 2 * (np.abs(R) + np.abs(I)) * E + 2 * E * E + 4 * 2 ** -24 * S
        bound = (np.where(S + 1e-10 - dS > 0, dS / np.maximum(S + 1e-10 - dS, 1e-300), np.inf)
                 + 2.0 ** -21 + 4 * 2.0 ** -23 * np.abs(ref))
        assert np.all(np.abs(got[b * 2998 + frames] - ref) <= bound)
