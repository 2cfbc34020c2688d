"""Parity of the tcgen05 tensor-core forms (BF16, split-BF16, FP8) with the oracle.

Two comparisons per form:
* element by element against the oracle evaluated on the same rounded
  operands (products exact, only the FP32 accumulation may differ), within a
  bound derived from the sum of |products|;
* against the exact FP64 oracle: the form's real error in dB, printed and
  held to a loose ceiling (bins within 60 dB of their frame's maximum).
"""
import numpy as np
import pytest

from oracle import melt_oracle as O
from paper_2606_01009_gb300 import inputs as G
from tests.helpers import (acc_rel, check_form_tolerance, dct_rel, db_report, fp32_sum_error, gpu_features,
                           log_error_bound, oracle_features, rounded_log_bound, LOGF_ABS, LOGF_REL)

pytestmark = pytest.mark.gpu

FORMS = ["bf16", "bf16x3", "fp8"]


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


acc_rel_ = acc_rel


def _check(melt, prec, clips, acc_rel=None, **kw):
    spec = _spec(**kw)
    fe = melt.Frontend(precision=prec, **kw)
    got = gpu_features(fe, clips)
    ref_r = oracle_features(spec, clips, rounded=prec)
    assert got.shape == ref_r.shape
    bound = rounded_log_bound(spec, clips, prec,
                              acc_rel_(prec, spec.n_fft, spec.hop) if acc_rel is None else acc_rel)
    bad = np.abs(got - ref_r) > bound
    assert not bad.any(), (prec, int(bad.sum()), np.argwhere(bad)[:5])
    exact = oracle_features(spec, clips)
    rep = db_report(got, exact)
    # the form's error vs FP64 is the operand rounding's: the oracle predicts it
    pred = db_report(ref_r, exact)
    for key in rep:
        assert rep[key][1] <= pred[key][1] * 1.02 + 2e-3, (key, rep[key], pred[key])
        assert rep[key][0] <= pred[key][0] + 0.05, (key, rep[key], pred[key])
    fe.close()
    return rep


@pytest.mark.parametrize("prec", FORMS)
def test_tones_8x1s(melt, prec):
    clips, _ = G.workload("tones_8x1s")
    rep = _check(melt, prec, clips)
    print(prec, "tones_8x1s vs FP64:", rep)


@pytest.mark.parametrize("prec", FORMS)
def test_ragged_and_multi_tile(melt, prec):
    lens = [0, 399, 400, 401, 560, 128 * 160 + 240, 129 * 160 + 240, 300 * 160 + 397, 16000, 3]
    clips = [G.rich_clip(21, i, L) if L >= 16 else np.ones(L, np.float32) for i, L in enumerate(lens)]
    rep = _check(melt, prec, clips)
    print(prec, "ragged vs FP64:", rep)


@pytest.mark.parametrize("prec", FORMS)
@pytest.mark.parametrize("n_mels", [128, 13, 40])
def test_mel_counts(melt, prec, n_mels):
    clips = [G.rich_clip(31, i, 30000) for i in range(3)]
    _check(melt, prec, clips, n_mels=n_mels)


@pytest.mark.parametrize("prec", FORMS)
def test_22k_group(melt, prec):
    """22.05 kHz, N = 1024, H = 256: J = 4 polyphase slices, 1024-term sums."""
    clips = [G.rich_clip(41, i, 22050 * 3 + 5, sr=22050.0) for i in range(3)]
    _check(melt, prec, clips, sr=22050.0, n_fft=1024, hop=256)


@pytest.mark.parametrize("prec", FORMS)
def test_mfcc(melt, prec):
    clips = [G.rich_clip(51, i, 25000) for i in range(2)]
    spec = _spec(n_mfcc=40)
    fe = melt.Frontend(precision=prec, n_mfcc=40)
    got = gpu_features(fe, clips)
    spec_l = _spec()
    lb = rounded_log_bound(spec_l, clips, prec, acc_rel(prec))
    D = O.dct2_ortho(40, 80)
    logmel_r = oracle_features(spec_l, clips, rounded=prec)
    ref = logmel_r @ D.T
    bound = lb @ np.abs(D).T + dct_rel(prec, 80) * (np.abs(logmel_r) @ np.abs(D).T)
    assert np.all(np.abs(got - ref) <= bound)
    fe.close()


def test_silent_and_tiny_inputs(melt):
    clips = [np.zeros(3000, np.float32), np.full(1000, 1e-30, np.float32), np.ones(600, np.float32) * 0.5]
    for prec in FORMS:
        _check(melt, prec, clips)


@pytest.fixture(scope="module")
def levels():
    """The 1024 x 10 s sweep workload and the FP64 oracle on its checked clips."""
    clips, sr = G.workload("levels_1024x10s")
    idx = list(range(0, 1024, 32))
    sub = [clips[b] for b in idx]
    return clips, sr, idx, sub, oracle_features(_spec(), sub)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32"] + FORMS)
def test_precision_sweep_1024x10s(melt, levels, prec):
    """The precision sweep: all 1024 clips of 10 s (levels -60..0 dBFS) in
    one launch per form.  Every 32nd clip (32 clips, 31,936 frames) is
    checked element by element (reduced forms: against the rounded-operand
    oracle within the accumulation bound; FP32: against FP64 within the FP32
    bound), and each form's error against FP64 must stay within its stated
    tolerance at every depth below the frame maximum."""
    clips, sr, idx, sub, exact = levels
    spec = _spec()
    fe = melt.Frontend(sr=sr, precision=prec)
    got = gpu_features(fe, clips)
    fe.close()
    assert got.shape == (1024 * 998, 80)
    rows = np.concatenate([np.arange(998) + b * 998 for b in idx])
    if prec == "fp32":
        ref, bound = exact, log_error_bound(spec, sub, fp32_sum_error(spec.n_fft))
    else:
        ref = oracle_features(spec, sub, rounded=prec)
        bound = rounded_log_bound(spec, sub, prec, acc_rel(prec))
    bad = np.abs(got[rows] - ref) > bound
    assert not bad.any(), (prec, int(bad.sum()))
    rep = db_report(got[rows], exact)
    print(prec, "levels_1024x10s (32 clips) vs FP64:",
          {k: (round(v[0], 6), round(v[1], 7)) for k, v in rep.items()})
    assert not check_form_tolerance(prec, rep), check_form_tolerance(prec, rep)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
@pytest.mark.parametrize("n_mels", [144, 256, 400, 512])
def test_more_than_128_mel_bins(melt, prec, n_mels):
    """More than 128 Mel bins (the accumulator in blocks of 128 bins, the basis
    streamed block by block): element by element against the rounded-operand
    oracle, clips ending mid-tile included."""
    clips = [G.rich_clip(33, i, L) for i, L in enumerate((30000, 128 * 160 + 240, 16000))]
    _check(melt, prec, clips, n_mels=n_mels)


def test_more_than_128_mel_bins_needs_bf16_log_mel(melt):
    for kw in (dict(precision="fp32"), dict(precision="fp8"), dict(precision="bf16", n_mfcc=40)):
        with pytest.raises(melt.MeltError) as ei:
            melt.Frontend(n_mels=256, **kw)
        assert ei.value.status == melt.MELT_ERR_UNSUPPORTED, kw


def test_epilogue_log_error_bound(melt):
    """The epilogues' natural log (hardware log2 times ln 2, subnormals
    flushed) against the exact function: within the bound every parity test
    assumes for it, LOGF_ABS + LOGF_REL |ln x|, on 4096 mantissas of every
    normal binade and on random values."""
    import torch
    e = np.arange(-126, 128)
    m = 1.0 + np.arange(4096) / 4096.0
    x = (m[None, :] * np.exp2(e[:, None].astype(np.float64))).astype(np.float32).ravel()
    x = x[np.isfinite(x)]
    rng = np.random.default_rng(5)
    x = np.concatenate([x, np.exp(rng.uniform(-80, 80, 200000)).astype(np.float32),
                        np.array([1e-10, 1.0, 0.5, 2.0, np.nextafter(np.float32(1), 0)], np.float32)])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    melt.melt_diag_log(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.float64)
    exact = np.log(x.astype(np.float64))
    err = np.abs(y - exact)
    bound = LOGF_ABS + LOGF_REL * np.abs(exact)
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), x[bad][:5], err[bad][:5])
    near = (x >= 0.5) & (x <= 2)
    print("epilogue log: max abs error on [0.5, 2] %.3g (2^%.2f); max relative error elsewhere %.3g (2^%.2f)" %
          (err[near].max(), np.log2(err[near].max()), (err[~near] / np.abs(exact[~near])).max(),
           np.log2((err[~near] / np.abs(exact[~near])).max())))
