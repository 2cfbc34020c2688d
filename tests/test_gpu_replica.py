"""The paper's two frontend configurations (Sec. IV, Table "Audio frontend
configuration") through every form, against the oracle.

* spectral: 16 kHz, N = 400 (25 ms), H = 160, M = 80, f 80-7600 Hz;
* cepstral: 16 kHz, N = 1200 (75 ms), H = 160, M = 128, K = 40, f 0-8000 Hz.

The paper states a symmetric Hann window, which these tests use.  Each form
is compared element by element with the oracle evaluated on the operands the
form multiplies (bounds as in the other parity tests), and its real error
against the exact FP64 oracle is held to what the operand rounding predicts.
A tensor-core form whose operands do not fit shared memory for a
configuration reports MELT_ERR_UNSUPPORTED at creation, which the test
accepts only for that reason.
"""
import numpy as np
import pytest

from oracle import melt_oracle as O
from paper_2606_01009_gb300 import inputs as G
from tests.helpers import (acc_rel, db_report, dct_rel, fp32_sum_error, gpu_features, log_error_bound, oracle_features,
                           rounded_log_bound)

pytestmark = pytest.mark.gpu

SPECTRAL = dict(sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=80.0, fmax=7600.0)
CEPSTRAL = dict(sr=16000.0, n_fft=1200, hop=160, n_mels=128, fmin=0.0, fmax=8000.0)
FORMS = ["fp32", "bf16", "bf16x3", "fp8"]


@pytest.fixture(scope="module")
def melt():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt as m
    return m


def _clips():
    # two 2.5 s clips and one that ends mid-tile, from the rich generator
    return [G.rich_clip(2606, i, L) for i, L in enumerate((40000, 40000, 23457))]


def _frontend(melt, prec, cfg, n_mfcc=0):
    try:
        return melt.Frontend(precision=prec, window=melt.MELT_WIN_HANN_SYMMETRIC, n_mfcc=n_mfcc, **cfg)
    except melt.MeltError as e:
        assert e.status == melt.MELT_ERR_UNSUPPORTED, e
        pytest.skip(f"{prec} does not fit shared memory for {cfg} (MELT_ERR_UNSUPPORTED)")


def _log_mel_bound(spec, clips, prec):
    if prec == "fp32":
        return log_error_bound(spec, clips, fp32_sum_error(spec.n_fft)), oracle_features(spec, clips)
    rel = acc_rel(prec, spec.n_fft, spec.hop)
    return rounded_log_bound(spec, clips, prec, rel), oracle_features(spec, clips, rounded=prec)


@pytest.mark.parametrize("prec", FORMS)
def test_spectral_configuration(melt, prec):
    clips = _clips()
    spec = O.MelTSpec(periodic=False, **SPECTRAL)
    fe = _frontend(melt, prec, SPECTRAL)
    got = gpu_features(fe, clips)
    fe.close()
    bound, ref = _log_mel_bound(spec, clips, prec)
    assert got.shape == ref.shape == (sum(O.num_frames(len(c), 400, 160) for c in clips), 80)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (prec, int(bad.sum()), np.argwhere(bad)[:5])
    exact = oracle_features(spec, clips)
    rep, pred = db_report(got, exact), db_report(ref, exact)
    print(prec, "spectral dB error (max, rms):", rep)
    for key in rep:
        assert rep[key][1] <= pred[key][1] * 1.02 + 2e-3, (key, rep[key], pred[key])


@pytest.mark.parametrize("prec", FORMS)
def test_cepstral_configuration(melt, prec):
    clips = _clips()
    spec_l = O.MelTSpec(periodic=False, **CEPSTRAL)
    fe = _frontend(melt, prec, CEPSTRAL, n_mfcc=40)
    got = gpu_features(fe, clips)
    fe.close()
    lb, logmel = _log_mel_bound(spec_l, clips, prec)
    D = O.dct2_ortho(40, 128)
    ref = logmel @ D.T
    assert got.shape == ref.shape
    # the log-Mel bound carried through the DCT, plus the DCT's own error
    bound = lb @ np.abs(D).T + dct_rel(prec, 128) * (np.abs(logmel) @ np.abs(D).T)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (prec, int(bad.sum()), np.argwhere(bad)[:5])
    exact = O.MelTSpec(periodic=False, n_mfcc=40, **CEPSTRAL)
    err = np.abs(got - oracle_features(exact, clips))
    print(prec, "cepstral max |error| vs FP64:", float(err.max()))
