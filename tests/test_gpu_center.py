"""Centred framing: melt_pad_reflect and Frontend(center=True) against the oracle.

The padding is a copy, so it must equal the oracle's reflection exactly; the
centred features are the forward on the padded clips, held to the same
bounds as the uncentred parity tests.
"""
import numpy as np
import pytest

from oracle import melt_oracle as O
from paper_2606_01009_gb300 import inputs as G
from tests.helpers import fp32_sum_error, gpu_features, log_error_bound, oracle_features, rounded_log_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def melt():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt as m
    return m


def _clips():
    # lengths: the shortest a pad of 200 allows, ragged, several tiles, and a
    # clip whose reflected tail spans a whole frame
    lens = (201, 401, 16000, 23457, 48000 + 77)
    return [G.rich_clip(321, i, L) for i, L in enumerate(lens)]


def test_pad_reflect_equals_oracle(melt):
    import torch
    clips = _clips()
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    for pad in (0, 1, 7, 200):  # the shortest clip (201 samples) allows up to 200
        lens, offs, total = melt.padded_layout(pk.lengths, pad)
        out = torch.full((total,), float("nan"), device="cuda")
        melt.melt_pad_reflect(wave, pk.offsets, pk.lengths, pad, out, offs)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for c, o, L in zip(clips, offs, lens):
            ref = O.reflect_pad(c, pad).astype(np.float32)
            np.testing.assert_array_equal(got[o:o + L], ref)


def test_pad_reflect_many_clips_and_rejections(melt):
    import torch
    # more clips than one launch carries (1000), packed input, explicit output offsets
    rng = np.random.default_rng(5)
    lens = rng.integers(9, 300, size=2345)
    clips = [rng.standard_normal(int(L)).astype(np.float32) for L in lens]
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    plens, offs, total = melt.padded_layout(lens, 8)
    offs = offs + 16  # start after a gap, still 16-byte aligned
    out = torch.zeros(total + 16, device="cuda")
    melt.melt_pad_reflect(wave, None, lens, 8, out, offs)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[:16] == 0)
    for c, o, L in zip(clips, offs, plens):
        np.testing.assert_array_equal(got[o:o + L], O.reflect_pad(c, 8).astype(np.float32))
    # a clip of at most `pad` samples cannot be reflected: rejected before any launch
    with pytest.raises(melt.MeltError) as ei:
        melt.melt_pad_reflect(wave, pk.offsets, [8] + list(lens[1:]), 8, out, offs)
    assert ei.value.status == melt.MELT_ERR_ARG
    with pytest.raises(melt.MeltError) as ei:
        melt.melt_pad_reflect(wave, pk.offsets, lens, -1, out, offs)
    assert ei.value.status == melt.MELT_ERR_ARG


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_centred_features_match_oracle(melt, prec):
    clips = _clips()
    spec = O.MelTSpec()
    fe = melt.Frontend(precision=prec, center=True)
    assert [fe.num_frames(len(c)) for c in clips] == [len(c) // 160 + 1 for c in clips]
    got = gpu_features(fe, clips)
    fe.sync()
    fe.close()
    padded = [O.reflect_pad(c.astype(np.float64), 200) for c in clips]
    ref = np.concatenate([O.melt_clip_centred(c, spec) for c in clips])
    assert got.shape == ref.shape
    if prec == "fp32":
        bound = log_error_bound(spec, padded, fp32_sum_error(400))
    else:
        ref = oracle_features(spec, padded, rounded="bf16")
        bound = rounded_log_bound(spec, padded, "bf16", 4 * fp32_sum_error(400))
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (prec, int(bad.sum()), np.argwhere(bad)[:5])
