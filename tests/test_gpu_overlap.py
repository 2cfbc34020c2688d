"""melt_forward_ex with MELT_FWD_INPUT_READY: the launch reads and converts its
waveform while the kernel before it on the stream drains, and must give the
same features as melt_forward, bit for bit, over chains of back-to-back
launches on rotating buffers (GPU).
"""
import numpy as np
import pytest

from paper_2606_01009_gb300 import inputs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def melt():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt as m
    return m


def _batches(n):
    """n different batches (uneven clips, ragged tails, one empty clip)."""
    out = []
    for b in range(n):
        lens = [0 if b % 3 == 0 else 401, 48000 + 160 * b, 128 * 160 + 240, 160000 - 999 * b, 30001]
        clips = [G.rich_clip(90 + b, i, L) if L >= 16 else np.zeros(L, np.float32) for i, L in enumerate(lens)]
        out.append(G.pack_clips(clips))
    return out


@pytest.mark.parametrize("kw", [dict(precision="bf16"), dict(precision="fp8"), dict(precision="bf16x3"),
                                dict(precision="bf16", n_mfcc=40), dict(precision="bf16", n_mels=128),
                                dict(precision="fp32")])
def test_input_ready_chain_equals_melt_forward(melt, kw):
    import torch
    fe = melt.Frontend(**kw)
    batches = _batches(6)
    waves = [torch.from_numpy(pk.wave).cuda() for pk in batches]
    refs = []
    for pk, w in zip(batches, waves):
        refs.append(fe(w, pk.offsets, pk.lengths).cpu().numpy())
    fe.sync()
    torch.cuda.synchronize()
    # back-to-back launches, each batch into its own output, every batch twice
    outs = [torch.full((fe.total_frames(pk.lengths), fe.n_out), float("nan"), device="cuda") for pk in batches]
    for rep in range(2):
        for pk, w, o in zip(batches, waves, outs):
            melt.melt_forward_ex(fe.handle, w, pk.offsets, pk.lengths, o, melt.MELT_FWD_INPUT_READY)
    fe.sync()
    for ref, o in zip(refs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), ref)
    fe.close()


def test_input_ready_after_other_kernels_and_same_output(melt):
    """Launches that reuse one output buffer, with unrelated kernels between
    them on the stream: the stores still wait for the preceding kernel."""
    import torch
    fe = melt.Frontend(precision="bf16")
    batches = _batches(3)
    waves = [torch.from_numpy(pk.wave).cuda() for pk in batches]
    T = max(fe.total_frames(pk.lengths) for pk in batches)
    out = torch.empty((T, fe.n_out), device="cuda")
    scratch = torch.zeros(1 << 20, device="cuda")
    for pk, w in zip(batches, waves):
        scratch.add_(1.0)                      # a kernel of another library right before the launch
        melt.melt_forward_ex(fe.handle, w, pk.offsets, pk.lengths, out, melt.MELT_FWD_INPUT_READY)
        got = out[:fe.total_frames(pk.lengths)].clone()   # reads the output on the same stream
        ref = torch.empty_like(got)
        melt.melt_forward(fe.handle, w, pk.offsets, pk.lengths, ref)
        fe.sync()
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
    fe.close()


def test_unknown_flag_is_rejected(melt):
    import torch
    fe = melt.Frontend(precision="bf16")
    pk = _batches(1)[0]
    w = torch.from_numpy(pk.wave).cuda()
    out = torch.empty((fe.total_frames(pk.lengths), fe.n_out), device="cuda")
    with pytest.raises(melt.MeltError) as ei:
        melt.melt_forward_ex(fe.handle, w, pk.offsets, pk.lengths, out, 2)
    assert ei.value.status == melt.MELT_ERR_ARG
    fe.close()
