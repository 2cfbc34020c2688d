"""melt_forward_noalloc: the allocation-free forward gives the same features as
melt_forward, call after call (GPU).

Callers that cannot allocate device memory at run time (real-time audio
threads, processes whose memory another allocator owns) use this entry point;
its tile list lives in a fixed device array instead of library-allocated
memory.  This file is named to be collected last.
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


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_noalloc_matches_melt_forward_twice(melt, prec):
    import torch
    fe = melt.Frontend(precision=prec)
    batches = [[G.rich_clip(71, i, L) for i, L in enumerate([48000, 30001, 400, 16000])],
               [G.rich_clip(72, i, L) for i, L in enumerate([160000, 399, 20480 + 160 * 3])]]
    for clips in batches:                      # two calls in a row, different batches
        pk = G.pack_clips(clips)
        wave = torch.from_numpy(pk.wave).cuda()
        T = fe.total_frames(pk.lengths)
        ref = torch.full((T, fe.n_out), float("nan"), device="cuda")
        got = torch.full((T, fe.n_out), float("nan"), device="cuda")
        melt.melt_forward(fe.handle, wave, pk.offsets, pk.lengths, ref)
        melt.melt_forward_noalloc(fe.handle, wave, pk.offsets, pk.lengths, got)
        fe.sync()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(g).all()
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-6)
    fe.close()


def test_noalloc_rejects_too_many_tiles(melt):
    import torch
    fe = melt.Frontend(precision="bf16")
    # 16384 tiles is the array's capacity; 16385 clips of one frame each need 16385 tiles
    lengths = np.full(16385, 400, np.int64)
    wave = torch.zeros(16385 * 400, device="cuda")
    out = torch.empty((16385, 80), device="cuda")
    with pytest.raises(melt.MeltError) as ei:
        melt.melt_forward_noalloc(fe.handle, wave, None, lengths, out)
    assert ei.value.status == melt.MELT_ERR_ARG
    # the capacity itself is accepted
    melt.melt_forward_noalloc(fe.handle, wave, None, lengths[:16384], out[:16384])
    fe.sync()
    fe.close()
