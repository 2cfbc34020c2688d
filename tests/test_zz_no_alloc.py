"""melt_forward_noalloc: the allocation-free forward gives the same features as
melt_forward, call after call, and allocates nothing (GPU).

Callers that cannot allocate device memory at run time (real-time audio
threads, where cudaMalloc can block on driver locks and synchronise the
device; processes whose device memory another framework's caching allocator
already holds) use this entry point: its tile list lives in a fixed device
array instead of memory the library allocates.  This file is named to be
collected last.
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


def _batches():
    return [[G.rich_clip(71, i, L) for i, L in enumerate([48000, 30001, 400, 16000])],
            [G.rich_clip(72, i, L) for i, L in enumerate([160000, 399, 20480 + 160 * 3])]]


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp8"])
def test_noalloc_matches_melt_forward_twice(melt, prec):
    """Two calls in a row (different batches) on a basis that has never run
    melt_forward: bit-identical to melt_forward on a twin basis (the same
    kernels on the same tiles), with no allocation by the library and no
    change in the device's free memory."""
    import torch
    fe_ref = melt.Frontend(precision=prec)
    fe = melt.Frontend(precision=prec)         # only ever used through melt_forward_noalloc
    batches = _batches()
    # the per-device set-up (symbol address lookup, module load) happens on
    # the first call in the process: do it on the twin basis, outside the checks
    warm = G.pack_clips(batches[0])
    w0 = torch.from_numpy(warm.wave).cuda()
    o0 = torch.empty((fe_ref.total_frames(warm.lengths), fe_ref.n_out), device="cuda")
    melt.melt_forward_noalloc(fe_ref.handle, w0, warm.offsets, warm.lengths, o0)
    melt.melt_forward(fe_ref.handle, w0, warm.offsets, warm.lengths, o0)
    fe_ref.sync()
    for clips in batches:                      # two calls in a row, different batches
        pk = G.pack_clips(clips)
        wave = torch.from_numpy(pk.wave).cuda()
        T = fe.total_frames(pk.lengths)
        ref = torch.full((T, fe.n_out), float("nan"), device="cuda")
        got = torch.full((T, fe.n_out), float("nan"), device="cuda")
        melt.melt_forward(fe_ref.handle, wave, pk.offsets, pk.lengths, ref)
        fe_ref.sync()
        torch.cuda.synchronize()
        n0 = melt.melt_diag_alloc_count()
        free0 = torch.cuda.mem_get_info()[0]
        melt.melt_forward_noalloc(fe.handle, wave, pk.offsets, pk.lengths, got)
        fe.sync()
        free1 = torch.cuda.mem_get_info()[0]
        assert melt.melt_diag_alloc_count() == n0, "melt_forward_noalloc allocated"
        assert free1 == free0, (free0, free1)
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
    fe.close()
    fe_ref.close()


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


def test_noalloc_refuses_stream_capture(melt):
    """The plan is copied from a pageable host array, which a captured graph
    cannot replay: under capture the call is refused and enqueues nothing."""
    import torch
    fe = melt.Frontend(precision="bf16")
    pk = G.pack_clips(_batches()[0])
    wave = torch.from_numpy(pk.wave).cuda()
    out = torch.empty((fe.total_frames(pk.lengths), fe.n_out), device="cuda")
    melt.melt_forward_noalloc(fe.handle, wave, pk.offsets, pk.lengths, out)   # set-up before capture
    fe.sync()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=s):
        try:
            melt.melt_forward_noalloc(fe.handle, wave, pk.offsets, pk.lengths, out, stream=s)
        except melt.MeltError as e:
            status = e.status
    assert status == melt.MELT_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    fe.close()
