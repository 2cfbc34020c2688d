"""melt_forward_host: host buffers in, host buffers out, copies overlapped by the library.

The features must equal melt_forward's on the same device-resident batch bit
for bit (same kernels, same tiles; only where the samples come from differs),
for batches that make one chunk and several, with empty and short clips, with
explicit offsets that leave gaps, and with the correction MLP attached.
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


def _device_ref(melt, fe, pk):
    import torch
    out = fe(torch.from_numpy(pk.wave).cuda(), pk.offsets, pk.lengths)
    fe.sync()
    return out.cpu().numpy()


def _host(melt, fe, wave, offsets, lengths, rows, pinned=True):
    import torch
    w = torch.from_numpy(wave)
    o = torch.empty((rows, fe.n_out), dtype=torch.float32)
    if pinned:
        w, o = w.pin_memory(), o.pin_memory()
    s = torch.cuda.current_stream()
    melt.melt_forward_host(fe.handle, w, offsets, lengths, o, s)
    s.synchronize()
    fe.sync()
    return o.numpy()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_matches_device_path(melt, prec):
    lens = [0, 399, 400, 16000, 160000, 3, 48000 + 37, 480000, 22050, 128 * 160 + 240]
    clips = [G.rich_clip(61, i, L) if L >= 16 else np.zeros(L, np.float32) for i, L in enumerate(lens)]
    pk = G.pack_clips(clips)
    fe = melt.Frontend(precision=prec)
    ref = _device_ref(melt, fe, pk)
    got = _host(melt, fe, pk.wave, None, pk.lengths, ref.shape[0])
    assert np.array_equal(got, ref)
    got2 = _host(melt, fe, pk.wave, pk.offsets, pk.lengths, ref.shape[0], pinned=False)  # pageable
    assert np.array_equal(got2, ref)
    fe.close()


def test_many_chunks_gaps_and_repeats(melt):
    """A batch of ~58 MB (about eight chunks) with gaps between clips; a second call reuses the plan."""
    rng = np.random.default_rng(3)
    lens = [int(x) for x in rng.integers(1000, 480000, 60)]
    clips = [G.rich_clip(62, i, L) for i, L in enumerate(lens)]
    offs, o = [], 0
    for L in lens:
        offs.append(o)
        o += (L + 3) // 4 * 4 + 4 * int(rng.integers(0, 3))
    wave = np.zeros(o, np.float32)
    for c, off in zip(clips, offs):
        wave[off:off + len(c)] = c
    fe = melt.Frontend(precision="bf16")
    import torch
    dev = fe(torch.from_numpy(wave).cuda(), np.array(offs), np.array(lens))
    fe.sync()
    ref = dev.cpu().numpy()
    for _ in range(2):
        got = _host(melt, fe, wave, np.array(offs), np.array(lens), ref.shape[0])
        assert np.array_equal(got, ref)
    fe.close()


def test_correction_and_errors(melt):
    from oracle import mlp_oracle as P
    clips = [G.rich_clip(63, i, 16000 * 2) for i in range(3)]
    pk = G.pack_clips(clips)
    M, Hd = 80, 64
    params = melt.pack_mlp_params(G.xavier_uniform(1, Hd, M, 0), np.zeros(Hd), G.xavier_uniform(1, M, Hd, 1),
                                  np.zeros(M))
    mlp = melt.melt_mlp_create(M, Hd, params, np.full(M, -8, np.float32), np.full(M, 3, np.float32))
    fe = melt.Frontend(precision="bf16")
    melt.melt_basis_set_correction(fe.handle, mlp)
    ref = _device_ref(melt, fe, pk)
    got = _host(melt, fe, pk.wave, None, pk.lengths, ref.shape[0])
    assert np.array_equal(got, ref)
    melt.melt_basis_set_correction(fe.handle, None)
    out = np.zeros((ref.shape[0], 80), np.float32)
    for offs in ([4, 0, 8], [0, 2, 4]):               # unordered, unaligned
        with pytest.raises(melt.MeltError) as ei:
            melt.melt_forward_host(fe.handle, pk.wave, offs, pk.lengths, out)
        assert ei.value.status == melt.MELT_ERR_ARG
    fe.close()
    melt.melt_mlp_destroy(mlp)
