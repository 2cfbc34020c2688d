"""The seeded input generator against its documented recipe (no GPU).

Clip i of a workload must not depend on the batch it is drawn in; rich clips
are peak-normalised to the requested level; packed batches start every clip
on a 16-byte boundary; lengths and groups follow the stated distributions.
"""
import numpy as np

from paper_2606_01009_gb300 import inputs as G


def test_clip_i_does_not_depend_on_the_batch():
    full, sr = G.workload("tones_8x1s")
    one, _ = G.workload("tones_8x1s", clips=1, first=5)
    assert sr == 16000.0 and len(full) == 8
    np.testing.assert_array_equal(full[5], one[0])
    a, _ = G.workload("rich_64x30s", clips=2)
    b, _ = G.workload("rich_64x30s", clips=1, first=1)
    np.testing.assert_array_equal(a[1], b[0])
    c, _ = G.workload("rich_64x30s", seed=99, clips=1, first=1)
    assert not np.array_equal(b[0], c[0])


def test_shapes_dtypes_and_peak_levels():
    tones, _ = G.workload("tones_8x1s", clips=3)
    for x in tones:
        assert x.dtype == np.float32 and x.shape == (16000,)
        assert np.abs(x).max() < 4 * 0.5 + 0.2  # at most 4 tones of amplitude <= 0.5, plus -30 dBFS noise
    rich, _ = G.workload("rich_64x30s", clips=2)
    for x in rich:
        assert x.shape == (480000,)
        np.testing.assert_allclose(np.abs(x).max(), 1.0, rtol=1e-6)  # peak 0 dBFS
    lv = G.levels_dbfs(1234, 1024)
    assert lv.min() >= -60.0 and lv.max() <= 0.0
    quiet, _ = G.workload("levels_1024x10s", clips=2, first=3)
    for k, x in enumerate(quiet):
        assert x.shape == (160000,)
        np.testing.assert_allclose(np.abs(x).max(), 10 ** (lv[3 + k] / 20), rtol=1e-5)


def test_tone_frequencies_lie_in_the_stated_band():
    tones, sr = G.workload("tones_8x1s")
    for x in tones:
        spec = np.abs(np.fft.rfft(x.astype(np.float64)))
        f_peak = np.argmax(spec) * sr / x.shape[0]
        assert 45.0 <= f_peak <= 7505.0


def test_pack_clips_alignment_and_content():
    clips = [np.arange(n, dtype=np.float32) + 1 for n in (5, 0, 8, 13)]
    pk = G.pack_clips(clips)
    assert pk.lengths.tolist() == [5, 0, 8, 13]
    assert all(o % 4 == 0 for o in pk.offsets)
    assert pk.offsets.tolist() == [0, 8, 8, 16]
    for c, o in zip(clips, pk.offsets):
        np.testing.assert_array_equal(pk.wave[o:o + c.shape[0]], c)
    assert np.all(pk.wave[5:8] == 0)  # padding between clips


def test_lengths_and_groups_of_the_mixed_batch():
    L = G.loguniform_lengths(7, 2000, 0.5, 30.0, 16000.0)
    assert L.min() >= 0.5 * 16000 - 1 and L.max() <= 30.0 * 16000 + 1
    clips, ids = G.mixed_groups(count=64, n=12, pool=2)
    assert list(ids) == [i % 2 for i in range(12)]
    for x, g in zip(clips, ids):
        sr = G.MIXED_GROUPS[g][0]
        assert 0.5 * sr - 1 <= x.shape[0] <= 30.0 * sr + 1
