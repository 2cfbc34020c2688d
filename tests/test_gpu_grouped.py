"""Grouped launch over two basis groups (16 kHz 400/160/80 and 22.05 kHz 1024/256/80).

The grouped call must give exactly what melt_forward gives for each clip with
its own basis (the tile math is the same), with and without CUDA graphs, on
the first call and on graph replays, and after the layout cache evicts.
"""
import numpy as np
import pytest

from oracle import melt_oracle as O
from paper_2606_01009_gb300 import inputs as G
from tests.helpers import fp32_sum_error, oracle_features, rounded_log_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def melt():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt as m
    return m


def _frontends(melt, precisions=("bf16", "bf16")):
    fes = []
    for (sr, n_fft, hop, n_mels, fmin, fmax), prec in zip(G.MIXED_GROUPS, precisions):
        fes.append(melt.Frontend(sr=sr, n_fft=n_fft, hop=hop, n_mels=n_mels, fmin=fmin, fmax=fmax,
                                 precision=prec))
    return fes


def _per_clip_reference(fes, clips, ids):
    """melt_forward over each group's clips (one launch per group), rows put back in batch order."""
    import torch
    rows = []
    for c, g in zip(clips, ids):
        rows.append(fes[g].num_frames(len(c)))
    starts = np.concatenate([[0], np.cumsum(rows)])
    out = np.zeros((int(starts[-1]), fes[0].n_out), np.float32)
    for g, fe in enumerate(fes):
        sel = [b for b in range(len(clips)) if ids[b] == g]
        if not sel:
            continue
        pk = G.pack_clips([clips[b] for b in sel])
        o = fe(torch.from_numpy(pk.wave).cuda(), pk.offsets, pk.lengths).cpu().numpy()
        fe.sync()
        r = 0
        for b in sel:
            out[starts[b]:starts[b + 1]] = o[r:r + rows[b]]
            r += rows[b]
    return out


def _grouped(melt, fes, clips, ids, graphs=True, repeat=1):
    import torch
    gf = melt.GroupedFrontend(fes, graphs=graphs)
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    T = gf.total_frames(pk.lengths, ids)
    out = torch.full((T, gf.n_out), float("nan"), device="cuda")
    res = []
    for _ in range(repeat):
        out.fill_(float("nan"))
        gf(wave, pk.offsets, pk.lengths, ids, out=out)
        gf.sync()
        res.append(out.cpu().numpy())
    gf.close()
    return res


@pytest.mark.parametrize("graphs", [True, False])
def test_grouped_equals_per_group_launches(melt, graphs):
    clips, ids = G.mixed_groups(n=40)
    fes = _frontends(melt)
    ref = _per_clip_reference(fes, clips, ids)
    outs = _grouped(melt, fes, clips, ids, graphs=graphs, repeat=3)
    for o in outs:                                  # first call, then replays
        assert np.array_equal(o, ref)
    for fe in fes:
        fe.close()


def test_grouped_parity_with_oracle(melt):
    """Two short clips per group against the rounded-operand oracle."""
    clips = [G.rich_clip(61, 0, 9000), G.rich_clip(61, 1, 22050 * 2 + 77, sr=22050.0),
             G.rich_clip(61, 2, 400), G.rich_clip(61, 3, 1023, sr=22050.0),
             G.rich_clip(61, 4, 16000 * 3 + 13), G.rich_clip(61, 5, 1024, sr=22050.0)]
    ids = np.array([0, 1, 0, 1, 0, 1], np.int32)
    fes = _frontends(melt)
    got = _grouped(melt, fes, clips, ids)[0].astype(np.float64)
    r = 0
    for c, g in zip(clips, ids):
        sr, n_fft, hop, n_mels, fmin, fmax = G.MIXED_GROUPS[g]
        spec = O.MelTSpec(sr=sr, n_fft=n_fft, hop=hop, n_mels=n_mels, fmin=fmin, fmax=fmax)
        ref = oracle_features(spec, [c], rounded="bf16")
        bound = rounded_log_bound(spec, [c], "bf16", 4 * fp32_sum_error(n_fft))
        t = ref.shape[0]
        assert np.all(np.abs(got[r:r + t] - ref) <= bound), (g, len(c))
        r += t
    assert r == got.shape[0]
    for fe in fes:
        fe.close()


def test_mixed_precision_groups(melt):
    """Groups may differ in operand form: FP32 SIMT for one, BF16 tensor cores for the other."""
    clips, ids = G.mixed_groups(n=10, first=100)
    fes = _frontends(melt, ("fp32", "bf16"))
    ref = _per_clip_reference(fes, clips, ids)
    assert np.array_equal(_grouped(melt, fes, clips, ids)[0], ref)
    for fe in fes:
        fe.close()


def test_layout_cache_eviction(melt):
    """More batch layouts than the cache holds, then the first again."""
    import torch
    fes = _frontends(melt)
    gf = melt.GroupedFrontend(fes)
    clips, ids = G.mixed_groups(n=24, first=200)
    refs, outs = [], []
    for k in range(10):
        sub = list(range(k, 24 - (k % 3)))
        c = [clips[b] for b in sub]
        i = ids[sub]
        pk = G.pack_clips(c)
        wave = torch.from_numpy(pk.wave).cuda()
        outs.append(gf(wave, pk.offsets, pk.lengths, i).cpu().numpy())
        gf.sync()
        refs.append(_per_clip_reference(fes, c, i))
        assert np.array_equal(outs[-1], refs[-1]), k
    gf.close()
    for fe in fes:
        fe.close()


def test_grouped_rejects_bad_arguments(melt):
    import torch
    fes = _frontends(melt)
    gf = melt.GroupedFrontend(fes)
    clips, ids = G.mixed_groups(n=4)
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    out = torch.empty((gf.total_frames(pk.lengths, ids), 80), device="cuda")
    for bad in (np.array([0, 1, 2, 0], np.int32), np.array([0, -1, 0, 1], np.int32)):
        with pytest.raises(melt.MeltError) as ei:
            melt.melt_forward_grouped(gf.handle, wave, pk.offsets, pk.lengths, bad, out)
        assert ei.value.status == melt.MELT_ERR_ARG
    bad_off = pk.offsets.copy()
    bad_off[1] += 1                                   # not a multiple of 4 floats
    with pytest.raises(melt.MeltError):
        melt.melt_forward_grouped(gf.handle, wave, bad_off, pk.lengths, ids, out)
    gf.close()
    other = melt.Frontend(n_mels=40, precision="bf16")
    with pytest.raises(melt.MeltError) as ei:           # output widths differ
        melt.melt_group_create([fes[0], other])
    assert ei.value.status == melt.MELT_ERR_ARG
    other.close()
    for fe in fes:
        fe.close()


def test_group_autotune_and_plan_cache(melt, tmp_path):
    """melt_group_autotune times the grouped launch one basis at a time, keeps
    the chosen plans set, appends one cache line, and a later group of the same
    configurations reads the line back without timing.  The features under
    the tuned plans equal the per-group launches bit for bit, and a mixed
    FP32 + BF16 group tunes only the BF16 basis ("-" in the line)."""
    import torch
    clips, ids = G.mixed_groups(n=40)
    fes = _frontends(melt)
    ref = _per_clip_reference(fes, clips, ids)
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    path = str(tmp_path / "plans.txt")
    gf = melt.GroupedFrontend(fes)
    T = gf.total_frames(pk.lengths, ids)
    out = torch.empty((T, gf.n_out), device="cuda")
    gf(wave, pk.offsets, pk.lengths, ids, out=out)        # a cached layout and graph before tuning
    plans, hit = gf.autotune(wave, pk.offsets, pk.lengths, ids, out, path=path, reps=1)
    assert not hit and all(p is not None for p in plans)
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("melt-group-plan-v1 ")
    out.fill_(float("nan"))
    gf(wave, pk.offsets, pk.lengths, ids, out=out)        # captured anew with the tuned plans
    gf.sync()
    assert np.array_equal(out.cpu().numpy(), ref)
    gf.close()
    fes2 = _frontends(melt)
    gf2 = melt.GroupedFrontend(fes2)
    plans2, hit2 = gf2.autotune(wave, pk.offsets, pk.lengths, ids, out, path=path, reps=1)
    assert hit2 and plans2 == plans
    assert len(open(path).read().splitlines()) == 1
    out.fill_(float("nan"))
    gf2(wave, pk.offsets, pk.lengths, ids, out=out)
    gf2.sync()
    assert np.array_equal(out.cpu().numpy(), ref)
    gf2.close()
    for fe in fes + fes2:
        fe.close()
    mixed = _frontends(melt, ("fp32", "bf16"))
    gm = melt.GroupedFrontend(mixed)
    plans3, hit3 = gm.autotune(wave, pk.offsets, pk.lengths, ids, out, path=path, reps=1)
    assert not hit3 and plans3[0] is None and plans3[1] is not None
    last = open(path).read().splitlines()[-1]
    assert last.split(" : ")[1].startswith("- ")
    gm.close()
    for fe in mixed:
        fe.close()


@pytest.mark.parametrize("n,graphs", [(40, True), (7, False), (3, True)])
def test_shared_launch_equals_per_basis_launches(melt, n, graphs):
    """Two BF16 bases share one persistent launch (MELT_GROUP_SHARED; clusters
    split between them, each running its own layout; the 22.05 kHz basis
    takes a CTA-pair plan with its half basis streamed): bit for bit what one
    launch per basis gives, for batches large and small (a basis with a
    single tile), and at a set split."""
    import torch
    clips, ids = G.mixed_groups(n=n)
    fes = _frontends(melt)
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    outs = []
    for shared in (True, False):
        gf = melt.GroupedFrontend(fes, graphs=graphs, shared_launch=shared)
        T = gf.total_frames(pk.lengths, ids)
        out = torch.full((T, gf.n_out), float("nan"), device="cuda")
        for it in range(3):
            if shared and it == 2:
                melt.melt_group_set_split(gf.handle, 0.6)
            out.fill_(float("nan"))
            gf(wave, pk.offsets, pk.lengths, ids, out=out)
        gf.sync()
        outs.append(out.cpu().numpy())
        gf.close()
    assert not np.isnan(outs[0]).any()
    np.testing.assert_array_equal(outs[0], outs[1])
    ref = _per_clip_reference(fes, clips, ids)
    np.testing.assert_array_equal(outs[0], ref)
    for fe in fes:
        fe.close()


def test_shared_launch_follows_forced_plans(melt):
    """A forced single-CTA plan keeps the per-basis launches; a forced CTA-pair
    plan runs in the shared launch; both give the same bits."""
    import torch
    clips, ids = G.mixed_groups(n=12)
    fes = _frontends(melt)
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    ref = _per_clip_reference(fes, clips, ids)
    single = dict(basis_resident=0, a_buffers=2, prefetch_tiles=2, basis_slots=2, ksteps_per_slot=8, cta_pair=0,
                  schedule=0)
    pair = dict(basis_resident=0, a_buffers=2, prefetch_tiles=0, basis_slots=2, ksteps_per_slot=8, cta_pair=1,
                schedule=0)
    for pl in (single, pair):
        melt.melt_plan_set(fes[1].handle, pl)
        gf = melt.GroupedFrontend(fes, graphs=False, shared_launch=True)
        T = gf.total_frames(pk.lengths, ids)
        out = gf(wave, pk.offsets, pk.lengths, ids)
        gf.sync()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        gf.close()
    melt.melt_plan_set(fes[1].handle, None)
    for fe in fes:
        fe.close()
