"""Layout plans of the tensor-core pipeline: melt_plan_get / melt_plan_set / melt_autotune.

A plan changes only where operands sit in shared memory and how they are
copied there; every plan issues the same MMAs in the same k order into the
same accumulator, so every plan must give bit-identical output.
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


def _plans():
    out = []
    for zb, pf in ((1, 0), (2, 2), (2, 4)):
        out.append(dict(basis_resident=1, a_buffers=zb, prefetch_tiles=pf, basis_slots=0, ksteps_per_slot=1,
                        cta_pair=0))
    for pf, nb, kps in [(0, 2, 1), (1, 3, 2), (2, 2, 5), (2, 2, 8), (3, 2, 9), (2, 6, 1), (2, 2, 30)]:
        out.append(dict(basis_resident=0, a_buffers=2, prefetch_tiles=pf, basis_slots=nb, ksteps_per_slot=kps,
                        cta_pair=0))
    out.append(dict(basis_resident=0, a_buffers=1, prefetch_tiles=2, basis_slots=12, ksteps_per_slot=1, cta_pair=0))
    for zb, pf, sched in ((1, 0, 0), (2, 0, 0), (2, 1, 0), (2, 2, 0), (2, 0, 1), (1, 0, 1)):
        # CTA pairs (BF16 and FP8): half of the basis per CTA, 2-SM MMAs; static
        # or dynamic pair schedule
        out.append(dict(basis_resident=1, a_buffers=zb, prefetch_tiles=pf, basis_slots=0, ksteps_per_slot=1,
                        cta_pair=1, schedule=sched))
    for zb, pf, nb, kps in ((2, 0, 4, 4), (2, 1, 2, 1), (1, 0, 3, 8), (2, 2, 4, 2), (1, 1, 2, 16)):
        # CTA pairs with each CTA's half basis streamed through slots (BF16, split BF16)
        out.append(dict(basis_resident=0, a_buffers=zb, prefetch_tiles=pf, basis_slots=nb, ksteps_per_slot=kps,
                        cta_pair=1, schedule=0))
    return out


def _batch():
    import torch
    lens = [0, 401, 128 * 160 + 240, 129 * 160 + 240, 48000, 300 * 160 + 397, 160000]
    clips = [G.rich_clip(77, i, L) if L >= 16 else np.zeros(L, np.float32) for i, L in enumerate(lens)]
    pk = G.pack_clips(clips)
    return pk, torch.from_numpy(pk.wave).cuda()


@pytest.mark.parametrize("prec,n_mels", [("bf16", 80), ("bf16", 128), ("fp8", 80), ("bf16x3", 40)])
def test_every_plan_is_bit_identical(melt, prec, n_mels):
    import torch
    pk, wave = _batch()
    fe = melt.Frontend(precision=prec, n_mels=n_mels)
    T = fe.total_frames(pk.lengths)
    ref = fe(wave, pk.offsets, pk.lengths).cpu().numpy()
    fe.sync()
    default = melt.melt_plan_get(fe.handle)
    tried = 0
    for pl in _plans():
        try:
            melt.melt_plan_set(fe.handle, pl)
        except melt.MeltError as e:
            assert e.status == melt.MELT_ERR_UNSUPPORTED
            continue
        got = torch.full((T, fe.n_out), float("nan"), device="cuda")
        fe(wave, pk.offsets, pk.lengths, out=got)
        fe.sync()
        assert np.array_equal(got.cpu().numpy(), ref), (prec, n_mels, pl)
        tried += 1
    assert tried >= 2, (prec, n_mels)
    melt.melt_plan_set(fe.handle, None)
    assert melt.melt_plan_get(fe.handle) == default
    fe.close()


def test_plan_round_trip_and_rejections(melt):
    fe = melt.Frontend(precision="bf16")
    pl = dict(basis_resident=0, a_buffers=2, prefetch_tiles=3, basis_slots=3, ksteps_per_slot=4, cta_pair=0,
              schedule=0)
    melt.melt_plan_set(fe.handle, pl)
    assert melt.melt_plan_get(fe.handle) == pl
    pair = dict(basis_resident=1, a_buffers=2, prefetch_tiles=0, basis_slots=0, ksteps_per_slot=1, cta_pair=1,
                schedule=1)
    for bad in [dict(pl, a_buffers=3), dict(pl, prefetch_tiles=-1), dict(pl, prefetch_tiles=5),
                dict(pl, basis_slots=1), dict(pl, ksteps_per_slot=0),
                dict(pl, basis_slots=32, ksteps_per_slot=40), dict(pl, cta_pair=2),
                dict(pl, cta_pair=1, schedule=1),   # a streamed half basis needs the static schedule
                dict(pl, cta_pair=1, basis_slots=9),  # at most 8 slots
                dict(pl, schedule=1),           # the dynamic schedule is for CTA pairs only
                dict(pair, schedule=2), dict(pair, schedule=-1)]:
        with pytest.raises(melt.MeltError) as ei:
            melt.melt_plan_set(fe.handle, bad)
        assert ei.value.status == melt.MELT_ERR_UNSUPPORTED
    assert melt.melt_plan_get(fe.handle) == pl      # a rejected plan leaves the current one
    fe.close()
    f32 = melt.Frontend(precision="fp32")
    with pytest.raises(melt.MeltError) as ei:
        melt.melt_plan_get(f32.handle)
    assert ei.value.status == melt.MELT_ERR_UNSUPPORTED
    f32.close()


def test_autotune_keeps_output(melt):
    import torch
    pk, wave = _batch()
    fe = melt.Frontend(precision="bf16")
    T = fe.total_frames(pk.lengths)
    ref = fe(wave, pk.offsets, pk.lengths).cpu().numpy()
    out = torch.empty((T, fe.n_out), device="cuda")
    best = melt.melt_autotune(fe.handle, wave, pk.offsets, pk.lengths, out, reps=2)
    assert melt.melt_plan_get(fe.handle) == best
    got = fe(wave, pk.offsets, pk.lengths).cpu().numpy()
    fe.sync()
    assert np.array_equal(got, ref)
    fe.close()


def _ragged_batch(n_clips, seed):
    """Clips of 0.2 to 30 s (log-uniform) with an odd total tile count."""
    rng = np.random.default_rng(seed)
    lens = np.exp(rng.uniform(np.log(3200), np.log(480000), size=n_clips)).astype(np.int64)
    tiles = lambda L: -(-max(0, (int(L) - 400) // 160 + 1) // 128) if L >= 400 else 0
    if sum(tiles(L) for L in lens) % 2 == 0:
        lens[0] = 400 + 160 * 10   # one more single-tile clip makes the count odd
    return [G.rich_clip(seed, i, int(L)) for i, L in enumerate(lens)]


@pytest.mark.parametrize("batch", ["rich_64x30s", "ragged_300"])
def test_dynamic_pair_schedule_matches_static(melt, batch):
    """Dynamic and static pair schedules give the same features, launch after launch.

    The batches hold several rounds of pairs per cluster, so most pairs are
    claimed from the launch counter; back-to-back launches check that every
    launch leaves its counter at zero for the next one that uses it, and
    launches on two unordered streams that concurrent launches do not share
    a counter.
    """
    import torch
    clips = G.workload("rich_64x30s")[0] if batch == "rich_64x30s" else _ragged_batch(300, 99)
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    fe = melt.Frontend(precision="bf16")
    T = fe.total_frames(pk.lengths)
    base = dict(basis_resident=1, a_buffers=2, prefetch_tiles=0, basis_slots=0, ksteps_per_slot=1, cta_pair=1)
    melt.melt_plan_set(fe.handle, dict(base, schedule=0))
    ref = fe(wave, pk.offsets, pk.lengths).cpu().numpy()
    fe.sync()
    melt.melt_plan_set(fe.handle, dict(base, schedule=1))
    outs = [torch.full((T, fe.n_out), float("nan"), device="cuda") for _ in range(3)]
    for i in range(7):
        fe(wave, pk.offsets, pk.lengths, out=outs[i % 3])
    fe.sync()
    for o in outs:
        assert np.array_equal(o.cpu().numpy(), ref), batch
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for o in outs[:2]:
        o.fill_(float("nan"))
    torch.cuda.synchronize()
    for s, o in zip(streams, outs[:2]):
        fe(wave, pk.offsets, pk.lengths, out=o, stream=s)
    for s in streams:
        fe.sync(s)
    for o in outs[:2]:
        assert np.array_equal(o.cpu().numpy(), ref), batch
    fe.close()


def test_autotune_file_cache(melt, tmp_path):
    """melt_autotune_file tunes on a miss and appends one line; a second basis
    of the same configuration and batch size class reads that line back
    without timing; lines of other GPUs, other configurations or a malformed
    plan are skipped; the output under the cached plan equals the default's."""
    import torch
    pk, wave = _batch()
    path = str(tmp_path / "plans.txt")
    with open(path, "w") as f:     # lines that must not match
        f.write("melt-plan-v1 Some_Other_GPU 400 160 80 1 0 0 0 0 : 1 2 1 2 1 0 0\n")
        f.write("not a plan line\n")
    fe = melt.Frontend(precision="bf16")
    T = fe.total_frames(pk.lengths)
    ref = fe(wave, pk.offsets, pk.lengths).cpu().numpy()
    out = torch.empty((T, fe.n_out), device="cuda")
    best, hit = melt.melt_autotune_file(fe.handle, wave, pk.offsets, pk.lengths, out, path, reps=2)
    assert not hit
    assert melt.melt_plan_get(fe.handle) == best
    lines = open(path).read().splitlines()
    assert len(lines) == 3 and lines[-1].startswith("melt-plan-v1 ")
    fe.close()
    fe2 = melt.Frontend(precision="bf16")
    best2, hit2 = melt.melt_autotune_file(fe2.handle, wave, pk.offsets, pk.lengths, out, path, reps=2)
    assert hit2 and best2 == best
    assert melt.melt_plan_get(fe2.handle) == best
    assert len(open(path).read().splitlines()) == 3
    got = fe2(wave, pk.offsets, pk.lengths).cpu().numpy()
    fe2.sync()
    assert np.array_equal(got, ref)
    fe2.close()
    # another configuration (128 Mel bins) misses and appends its own line
    fe3 = melt.Frontend(precision="bf16", n_mels=128)
    out3 = torch.empty((fe3.total_frames(pk.lengths), 128), device="cuda")
    _, hit3 = melt.melt_autotune_file(fe3.handle, wave, pk.offsets, pk.lengths, out3, path, reps=1)
    assert not hit3 and len(open(path).read().splitlines()) == 4
    fe3.close()
