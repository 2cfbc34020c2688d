"""Correction MLP on the GPU against the FP64 oracle (oracle/mlp_oracle.py).

* gradients of one batch (gathered rows) element by element;
* AdamW updates on the same gradients;
* one train step == gradient + AdamW;
* the fused inference kernel, and its in-place use behind melt_forward;
* training on MelT frames toward the STFT+Mel (Slaney) targets lowers the
  held-out error (the use the correction exists for).

Tolerances: every GPU quantity is an FP32 sum of at most 1024 products fed by
FP32 values that already carry a few units of roundoff; 1024 x 2^-24 x a few
stages is about 2e-4 of the largest magnitude in play, which is the bound used.
"""
import numpy as np
import pytest

from oracle import melt_oracle as O
from oracle import mlp_oracle as P
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


def _problem(n=1500, M=80, Hd=128, seed=3):
    g = np.random.default_rng(seed)
    x = (g.standard_normal((n, M)) * 3 - 8).astype(np.float32)
    tgt = (x * g.uniform(0.7, 1.3, M) + g.uniform(-2, 2, M) + 0.1 * g.standard_normal((n, M))).astype(np.float32)
    W1 = G.xavier_uniform(seed, Hd, M, 0)
    W2 = G.xavier_uniform(seed, M, Hd, 1)
    b1 = (0.1 * g.standard_normal(Hd)).astype(np.float32)
    b2 = (0.1 * g.standard_normal(M)).astype(np.float32)
    mu, sd = P.band_stats(x)
    return x, tgt, [W1, b1, W2, b2], mu.astype(np.float32), sd.astype(np.float32)


def _close(got, ref, what, rel=2e-4):
    ref = np.asarray(ref, np.float64)
    tol = rel * np.max(np.abs(ref)) + 1e-3 * np.abs(ref)
    bad = np.abs(np.asarray(got, np.float64) - ref) > tol
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - ref))), float(np.max(np.abs(ref))))


def test_gradients_match_oracle(melt):
    import torch
    M, Hd, B = 80, 128, 1024
    x, tgt, params, mu, sd = _problem(M=M, Hd=Hd)
    rows = np.random.default_rng(5).choice(x.shape[0], B, replace=False).astype(np.int64)
    h = melt.melt_mlp_create(M, Hd, melt.pack_mlp_params(*params), mu, sd)
    X = torch.from_numpy(x).cuda()
    T = torch.from_numpy(tgt).cuda()
    R = torch.from_numpy(rows).cuda()
    grads = torch.zeros(melt.melt_mlp_num_params(M, Hd), device="cuda")
    loss = torch.zeros(1, device="cuda")
    melt.melt_mlp_grad(h, X, T, R, B, grads, loss)
    torch.cuda.synchronize()
    p64 = [np.asarray(p, np.float64) for p in params]
    y, cache = P.forward(p64, x[rows], mu.astype(np.float64), sd.astype(np.float64))
    ref = P.backward(p64, cache, y, tgt[rows], sd.astype(np.float64))
    got = melt.unpack_mlp_params(grads.cpu().numpy(), M, Hd)
    for name, gg, rr in zip(["dW1", "db1", "dW2", "db2"], got, ref[:4]):
        _close(gg, rr, name)
    sse = float(np.sum((y - tgt[rows]) ** 2))
    assert loss.item() == pytest.approx(sse, rel=1e-4)
    melt.melt_mlp_destroy(h)


def test_gradients_identity_rows_and_small_batch(melt):
    import torch
    M, Hd, B = 40, 64, 37                        # ragged against the 64 x 64 tiles
    x, tgt, params, mu, sd = _problem(n=37, M=M, Hd=Hd, seed=9)
    h = melt.melt_mlp_create(M, Hd, melt.pack_mlp_params(*params), mu, sd)
    grads = torch.zeros(melt.melt_mlp_num_params(M, Hd), device="cuda")
    melt.melt_mlp_grad(h, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(), None, B, grads)
    torch.cuda.synchronize()
    p64 = [np.asarray(p, np.float64) for p in params]
    y, cache = P.forward(p64, x, mu.astype(np.float64), sd.astype(np.float64))
    ref = P.backward(p64, cache, y, tgt, sd.astype(np.float64))
    for name, gg, rr in zip(["dW1", "db1", "dW2", "db2"], melt.unpack_mlp_params(grads.cpu().numpy(), M, Hd),
                            ref[:4]):
        _close(gg, rr, name)
    melt.melt_mlp_destroy(h)


def test_adamw_matches_oracle_and_train_step_composes(melt):
    import torch
    M, Hd, B = 80, 64, 256
    x, tgt, params, mu, sd = _problem(n=700, M=M, Hd=Hd, seed=11)
    packed = melt.pack_mlp_params(*params)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda()
    ha = melt.melt_mlp_create(M, Hd, packed, mu, sd)        # grad + adamw_apply
    hb = melt.melt_mlp_create(M, Hd, packed, mu, sd)        # train_step
    lr, wd = 3e-3, 0.02
    for hh in (ha, hb):
        melt.melt_mlp_set_adamw(hh, lr=lr, wd=wd)
    n = packed.size
    p_ref = [np.asarray(p, np.float64) for p in params]
    st = [(np.zeros_like(p), np.zeros_like(p)) for p in p_ref]
    grads = torch.zeros(n, device="cuda")
    order = G.batch_order(1, x.shape[0], 0)
    for t in range(1, 6):
        rows = torch.from_numpy(order[(t - 1) * 100:(t - 1) * 100 + B].copy()).cuda()
        melt.melt_mlp_grad(ha, X, T, rows, B, grads)
        g_host = grads.cpu().numpy().astype(np.float64)
        melt.melt_mlp_adamw_apply(ha, grads)
        melt.melt_mlp_train_step(hb, X, T, rows, B)
        # oracle AdamW on the very gradients the GPU used
        gsplit = melt.unpack_mlp_params(g_host, M, Hd)
        for i in range(4):
            p_ref[i], m, v = P.adamw_step(p_ref[i], gsplit[i], st[i][0], st[i][1], t, lr=lr, wd=wd)
            st[i] = (m, v)
        pa = melt.melt_mlp_get_params(ha, M, Hd)[0]
        pr = np.concatenate([p.reshape(-1) for p in p_ref])
        assert np.max(np.abs(pa - pr)) <= 2e-6 * (1 + np.max(np.abs(pr))), t
        pb = melt.melt_mlp_get_params(hb, M, Hd)[0]
        assert np.array_equal(pa, pb), t
        # continue the oracle from the GPU's parameters so later steps compare the update alone
        p_ref = [np.asarray(a, np.float64) for a in melt.unpack_mlp_params(pa.astype(np.float64), M, Hd)]
    melt.melt_mlp_destroy(ha)
    melt.melt_mlp_destroy(hb)


def test_forward_kernel_and_in_place(melt):
    import torch
    for M, Hd, n in [(80, 256, 1000), (128, 64, 130), (13, 128, 65), (80, 256, 1)]:
        x, tgt, params, mu, sd = _problem(n=n, M=M, Hd=Hd, seed=M + Hd)
        h = melt.melt_mlp_create(M, Hd, melt.pack_mlp_params(*params), mu, sd)
        X = torch.from_numpy(x).cuda()
        Y = torch.empty_like(X)
        melt.melt_mlp_forward(h, X, Y, n)
        p64 = [np.asarray(p, np.float64) for p in params]
        ref, _ = P.forward(p64, x, mu.astype(np.float64), sd.astype(np.float64))
        got = Y.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref)), (M, Hd, n)
        melt.melt_mlp_forward(h, X, X, n)                  # in place
        assert np.array_equal(X.cpu().numpy(), got)
        melt.melt_mlp_destroy(h)


def test_fit_stats(melt):
    import torch
    x = (np.random.default_rng(2).standard_normal((5000, 80)) * 4 - 7).astype(np.float32)
    x[:, 3] = 2.5                                          # constant band: sd floor
    mu, sd = P.band_stats(x.astype(np.float64))
    h = melt.melt_mlp_create(80, 64, np.zeros(melt.melt_mlp_num_params(80, 64), np.float32))
    melt.melt_mlp_fit_stats(h, torch.from_numpy(x).cuda(), x.shape[0])
    _, m, s = melt.melt_mlp_get_params(h, 80, 64)
    np.testing.assert_allclose(m, mu, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(s, sd, rtol=1e-5, atol=1e-6)
    assert s[3] == pytest.approx(1e-6)
    melt.melt_mlp_destroy(h)


def test_correction_behind_melt_forward(melt):
    import torch
    clips = [G.rich_clip(71, i, 16000 * 2 + 37 * i) for i in range(5)]
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    M, Hd = 80, 128
    _, _, params, mu, sd = _problem(n=10, M=M, Hd=Hd, seed=4)
    mlp = melt.melt_mlp_create(M, Hd, melt.pack_mlp_params(*params), mu, sd)
    for prec in ["fp32", "bf16"]:
        fe = melt.Frontend(precision=prec)
        plain = fe(wave, pk.offsets, pk.lengths)
        T = plain.shape[0]
        ref = torch.empty_like(plain)
        melt.melt_mlp_forward(mlp, plain, ref, T)
        melt.melt_basis_set_correction(fe.handle, mlp)
        got = fe(wave, pk.offsets, pk.lengths)
        got2 = torch.empty_like(got)
        melt.melt_forward_noalloc(fe.handle, wave, pk.offsets, pk.lengths, got2)
        fe.sync()
        assert torch.equal(got2, got), prec
        if prec == "fp32":   # separate FP32 pass after the kernel: the FP32 MLP exactly
            assert torch.equal(got, ref)
        else:                # fused in the BF16 epilogue (BF16 operands, FP32 sums)
            assert melt.melt_plan_get(fe.handle)["cta_pair"] == 1
            assert float((got - ref).abs().max()) < 0.1, float((got - ref).abs().max())
        gf = melt.GroupedFrontend([fe])
        with pytest.raises(melt.MeltError) as ei:
            gf(wave, pk.offsets, pk.lengths, np.zeros(len(clips), np.int32))
        assert ei.value.status == melt.MELT_ERR_UNSUPPORTED
        gf.close()
        melt.melt_basis_set_correction(fe.handle, None)
        assert torch.equal(fe(wave, pk.offsets, pk.lengths), plain)
        fe.close()
    mf = melt.Frontend(precision="bf16", n_mfcc=40)
    with pytest.raises(melt.MeltError) as ei:
        melt.melt_basis_set_correction(mf.handle, mlp)
    assert ei.value.status == melt.MELT_ERR_UNSUPPORTED
    mf.close()
    melt.melt_mlp_destroy(mlp)


def test_learned_correction_synthetic_config(melt):
    """The learned correction at the scale of the synthetic workload: ~200k training frames of
    the generator (201 clips of 10 s), AdamW (lr 1e-3, betas 0.9/0.999, weight decay 0.01),
    batches of 1024, 20 epochs, inputs the FP32 MelT features and targets the oracle's
    STFT(400, 160, Hann) + Slaney 80-band log-Mel; evaluated on 512 held-out 10 s clips by
    cosine, CCC and RMSE (dB) against the oracle, for plain BF16 MelT, the BF16 kernel with
    the correction fused in its epilogue, and FP32 MelT with the separate FP32 pass."""
    import torch
    spec = O.MelTSpec(sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0)
    train = [G.rich_clip(101, i, 160000) for i in range(201)]
    held = [G.rich_clip(102, i, 160000) for i in range(512)]
    f32 = melt.Frontend(precision="fp32")
    bf = melt.Frontend(precision="bf16")

    def feats(fe, clips):
        pk = G.pack_clips(clips)
        out = fe(torch.from_numpy(pk.wave).cuda(), pk.offsets, pk.lengths)
        fe.sync()
        return out

    Xtr = feats(f32, train)
    Ttr = torch.from_numpy(np.concatenate([O.stft_mel_clip(c, spec, scale="slaney") for c in train])
                           .astype(np.float32)).cuda()
    n = Xtr.shape[0]
    assert n >= 200_000
    M, Hd, B = 80, 256, 1024
    params = melt.pack_mlp_params(G.xavier_uniform(7, Hd, M, 0), np.zeros(Hd), G.xavier_uniform(7, M, Hd, 1),
                                  np.zeros(M))
    mlp = melt.melt_mlp_create(M, Hd, params)
    melt.melt_mlp_fit_stats(mlp, Xtr, n)
    melt.melt_mlp_set_adamw(mlp, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01)
    loss = torch.zeros(1, device="cuda")
    for ep in range(20):
        order = torch.from_numpy(G.batch_order(7, n, ep)).cuda()
        if ep == 19:
            loss.zero_()
        for s in range(0, n - B + 1, B):
            melt.melt_mlp_train_step(mlp, Xtr, Ttr, order[s:s + B], B, loss if ep == 19 else None)
    last_epoch_mse = float(loss.item()) / ((n // B) * B * M)
    ref = [O.stft_mel_clip(c, spec, scale="slaney") for c in held]
    rows = np.cumsum([0] + [r.shape[0] for r in ref])

    def clips_of(out):
        a = out.cpu().numpy().astype(np.float64)
        return [a[rows[i]:rows[i + 1]] for i in range(len(held))]

    plain = clips_of(feats(bf, held))
    melt.melt_basis_set_correction(bf.handle, mlp)
    assert melt.melt_plan_get(bf.handle)["cta_pair"] == 1           # fused in the epilogue
    fused = clips_of(feats(bf, held))
    melt.melt_basis_set_correction(f32.handle, mlp)
    sep = clips_of(feats(f32, held))
    r = {name: O.fidelity(list(zip(v, ref))) for name, v in
         [("plain_bf16", plain), ("fused_bf16", fused), ("separate_fp32", sep)]}
    print(f"\nheld-out 512 x 10 s vs oracle STFT + Slaney-Mel (last-epoch train MSE {last_epoch_mse:.4f} nat^2):")
    for name, m in r.items():
        print(f"  {name:14s} cosine {m['cosine']:.4f}  CCC {m['ccc']:.4f}  RMSE {m['rmse_db']:.2f} dB")
    assert r["fused_bf16"]["rmse_db"] < 0.5 * r["plain_bf16"]["rmse_db"]
    assert r["fused_bf16"]["cosine"] > r["plain_bf16"]["cosine"]
    assert r["fused_bf16"]["ccc"] > r["plain_bf16"]["ccc"]
    assert abs(r["fused_bf16"]["rmse_db"] - r["separate_fp32"]["rmse_db"]) < 0.1
    for fe in (f32, bf):
        melt.melt_basis_set_correction(fe.handle, None)
        fe.close()
    melt.melt_mlp_destroy(mlp)


def _fused_case(melt, seed, lens, Hd=256, M=80):
    import torch
    clips = [G.rich_clip(seed, i, L) for i, L in enumerate(lens)]
    pk = G.pack_clips(clips)
    wave = torch.from_numpy(pk.wave).cuda()
    fe = melt.Frontend(precision="bf16", n_mels=M)
    x = fe(wave, pk.offsets, pk.lengths)
    fe.sync()
    x = x.cpu().numpy().astype(np.float64)
    mu, sd = P.band_stats(x)
    g = np.random.default_rng(seed)
    params = [G.xavier_uniform(seed, Hd, M, 0), (0.2 * g.standard_normal(Hd)).astype(np.float32),
              G.xavier_uniform(seed, M, Hd, 1), (0.2 * g.standard_normal(M)).astype(np.float32)]
    mu32, sd32 = mu.astype(np.float32), sd.astype(np.float32)
    mlp = melt.melt_mlp_create(M, Hd, melt.pack_mlp_params(*params), mu32, sd32)
    return fe, mlp, pk, wave, x, params, mu32.astype(np.float64), sd32.astype(np.float64)


def test_fused_gelu_error_bound(melt):
    """The fused epilogue's GELU against the exact h Phi(h) (FP64) on a fine grid
    over [-12, 12] and on random values: relative error <= 2e-5 for |h| <= 5,
    absolute error <= 3e-6 everywhere (the stated bound)."""
    import torch
    g = np.random.default_rng(17)
    h = np.concatenate([np.linspace(-12, 12, 2_400_001), g.standard_normal(200000) * 3,
                        np.array([0.0, -0.0, 1e-30, -1e-30, 5.0, -5.0, 4.9999, -5.0001])]).astype(np.float32)
    ht = torch.from_numpy(h).cuda()
    y = torch.empty_like(ht)
    melt.melt_diag_gelu(ht, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    exact = P.gelu(h.astype(np.float64))
    err = np.abs(got - exact)
    assert err.max() <= 3e-6, float(err.max())
    inner = (np.abs(h) <= 5) & (exact != 0)
    rel = err[inner] / np.abs(exact[inner])
    assert rel.max() <= 2e-5, float(rel.max())
    print(f"fused GELU: max abs {err.max():.2e}, max rel (|h| <= 5) {rel.max():.2e}")


def _fused_bound(params, x, mu, sd):
    """Oracle with the fused path's BF16 operand rounding, and a bound on the GPU's distance to it.

    The GPU sums in FP32 (x-hat: 80 terms, the hidden layer: 256) and rounds
    x-hat and GELU(h) to bfloat16 after FP32 arithmetic; where that lands on
    the other side of a bfloat16 rounding boundary the operand moves by one
    bfloat16 ulp (2^-8 relative).  Allowing that for every operand:
      |dh_j| <= 2^-8 sum_m |W1b[j,m] xh_m| + 100 u sum_m |W1b xh| + u |b1_j|
      |da_j| <= 1.13 |dh_j| + 2^-8 |a_j|          (|GELU'| <= 1.13)
      |dy_o| <= sum_j |W2b[o,j]| |da_j| + 300 u (|x_o| + sum_j |W2b a| + |b2_o|)
    with u = 2^-24; the log-Mel x itself is the kernel's (same value both ways).
    """
    y, (xh_b, h, a_b, W1_b, W2_b) = P.forward_bf16(params, x, mu, sd)
    u = 2.0 ** -24
    s1 = np.abs(xh_b) @ np.abs(W1_b).T
    dh = 2.0 ** -8 * s1 + 100 * u * s1 + u * np.abs(np.asarray(params[1], np.float64))
    # GELU(h + b1) itself: the epilogue's polynomial form (relative error <= 2e-5
    # for |h| <= 5, absolute <= 3e-6) before its BF16 rounding
    da = 1.13 * dh + (2.0 ** -8 + 2e-5) * np.abs(a_b) + 3e-6
    s2 = np.abs(a_b) @ np.abs(W2_b).T
    bound = da @ np.abs(W2_b).T + 300 * u * (np.abs(x) + s2 + np.abs(np.asarray(params[3], np.float64)))
    return y, bound


@pytest.mark.parametrize("lens", [[16000 * 3 + 97 * i for i in range(7)],          # odd tile count
                                  [400, 128 * 160 + 240, 3 * 16000, 129 * 160 + 240, 401]])
def test_fused_correction_matches_bf16_oracle(melt, lens):
    """The correction fused in the BF16 pair kernel's epilogue against the FP64 oracle with
    the same BF16 operand rounding, element by element; the allocation-free and host-buffer
    entry points give the same bits."""
    import torch
    fe, mlp, pk, wave, x, params, mu, sd = _fused_case(melt, 91, lens)
    melt.melt_basis_set_correction(fe.handle, mlp)
    assert melt.melt_plan_get(fe.handle)["cta_pair"] == 1
    got = fe(wave, pk.offsets, pk.lengths)
    got_na = torch.empty_like(got)
    melt.melt_forward_noalloc(fe.handle, wave, pk.offsets, pk.lengths, got_na)
    fe.sync()
    got = got.cpu().numpy()
    assert np.array_equal(got_na.cpu().numpy(), got)
    host = torch.empty(got.shape, dtype=torch.float32).pin_memory()
    melt.melt_forward_host(fe.handle, torch.from_numpy(pk.wave).pin_memory(), pk.offsets, pk.lengths, host)
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy(), got)
    y_ref, bound = _fused_bound(params, x, mu, sd)
    err = np.abs(got - y_ref)
    assert np.all(err <= bound), (float(err.max()), int((err > bound).sum()))
    # the typical error is far below the worst-case bound
    assert float(np.sqrt(np.mean(err ** 2))) < 0.1 * float(np.mean(bound))
    # and the MLP changes the features substantially, so the comparison is not vacuous
    assert float(np.abs(y_ref - x).mean()) > 50 * float(np.sqrt(np.mean(err ** 2)))
    melt.melt_basis_set_correction(fe.handle, None)
    fe.close()
    melt.melt_mlp_destroy(mlp)


def test_fused_correction_follows_training_and_hidden_sizes(melt):
    """Parameters updated by training reach the fused epilogue on the next forward; a smaller
    hidden layer is fused too, and one too small to hold the output beside GELU(H) in TMEM
    (Hd < 2 x 80) falls back to the separate FP32 pass."""
    import torch
    fe, mlp, pk, wave, x, params, mu, sd = _fused_case(melt, 94, [16000 * 2, 16000 * 3], Hd=64)
    melt.melt_basis_set_correction(fe.handle, mlp)
    plain = torch.from_numpy(x.astype(np.float32)).cuda()
    ref = torch.empty_like(plain)
    melt.melt_mlp_forward(mlp, plain, ref, x.shape[0])
    got = fe(wave, pk.offsets, pk.lengths)
    fe.sync()
    assert torch.equal(got, ref)
    fe.close()
    melt.melt_mlp_destroy(mlp)
    for Hd in (256, 192):
        fe, mlp, pk, wave, x, params, mu, sd = _fused_case(melt, 93, [16000 * 2, 16000 * 3], Hd=Hd)
        melt.melt_basis_set_correction(fe.handle, mlp)
        assert melt.melt_plan_get(fe.handle)["cta_pair"] == 1, Hd
        X = torch.from_numpy(x.astype(np.float32)).cuda()
        T = torch.from_numpy((x * 0.9 + 0.3).astype(np.float32)).cuda()
        for _ in range(3):
            melt.melt_mlp_train_step(mlp, X, T, None, x.shape[0])
        trained = melt.unpack_mlp_params(melt.melt_mlp_get_params(mlp, 80, Hd)[0].astype(np.float64), 80, Hd)
        got = fe(wave, pk.offsets, pk.lengths)
        fe.sync()
        y_ref, bound = _fused_bound(trained, x, mu, sd)
        err = np.abs(got.cpu().numpy() - y_ref)
        assert np.all(err <= bound), (Hd, float(err.max()))
        fe.close()
        melt.melt_mlp_destroy(mlp)


@pytest.mark.parametrize("M,Hd", [(16, 64), (40, 192), (64, 128)])
def test_fused_correction_other_band_and_hidden_counts(melt, M, Hd):
    """Band and hidden-unit counts whose runs over the three epilogue warps of a lane
    quarter are uneven or empty: M = 16 (one band chunk: two warps have no bands), 40
    (three chunks) and 64 (four), with 4, 12 and 8 hidden chunks; the fused epilogue
    against the FP64 oracle with the same BF16 operand rounding, element by element."""
    fe, mlp, pk, wave, x, params, mu, sd = _fused_case(melt, 95, [16000 * 2 + 321, 16000 * 3, 400], Hd=Hd, M=M)
    melt.melt_basis_set_correction(fe.handle, mlp)
    assert melt.melt_plan_get(fe.handle)["cta_pair"] == 1
    got = fe(wave, pk.offsets, pk.lengths)
    fe.sync()
    got = got.cpu().numpy()
    assert got.shape == x.shape
    y_ref, bound = _fused_bound(params, x, mu, sd)
    err = np.abs(got - y_ref)
    assert np.all(err <= bound), (M, Hd, float(err.max()), int((err > bound).sum()))
    assert float(np.abs(y_ref - x).mean()) > 50 * float(np.sqrt(np.mean(err ** 2)))
    melt.melt_basis_set_correction(fe.handle, None)
    fe.close()
    melt.melt_mlp_destroy(mlp)
