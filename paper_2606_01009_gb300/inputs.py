"""Seeded synthetic inputs for the MelT hot path.

This module only *draws* inputs: waveforms, clip lengths, packing offsets,
initial MLP weights and batch orders.  It contains none of the MelT
arithmetic (no Mel scale, window, basis, projection, power, log or DCT), so
both the CPU oracle side (tests, bench baseline) and the CUDA side can take
their inputs from it without sharing any of the method's code.

The paper measures on LibriSpeech speech (Sec. IV-A, "Datasets and
Sampling"); that corpus is not available here, so these generators stand in
for it with the same sample rates, durations and batch shapes.  Signal
recipe (all seeded, float64 synthesis, returned as float32):

* ``tones``: 1-4 sinusoids, f ~ U[50, 7500] Hz, amplitude ~ U[0.1, 0.5],
  random phase, plus white Gaussian noise whose RMS is -30 dBFS
  (full scale = 1.0).
* ``rich``: pink-noise bed plus amplitude-modulated bursts (Hann envelope,
  0.08-0.8 s) of exponential chirps (start/end ~ log-U[50, 7500] Hz) and
  harmonic stacks (f0 ~ U[80, 400] Hz, harmonics up to 7.5 kHz with 1/h
  amplitudes), about 3 bursts per second, peak-normalised to +-1 and then
  scaled to a peak level in dBFS (0 dBFS unless a level is given).

Random numbers come from numpy's PCG64 seeded with ``(seed, stream, index)``
so that clip ``i`` of a workload is the same whatever batch it is drawn in.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng_for",
    "tones_clip",
    "rich_clip",
    "loguniform_lengths",
    "pack_clips",
    "PackedBatch",
    "workload",
    "mixed_groups",
    "MIXED_GROUPS",
    "xavier_uniform",
    "batch_order",
]

_STREAM_TONES = 1
_STREAM_RICH = 2
_STREAM_LEN = 3
_STREAM_LEVEL = 4
_STREAM_MLP = 5
_STREAM_ORDER = 6


def rng_for(seed: int, stream: int, index: int = 0) -> np.random.Generator:
    """Independent PCG64 stream for (seed, stream, index)."""
    return np.random.Generator(np.random.PCG64([int(seed), int(stream), int(index)]))


def tones_clip(seed: int, index: int, length: int = 16000, sr: float = 16000.0,
               noise_dbfs: float = -30.0) -> np.ndarray:
    """Sum of 1-4 random sinusoids plus white noise at ``noise_dbfs`` RMS."""
    g = rng_for(seed, _STREAM_TONES, index)
    n = np.arange(length, dtype=np.float64)
    k = int(g.integers(1, 5))
    x = np.zeros(length, dtype=np.float64)
    for _ in range(k):
        f = g.uniform(50.0, 7500.0)
        a = g.uniform(0.1, 0.5)
        ph = g.uniform(0.0, 2.0 * math.pi)
        x += a * np.cos(2.0 * math.pi * f / sr * n + ph)
    x += (10.0 ** (noise_dbfs / 20.0)) * g.standard_normal(length)
    return x.astype(np.float32)


def _pink(g: np.random.Generator, length: int) -> np.ndarray:
    """White Gaussian noise shaped to a 1/f power spectrum (unit RMS)."""
    nfft = 1 << max(4, int(math.ceil(math.log2(max(length, 2)))))
    spec = g.standard_normal(nfft // 2 + 1) + 1j * g.standard_normal(nfft // 2 + 1)
    k = np.arange(nfft // 2 + 1, dtype=np.float64)
    k[0] = 1.0
    spec /= np.sqrt(k)
    spec[0] = 0.0
    y = np.fft.irfft(spec, nfft)[:length]
    rms = math.sqrt(float(np.mean(y * y))) or 1.0
    return y / rms


def _hann_env(n: int) -> np.ndarray:
    if n <= 1:
        return np.ones(max(n, 0))
    return 0.5 - 0.5 * np.cos(2.0 * math.pi * np.arange(n) / (n - 1))


def _harmonic_table(g: np.random.Generator, f0: float, sr: float, size: int = 4096) -> np.ndarray:
    """One period of sum_h (1/h) sin(2 pi h u + phi_h), h*f0 <= 7.5 kHz."""
    hmax = max(1, min(size // 2 - 1, int(7500.0 // f0)))
    spec = np.zeros(size // 2 + 1, dtype=np.complex128)
    h = np.arange(1, hmax + 1)
    spec[1:hmax + 1] = (1.0 / h) * np.exp(1j * g.uniform(0, 2 * math.pi, hmax))
    tab = np.fft.irfft(spec, size) * size / 2.0
    return np.concatenate([tab, tab[:1]])


def rich_clip(seed: int, index: int, length: int, sr: float = 16000.0,
              level_dbfs: float = 0.0, burst_rate: float = 3.0) -> np.ndarray:
    """Chirps + harmonic stacks as AM bursts over pink noise; peak at ``level_dbfs``."""
    g = rng_for(seed, _STREAM_RICH, index)
    x = _pink(g, length) * (10.0 ** (g.uniform(-40.0, -20.0) / 20.0))
    dur = length / sr
    n_ev = max(1, int(g.poisson(burst_rate * dur)))
    for _ in range(n_ev):
        blen = int(g.uniform(0.08, 0.8) * sr)
        blen = max(16, min(blen, length))
        start = int(g.integers(0, max(1, length - blen + 1)))
        amp = g.uniform(0.2, 1.0)
        env = _hann_env(blen) * amp
        t = np.arange(blen, dtype=np.float64) / sr
        if g.uniform() < 0.5:
            f1 = math.exp(g.uniform(math.log(50.0), math.log(7500.0)))
            f2 = math.exp(g.uniform(math.log(50.0), math.log(7500.0)))
            T = blen / sr
            if abs(f2 - f1) < 1e-6:
                ph = 2 * math.pi * f1 * t
            else:
                k = math.log(f2 / f1) / T
                ph = 2 * math.pi * f1 * (np.exp(k * t) - 1.0) / k
            seg = np.sin(ph + g.uniform(0, 2 * math.pi))
        else:
            f0 = g.uniform(80.0, 400.0)
            tab = _harmonic_table(g, f0, sr)
            size = tab.shape[0] - 1
            u = (f0 * t + g.uniform()) % 1.0
            seg = np.interp(u * size, np.arange(size + 1), tab)
            pk = float(np.max(np.abs(seg))) or 1.0
            seg = seg / pk
        x[start:start + blen] += env * seg
    pk = float(np.max(np.abs(x))) or 1.0
    x *= (10.0 ** (level_dbfs / 20.0)) / pk
    return x.astype(np.float32)


def loguniform_lengths(seed: int, count: int, lo_s: float, hi_s: float, sr: float) -> np.ndarray:
    g = rng_for(seed, _STREAM_LEN, 0)
    d = np.exp(g.uniform(math.log(lo_s), math.log(hi_s), count))
    return np.maximum(1, np.round(d * sr)).astype(np.int64)


def levels_dbfs(seed: int, count: int, lo: float = -60.0, hi: float = 0.0) -> np.ndarray:
    return rng_for(seed, _STREAM_LEVEL, 0).uniform(lo, hi, count)


@dataclass
class PackedBatch:
    """Clips packed into one float32 buffer.

    ``offsets[b]`` (a multiple of ``align`` floats) is where clip ``b`` starts,
    ``lengths[b]`` its sample count; the gap after each clip is zero-filled.
    """
    wave: np.ndarray      # float32 [total]
    offsets: np.ndarray   # int64 [B]
    lengths: np.ndarray   # int64 [B]

    @property
    def batch(self) -> int:
        return int(self.lengths.shape[0])

    def clip(self, b: int) -> np.ndarray:
        o = int(self.offsets[b])
        return self.wave[o:o + int(self.lengths[b])]


def pack_clips(clips, align: int = 4) -> PackedBatch:
    lengths = np.array([len(c) for c in clips], dtype=np.int64)
    padded = (lengths + align - 1) // align * align
    offsets = np.zeros(len(clips), dtype=np.int64)
    if len(clips) > 1:
        offsets[1:] = np.cumsum(padded)[:-1]
    total = int(padded.sum()) if len(clips) else 0
    wave = np.zeros(max(total, align), dtype=np.float32)
    for c, o in zip(clips, offsets):
        wave[o:o + len(c)] = c
    return PackedBatch(wave=wave, offsets=offsets, lengths=lengths)


def workload(name: str, seed: int = 1234, clips: int | None = None, first: int = 0):
    """Clips of one named synthetic workload (see module docstring).

    ``clips``/``first`` select a sub-range of the workload's clips (same
    content as in the full workload).  Returns (list of float32 arrays, sr).
    """
    if name == "tones_8x1s":            # 8 clips of 1 s at 16 kHz
        n = 8 if clips is None else clips
        return [tones_clip(seed, first + i) for i in range(n)], 16000.0
    if name == "rich_64x30s":           # 64 clips of 30 s at 16 kHz, peak 0 dBFS
        n = 64 if clips is None else clips
        return [rich_clip(seed, first + i, 480000) for i in range(n)], 16000.0
    if name == "levels_1024x10s":       # 1024 clips of 10 s, peak U[-60, 0] dBFS
        n = 1024 if clips is None else clips
        lv = levels_dbfs(seed, 1024)
        return [rich_clip(seed, first + i, 160000, level_dbfs=float(lv[(first + i) % 1024]))
                for i in range(n)], 16000.0
    raise ValueError(f"unknown workload {name!r}")


# Two basis groups of the mixed-geometry workload: (sr, n_fft, hop, n_mels, fmin, fmax).
MIXED_GROUPS = ((16000.0, 400, 160, 80, 0.0, 8000.0), (22050.0, 1024, 256, 80, 0.0, 8000.0))


def mixed_groups(seed: int = 1234, count: int = 4096, first: int = 0, n: int | None = None,
                 pool: int = 0):
    """Mixed-geometry batch: ``count`` clips with durations log-uniform in
    0.5-30 s (mean about 7.2 s); clip i belongs to group i % 2 of
    ``MIXED_GROUPS`` and is drawn at that group's sample rate.

    ``pool`` > 0 cuts each clip out of one of ``pool`` 30 s clips per group
    (at a seeded offset) instead of synthesising it: same lengths, much faster
    for the full 4096-clip batch.  Returns (clips, group ids) for clips
    ``first .. first+n-1``.
    """
    n = count - first if n is None else n
    d = np.exp(rng_for(seed, _STREAM_LEN, 1).uniform(math.log(0.5), math.log(30.0), count))
    starts = rng_for(seed, _STREAM_LEN, 2).uniform(0.0, 1.0, count)
    pools = {}
    clips, ids = [], []
    for i in range(first, first + n):
        gid = i % 2
        sr = MIXED_GROUPS[gid][0]
        L = max(16, int(round(d[i] * sr)))
        if pool > 0:
            key = (gid, (i // 2) % pool)
            if key not in pools:
                pools[key] = rich_clip(seed, 200000 + 1000 * gid + key[1], int(30 * sr), sr=sr)
            src = pools[key]
            L = min(L, src.shape[0])
            s0 = int(starts[i] * (src.shape[0] - L))
            clips.append(src[s0:s0 + L].copy())
        else:
            clips.append(rich_clip(seed, 100000 + i, L, sr=sr))
        ids.append(gid)
    return clips, np.asarray(ids, dtype=np.int32)


def xavier_uniform(seed: int, fan_out: int, fan_in: int, tag: int = 0) -> np.ndarray:
    """Xavier/Glorot-uniform init, shape [fan_out, fan_in], float32."""
    g = rng_for(seed, _STREAM_MLP, tag)
    a = math.sqrt(6.0 / (fan_in + fan_out))
    return g.uniform(-a, a, (fan_out, fan_in)).astype(np.float32)


def batch_order(seed: int, n: int, epoch: int) -> np.ndarray:
    """Shuffled sample order for one training epoch (int64)."""
    return rng_for(seed, _STREAM_ORDER, epoch).permutation(n).astype(np.int64)
