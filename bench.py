#!/usr/bin/env python3
"""Throughput benchmark of the MelT hot path on GB300.

Workload (one "step"): MelT log-Mel of 64 synthetic clips of 30 s at 16 kHz
(n_fft=400, hop=160, 80 Mel bins over 0-8000 Hz, periodic Hann, eps=1e-10),
i.e. 64 x 2998 = 191,872 frames, through libmelt's C ABI (melt_forward_ex with
MELT_FWD_INPUT_READY: the rotating inputs are never written by a kernel on
the stream, so each launch stages samples while the previous one drains).

  value     frames/s with inputs resident in HBM (CUDA events, kernel stream)
  e2e       frames/s through the public Python API with pinned HOST buffers:
            H2D of the step's waveforms, the forward, D2H of its features
  roofline  dominant kernel vs the measured HBM copy bandwidth
            (bound "hbm" for the tensor-core forms, "alu" for FP32 SIMT)
  cpu_baseline  the FP64 oracle on the host cores on a bounded sample

Inputs larger than L2: the step's inputs and outputs rotate over several
device copies (together well above the 129 MB L2).

--impl reference times the FP64 CPU oracle on the same workload (bounded
sample per step) and prints the same JSON line with "impl": "reference".
Multi-GPU (torchrun): replicas only; every rank runs the same per-GPU
workload (weak scaling), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator workload, sr, n_fft, hop, n_mels, fmin, fmax)
    "rich_64x30s": ("rich_64x30s", 16000.0, 400, 160, 80, 0.0, 8000.0),
    "levels_1024x10s": ("levels_1024x10s", 16000.0, 400, 160, 80, 0.0, 8000.0),
    "tones_8x1s": ("tones_8x1s", 16000.0, 400, 160, 80, 0.0, 8000.0),
}
L2_BYTES = 129e6
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def kernel_sources_sha256() -> str:
    """Hash of the sources that define the tensor-core kernels and their launch
    configuration (device headers, the CTA-pair instantiation, the planner, the
    shared types, the ABI header and the build flags): ties an ncu traffic
    figure to the kernel it measured.  Translation units of other kernels and
    of host-only calls are left out, so adding one does not disown the figure."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2606_01009_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cuh"))
                   + [os.path.join(csrc, f) for f in ("melt_tc2.cu", "melt_tc.cu", "melt_tc.h", "melt_internal.h")]
                   + [os.path.join(ROOT, "include", "melt.h"),
                      os.path.join(ROOT, "paper_2606_01009_gb300", "build.py")])
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(key: str):
    """DRAM bytes per launch from an ncu capture of this exact kernel source, else None."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sources_sha256") != kernel_sources_sha256():
        return None   # the kernel changed since the counters were taken
    return rec["dram_bytes_per_launch"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="melt", choices=["melt", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "bf16x3", "fp8"])
    ap.add_argument("--workload", default="rich_64x30s", choices=sorted(WORKLOADS))
    ap.add_argument("--n-mels", type=int, default=None)
    ap.add_argument("--mfcc", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--trials", type=int, default=20,
                    help="at least this many timed trials of --steps launches (median reported)")
    ap.add_argument("--trial-seconds", type=float, default=1.0,
                    help="add trials until the timed region holds about this much GPU time")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grouped", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the mixed two-group 4096-clip batch (grouped graph vs per-clip launches)")
    ap.add_argument("--correction", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the correction MLP: fused in the epilogue vs a separate pass")
    ap.add_argument("--forms", action=argparse.BooleanOptionalAction, default=True,
                    help="also time every other operand form")
    ap.add_argument("--stft", action=argparse.BooleanOptionalAction, default=True,
                    help="also time torch.stft + Mel matmul on the same GPU (context)")
    ap.add_argument("--configs", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the M = 128 and MFCC variants and the 1024 x 10 s precision sweep")
    ap.add_argument("--sweeps", action=argparse.BooleanOptionalAction, default=True,
                    help="also run the batch sweep (4 s clips) and the Mel-count sweep (160 s clip)")
    ap.add_argument("--plan-cache", default=os.environ.get("MELT_AUTOTUNE_CACHE",
                                                           os.path.join(tempfile.gettempdir(), "melt_plans.txt")),
                    help="on-disk plan cache of melt_group_autotune (grouped leg)")
    ap.add_argument("--energy", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure J per frame with NVML's total-energy counter")
    return ap.parse_args()


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 100 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        return self.parse(self.f.read())

    @staticmethod
    def parse(text):
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in text.splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            try:
                pw.append(float(p[3]))
            except ValueError:
                pass
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(pw) if pw else None}


# ------------------------------------------------------------ workload
def make_inputs(args):
    from paper_2606_01009_gb300 import inputs as G
    gen, sr, n_fft, hop, n_mels, fmin, fmax = WORKLOADS[args.workload]
    if args.n_mels:
        n_mels = args.n_mels
    clips, sr = G.workload(gen)
    pk = G.pack_clips(clips)
    return clips, pk, dict(sr=sr, n_fft=n_fft, hop=hop, n_mels=n_mels, fmin=fmin, fmax=fmax)


def frames_of(lengths, n_fft, hop):
    return int(sum((L - n_fft) // hop + 1 for L in lengths if L >= n_fft))


def algorithmic_bytes(lengths, n_fft, hop, n_out):
    """Bytes a perfect implementation moves: each needed sample read once,
    each feature written once (FP32)."""
    tot = 0
    for L in lengths:
        if L < n_fft:
            continue
        T = (L - n_fft) // hop + 1
        tot += 4 * ((T - 1) * hop + n_fft) + 4 * T * n_out
    return tot


def cpu_oracle_baseline(clips, cfg, n_mfcc, seconds):
    """Time the FP64 oracle as it stands on the host cores; bounded sample."""
    from oracle import melt_oracle as O
    spec = O.MelTSpec(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"],
                      fmin=cfg["fmin"], fmax=cfg["fmax"], n_mfcc=n_mfcc)
    frames = 0
    n_clips = 0
    t0 = time.perf_counter()
    i = 0
    while True:
        c = clips[i % len(clips)]
        out = O.melt_clip(c, spec)
        frames += out.shape[0]
        n_clips += 1
        i += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": frames / el, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_clips} clips ({frames} frames) of the workload, FP64 numpy oracle, {el:.1f} s"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------- main arm
class Workload:
    """Device-resident copies of one batch, rotated so inputs+outputs exceed L2."""

    def __init__(self, args, dev):
        import torch
        self.clips, self.pk, self.cfg = make_inputs(args)
        self.name = args.workload
        self.lens = np.ascontiguousarray(self.pk.lengths, dtype=np.int64)
        self.offs = np.ascontiguousarray(self.pk.offsets, dtype=np.int64)
        self.wave_h = torch.from_numpy(self.pk.wave)
        self.in_bytes = self.pk.wave.nbytes
        self.dev = dev
        self.waves = None

    def device_copies(self, n_out, T):
        import torch
        out_bytes = T * n_out * 4
        copies = max(2, math.ceil(2.5 * L2_BYTES / (self.in_bytes + out_bytes)))
        if self.waves is None or len(self.waves) < copies:
            self.waves = [self.wave_h.to(self.dev) for _ in range(copies)]
        outs = [torch.empty((T, n_out), device=self.dev) for _ in range(copies)]
        return self.waves[:copies], outs, copies


def trial_count(args, one_step, stream, dev, steps):
    """Trials of `steps` launches to time: at least args.trials, and enough
    for about args.trial_seconds of load so that the clock sampler (10 Hz)
    sees the region; at most 5000."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(3):
        one_step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    est_ms = max(a.elapsed_time(b) / 3, 1e-3) * steps
    return int(min(5000, max(args.trials, math.ceil(args.trial_seconds * 1e3 / est_ms))))


def trial_stats(trial_ms, steps):
    """Median, spread and count of the per-launch times of the trials (ms)."""
    per = sorted(t / steps for t in trial_ms)
    q = lambda f: per[min(len(per) - 1, int(f * (len(per) - 1) + 0.5))]
    return {"count": len(per), "launches_per_trial": steps, "median_ms": statistics.median(per),
            "min_ms": per[0], "p10_ms": q(0.1), "p90_ms": q(0.9), "max_ms": per[-1]}


def whole_job(ms_total, frames_per_step, steps, world, dev):
    """(slowest rank's timed region in ms, whole-job frames/s).  Every rank
    times its own replica of the workload (weak scaling); the job takes as long
    as its slowest rank, which processed world x frames_per_step x steps frames
    in all.  With world > 1 this is a collective: every rank must call it."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms_total)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    return ms_total, world * frames_per_step * steps / (ms_total / 1e3)


def time_form(args, W, precision, steps, warmup, world, want_e2e):
    """Time melt_forward_ex (MELT_FWD_INPUT_READY) for one operand form; returns a dict of measurements."""
    import ctypes as C
    import torch
    from paper_2606_01009_gb300 import melt

    cfg, dev = W.cfg, W.dev
    fe = melt.Frontend(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"],
                       fmin=cfg["fmin"], fmax=cfg["fmax"], precision=precision, n_mfcc=args.mfcc)
    n_out = fe.n_out
    T = fe.total_frames(W.lens)
    waves, outs, copies = W.device_copies(n_out, T)
    stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream)
    lp = W.lens.ctypes.data_as(C.POINTER(C.c_int64))
    op = W.offs.ctypes.data_as(C.POINTER(C.c_int64))
    wp = [C.c_void_p(w.data_ptr()) for w in waves]
    outp = [C.c_void_p(o.data_ptr()) for o in outs]
    # the rotating input copies are written before the timed launches and
    # never by a kernel on this stream, so each launch may stage its samples
    # while the previous one drains (MELT_FWD_INPUT_READY)
    fwd = melt.lib.melt_forward_ex
    flags = C.c_uint(melt.MELT_FWD_INPUT_READY)
    B = int(W.lens.shape[0])

    def step(i):
        st = fwd(fe.handle, wp[i % copies], op, lp, B, outp[i % copies], sp, flags)
        if st != 0:
            raise melt.MeltError(st, "melt_forward_ex")

    for i in range(warmup):
        step(i)
    fe.sync(stream)
    trials = trial_count(args, lambda: step(0), stream, dev, steps)
    clocks = ClockSampler(dev.index)
    clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(trials + 1)]
    # Trials of `steps` launches run back to back; only the forward kernels
    # run between two events.  An event between two launches cuts the
    # programmatic (early-launch) edge between them, so it is recorded only at
    # trial boundaries, and one launch's average duration is a trial / steps.
    ev[0].record(stream)
    i = 0
    for t in range(trials):
        for _ in range(steps):
            step(i)
            i += 1
        ev[t + 1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    fe.sync(stream)
    trial_ms = [ev[t].elapsed_time(ev[t + 1]) for t in range(trials)]
    ms_total = statistics.median(trial_ms)
    launch_ms = ms_total / steps
    ms_total, value = whole_job(ms_total, T, steps, world, dev)
    res = {"precision": precision, "T": T, "n_out": n_out, "copies": copies, "steps": steps,
           "ms_total": ms_total, "ms_per_step": ms_total / steps, "launch_ms": launch_ms,
           "value": value, "clocks": ck, "trials": trial_stats(trial_ms, steps), "step": step,
           "out_sample": outs[0], "fe": fe,
           # `step` holds raw pointers into these buffers: they live as long as it does
           "buffers": (waves, outs)}

    if want_e2e:
        # end to end through the public C ABI with pinned HOST buffers:
        # melt_forward_host copies each chunk in, runs it and copies its
        # features out, overlapping the transfers with the kernels
        wave_pin = W.wave_h.pin_memory()
        out_pin = torch.empty((T, n_out), dtype=torch.float32).pin_memory()

        def e2e_step():
            melt.melt_forward_host(fe.handle, wave_pin, W.offs, W.lens, out_pin, stream)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize(dev)
        E = args.e2e_steps
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(E):
            e2e_step()
        a1.record(stream)
        torch.cuda.synchronize(dev)
        fe.sync(stream)
        e2e_ms = a0.elapsed_time(a1) / E
        res["e2e"] = {"value": world * T / (e2e_ms / 1e3), "unit": "frames/s",
                      "h2d_bytes_per_step": W.in_bytes, "d2h_bytes_per_step": T * n_out * 4,
                      "ms_per_step": e2e_ms}
    return res


def roofline(cfg, W, r, peaks, peak_kind):
    prec, T, n_out = r["precision"], r["T"], r["n_out"]
    flops = 2 * cfg["n_fft"] * 2 * cfg["n_mels"] * T * (3 if prec == "bf16x3" else 1)
    alg_bytes = algorithmic_bytes(W.lens, cfg["n_fft"], cfg["hop"], n_out)
    sec = r["launch_ms"] / 1e3
    if prec == "fp32":
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = flops / sec / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "peak_note": "FP32 FFMA peak derived: 152 SMs x 128 lanes x 2 FLOP x "
                f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz max SM clock",
                "algorithmic_flops_per_launch": flops, "launch_ms": r["launch_ms"]}
    ach = alg_bytes / sec / 1e9
    peak = peaks["hbm_gbs"]
    key = f"{prec}/{W.name}/n_mels={cfg['n_mels']}/n_out={n_out}"
    out = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "traffic": measured_traffic(key), "traffic_key": key, "peak_note": f"hbm_gbs of {peak_kind} peaks (copy bandwidth)",
           "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": r["launch_ms"],
           "tensor_tflops": flops / sec / 1e12}
    out["tensor_frac_of_bf16_peak"] = out["tensor_tflops"] / peaks.get("bf16_tflops", 1900.0)
    return out


def accuracy_vs_oracle(W, forms, cfg, mfcc, n_clips=2):
    """dB error of each form's output vs the FP64 oracle on the first clips (CPU leg)."""
    from oracle import melt_oracle as O
    spec = O.MelTSpec(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"],
                      fmin=cfg["fmin"], fmax=cfg["fmax"], n_mfcc=mfcc)
    ref = np.concatenate([O.melt_clip(c, spec) for c in W.clips[:n_clips]])
    rows = ref.shape[0]
    acc = {}
    for name, r in forms.items():
        got = r["out_sample"][:rows].cpu().numpy().astype(np.float64)
        mx, rms = O.err_db(got, ref)
        mask = O.within_db_of_frame_max(ref, 60.0) if not mfcc else None
        mx60, rms60 = O.err_db(got, ref, mask) if mask is not None else (mx, rms)
        acc[name] = {"max_db": mx, "rms_db": rms, "max_db_within_60dB": mx60, "rms_db_within_60dB": rms60}
    return acc, f"first {n_clips} clips ({rows} frames) vs the FP64 oracle"


def energy_estimate(r):
    """Joules per frame from the board power sampled around the timed region
    (median of the nvidia-smi power.draw samples x launch time / frames).  An
    estimate, beside frames/s: the readings average over a window that takes
    in the idle edges of a short region."""
    w = (r.get("clocks") or {}).get("power_w_median")
    if not w or not r.get("T") or not r.get("launch_ms") or w <= 0 or r["launch_ms"] <= 0:
        return None
    j = w * (r["launch_ms"] / 1e3) / r["T"]
    return {"watts_median": w, "joules_per_frame": j, "frames_per_joule": 1.0 / j,
            "samples": r["clocks"].get("samples"),
            "method": "median nvidia-smi power.draw over the timed region x launch time / frames (estimate)"}


def run_melt(args, rank, world):
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    W = Workload(args, dev)
    cfg = W.cfg
    peaks, peak_kind = load_peaks()
    head = time_form(args, W, args.precision, args.steps, args.warmup, world, want_e2e=True)
    forms = {args.precision: head}
    if args.forms:
        for prec in ["fp32", "bf16", "bf16x3", "fp8"]:
            if prec == args.precision:
                continue
            # scale the step count so each form's timed region is ~1 s at most
            k = max(10, min(args.steps, int(1000.0 / max(head["ms_per_step"], 1e-3) * 0.3)))
            try:
                forms[prec] = time_form(args, W, prec, k if prec != "fp32" else max(10, k // 20),
                                        max(3, args.warmup // 10), world, want_e2e=False)
            except Exception as e:  # a form this configuration cannot run
                forms[prec] = {"error": str(e)}
    T, n_out = head["T"], head["n_out"]
    B = int(W.lens.shape[0])
    res = {
        "metric": "log-Mel frames/s on 1 GB300 (MelT, %s)" % args.precision,
        "value": head["value"], "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3", "fp8": "fp8e4m3"}[args.precision],
        "data": "synthetic (seeded chirps, harmonic stacks, pink noise, AM bursts; stands in for LibriSpeech)",
        "config": {"workload": f"{args.workload}: {B} clips, {T} frames, sr={cfg['sr']:.0f}, n_fft={cfg['n_fft']}, "
                               f"hop={cfg['hop']}, n_mels={cfg['n_mels']}, n_mfcc={args.mfcc}, periodic Hann, eps=1e-10",
                   "precision": args.precision, "frames_per_step": T,
                   "launch": "melt_forward_ex(MELT_FWD_INPUT_READY), back to back on one stream",
                   "l2": f"inputs+outputs rotate over {head['copies']} device copies "
                         f"({head['copies'] * (W.in_bytes + T * n_out * 4) / 1e6:.0f} MB > 129 MB L2)",
                   "parallelism": f"replicas x{world}"},
        "e2e": head["e2e"],
        "gpu_launches": args.steps * head["trials"]["count"],
        "roofline": roofline(cfg, W, head, peaks, peak_kind),
        "clocks": {k: head["clocks"][k] for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")},
        "trials": head["trials"],
        "energy": None,
    }
    if args.forms:
        res["forms"] = {}
        for name, r in forms.items():
            if "error" in r:
                res["forms"][name] = r
                continue
            rf = roofline(cfg, W, r, peaks, peak_kind)
            res["forms"][name] = {"value": r["value"], "ms_per_step": r["ms_per_step"], "steps": r["steps"],
                                  "trials": r["trials"],
                                  "roofline_frac": rf["frac"], "bound": rf["bound"],
                                  "achieved": rf["achieved"], "unit": rf["unit"],
                                  "clocks_sm_mhz": r["clocks"]["sm_mhz"],
                                  "energy": None}
    if args.energy and rank == 0:
        nv = NvmlEnergy(dev.index)
        for name in [args.precision] + [f for f in ("fp8", "fp32", "bf16", "bf16x3") if f != args.precision]:
            r = forms.get(name)
            if not r or "error" in r:
                continue
            e = measure_energy(nv, r["step"], r["T"], torch.cuda.current_stream(dev), dev)
            if "unavailable" in e:
                e["estimate"] = energy_estimate(r)
            if name == args.precision:
                res["energy"] = e
            if args.forms and name in res.get("forms", {}):
                res["forms"][name]["energy"] = e
    return res, W, forms


def run_reference(args, rank, world):
    if rank != 0:
        return None
    clips, pk, cfg = make_inputs(args)
    from oracle import melt_oracle as O
    spec = O.MelTSpec(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"],
                      fmin=cfg["fmin"], fmax=cfg["fmax"], n_mfcc=args.mfcc)
    T_all = frames_of(pk.lengths, cfg["n_fft"], cfg["hop"])
    # bounded sample per step: a few clips of the workload
    per_step = max(1, min(len(clips), 4))
    for i in range(args.warmup):
        O.melt_clip(clips[i % len(clips)], spec)
    K = args.steps
    frames = 0
    t0 = time.perf_counter()
    for s in range(K):
        for j in range(per_step):
            frames += O.melt_clip(clips[(s * per_step + j) % len(clips)], spec).shape[0]
    el = time.perf_counter() - t0
    value = frames / el
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {
        "impl": "reference", "metric": "log-Mel frames/s on 1 GB300 (MelT, %s)" % args.precision,
        "value": value, "unit": "frames/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {len(clips)} clips, {T_all} frames (each step: a {per_step}-clip sample)",
                   "precision": "fp64 oracle", "parallelism": "host CPU"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} clips per step, {K} steps, {frames} frames"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _jsonable(o):
    if hasattr(o, "item"):
        return o.item()
    return str(o)


def time_grouped(args, dev, steps=20, warmup=3, per_clip_steps=2):
    """Mixed-geometry batch of 4096 clips (16 kHz 400/160/80 and 22.05 kHz 1024/256/80, BF16):
    melt_forward_grouped as one shared persistent launch and as one launch per
    basis, with a CUDA graph and without, and one melt_forward per clip."""
    import torch
    from paper_2606_01009_gb300 import inputs as G
    from paper_2606_01009_gb300 import melt
    clips, ids = G.mixed_groups(pool=16)
    pk = G.pack_clips(clips)
    fes = [melt.Frontend(sr=sr, n_fft=n, hop=h, n_mels=m, fmin=lo, fmax=hi, precision="bf16")
           for (sr, n, h, m, lo, hi) in G.MIXED_GROUPS]
    wave = torch.from_numpy(pk.wave).to(dev)
    T = sum(fes[g].num_frames(int(L)) for L, g in zip(pk.lengths, ids))
    out = torch.empty((T, fes[0].n_out), device=dev)
    stream = torch.cuda.current_stream(dev)
    frames_per_group = [sum(fes[g].num_frames(int(L)) for L, gg in zip(pk.lengths, ids) if gg == g)
                        for g in range(2)]
    in_b = pk.wave.nbytes
    res = {"workload": f"mixed_4096: 4096 clips, log-uniform 0.5-30 s, alternating 16 kHz 400/160/80 and "
                       f"22.05 kHz 1024/256/80; {T} frames ({frames_per_group[0]} + {frames_per_group[1]}), "
                       f"{in_b / 1e9:.2f} GB in, {T * fes[0].n_out * 4 / 1e9:.2f} GB out (> L2)",
           "precision": "bf16", "frames_per_step": T}

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / k

    # default plans: one launch per basis, and both bases in one shared
    # persistent launch (MELT_GROUP_SHARED); then the plans
    # melt_group_autotune picks by timing the per-basis grouped call (kept in
    # the on-disk plan cache for later processes)
    gf = melt.GroupedFrontend(fes, graphs=True)
    ms = timed(lambda: gf(wave, pk.offsets, pk.lengths, ids, out=out, stream=stream), steps, warmup)
    res["grouped_graph_default_plans"] = {"ms_per_step": ms, "frames_per_s": T / (ms / 1e3),
                                          "plans": [melt.melt_plan_get(fe.handle) for fe in fes]}
    gf.close()
    gf = melt.GroupedFrontend(fes, graphs=True, shared_launch=True)
    ms = timed(lambda: gf(wave, pk.offsets, pk.lengths, ids, out=out, stream=stream), steps, warmup)
    res["grouped_graph_shared_launch_default_plans"] = {"ms_per_step": ms, "frames_per_s": T / (ms / 1e3),
                                                        "launches_per_step": 1}
    gf.close()
    gf = melt.GroupedFrontend(fes, graphs=True)
    t0 = time.perf_counter()
    plans, hit = gf.autotune(wave, pk.offsets, pk.lengths, ids, out, path=args.plan_cache, stream=stream)
    res["autotune"] = {"plans": plans, "cache_hit": hit, "seconds": round(time.perf_counter() - t0, 3),
                       "plan_cache": args.plan_cache}
    gf.close()
    # with the tuned plans: one launch per basis (graph, and direct)
    for name, graphs, shared in (("grouped_graph", True, False), ("grouped_direct", False, False)):
        gf = melt.GroupedFrontend(fes, graphs=graphs, shared_launch=shared)
        ms = timed(lambda: gf(wave, pk.offsets, pk.lengths, ids, out=out, stream=stream), steps, warmup)
        gf.sync(stream)
        res[name] = {"ms_per_step": ms, "frames_per_s": T / (ms / 1e3)}
        gf.close()
    # one melt_forward per clip, rows at the clip's place in the packed output
    rows = np.concatenate([[0], np.cumsum([fes[g].num_frames(int(L)) for L, g in zip(pk.lengths, ids)])])
    fwd = melt.lib.melt_forward
    import ctypes as C
    sp = C.c_void_p(stream.cuda_stream)
    calls = []
    for b in range(len(clips)):
        if rows[b + 1] == rows[b]:
            continue
        L = np.array([pk.lengths[b]], np.int64)
        calls.append((fes[ids[b]].handle, C.c_void_p(wave.data_ptr() + 4 * int(pk.offsets[b])), L,
                      C.c_void_p(out.data_ptr() + 4 * fes[0].n_out * int(rows[b]))))

    def per_clip():
        for h, wp, L, op in calls:
            st = fwd(h, wp, None, L.ctypes.data_as(C.POINTER(C.c_int64)), 1, op, sp)
            if st != 0:
                raise melt.MeltError(st, "melt_forward")
    ms = timed(per_clip, per_clip_steps, 1)
    for fe in fes:
        fe.sync(stream)
    res["per_clip_launches"] = {"ms_per_step": ms, "frames_per_s": T / (ms / 1e3), "launches": len(calls)}
    for fe in fes:
        fe.close()
    return res


def htk_mel_filterbank(sr, n_fft, n_mels, fmin, fmax):
    """Triangular Mel filterbank on the HTK scale, [n_mels, n_fft // 2 + 1],
    peak 1 at each of the M interior points of M + 2 Mel-uniform points: the
    Mel step of the conventional pipeline timed as context."""
    mel = lambda f: 2595.0 * np.log10(1.0 + f / 700.0)
    hz = lambda m: 700.0 * (10.0 ** (m / 2595.0) - 1.0)
    pts = hz(np.linspace(mel(fmin), mel(fmax), n_mels + 2))
    bins = np.arange(n_fft // 2 + 1) * sr / n_fft
    fb = np.zeros((n_mels, bins.size))
    for m in range(n_mels):
        lo, c, hi = pts[m], pts[m + 1], pts[m + 2]
        fb[m] = np.clip(np.minimum((bins - lo) / (c - lo), (hi - bins) / (hi - c)), 0.0, None)
    return fb


def time_torch_stft(W, dev, steps=20, warmup=3, eps=1e-10):
    """Context, not a product path: the conventional pipeline on the same GPU
    and clips - torch.stft (cuFFT, no centring), |X|^2, a dense Mel matmul and
    the log, in FP32 - timed like the headline (CUDA events around the loop,
    two input copies rotated).  Its output is [B, M, T] rather than frame-major."""
    cfg = W.cfg
    lens, offs = W.lens, W.offs
    B, L = len(lens), int(lens[0])
    if not (np.all(lens == L) and np.array_equal(offs, np.arange(B, dtype=np.int64) * L)):
        return {"skipped": "the batch is not B clips of one length packed back to back"}
    return time_stft_batch(W.wave_h[: B * L].view(B, L), cfg, dev, steps, warmup, eps)


def time_stft_batch(x, cfg, dev, steps=20, warmup=3, eps=1e-10):
    """torch.stft + |X|^2 + dense HTK Mel matmul + log on a [B, L] host batch (context)."""
    import torch
    n_fft, hop, M = cfg["n_fft"], cfg["hop"], cfg["n_mels"]
    B, L = x.shape
    xs = [x.to(dev) for _ in range(2)]
    win = torch.hann_window(n_fft, periodic=True, dtype=torch.float32, device=dev)
    fb = torch.from_numpy(htk_mel_filterbank(cfg["sr"], n_fft, M, cfg["fmin"], cfg["fmax"])).to(dev, torch.float32)

    def step(i):
        X = torch.stft(xs[i % 2], n_fft, hop_length=hop, win_length=n_fft, window=win, center=False,
                       return_complex=True)
        return torch.log(torch.matmul(fb, X.real.square() + X.imag.square()) + eps)

    T = (L - n_fft) // hop + 1 if L >= n_fft else 0
    for i in range(warmup):
        step(i)
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)
        stream = torch.cuda.current_stream(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(steps):
            step(i)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / steps
    else:
        t0 = time.perf_counter()
        for i in range(steps):
            step(i)
        ms = (time.perf_counter() - t0) * 1e3 / steps
    return {"pipeline": "torch.stft (cuFFT) + |X|^2 + dense HTK Mel matmul + log, FP32, no centring",
            "frames_per_step": B * T, "ms_per_step": ms, "frames_per_s": B * T / (ms / 1e3),
            "device": str(dev)}


# ----------------------------------------------------- energy (NVML counter)
class NvmlEnergy:
    """Board energy from NVML's total-energy counter (millijoules since the
    driver loaded; a read-only query, as in the paper's energy protocol).  The
    device is found by its UUID, else by index when NVML sees one device."""

    def __init__(self, dev_index):
        import ctypes as C
        self.C, self.ok, self.why = C, False, ""
        try:
            self.lib = C.CDLL("libnvidia-ml.so.1")
        except OSError as e:
            self.why = f"libnvidia-ml not loadable: {e}"
            return
        if self.lib.nvmlInit_v2() != 0:
            self.why = "nvmlInit failed"
            return
        h = C.c_void_p()
        st = 1
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(dev_index).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            st = self.lib.nvmlDeviceGetHandleByUUID(C.c_char_p(uuid.encode()), C.byref(h))
        except Exception:
            st = 1
        if st != 0:
            n = C.c_uint(0)
            self.lib.nvmlDeviceGetCount_v2(C.byref(n))
            if n.value != 1:
                self.why = f"GPU not found by UUID and NVML sees {n.value} devices"
                return
            st = self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(0), C.byref(h))
        if st != 0:
            self.why = f"no NVML handle (status {st})"
            return
        self.h = h
        self.ok = self.read_mj() is not None
        if not self.ok:
            self.why = "nvmlDeviceGetTotalEnergyConsumption unsupported"

    def read_mj(self):
        v = self.C.c_ulonglong(0)
        st = self.lib.nvmlDeviceGetTotalEnergyConsumption(self.h, self.C.byref(v))
        return int(v.value) if st == 0 else None


def measure_energy(nv, step, frames_per_step, stream, dev, min_quanta=30, min_s=1.5, max_s=8.0):
    """Joules per frame over a window of back-to-back launches that spans at
    least `min_quanta` updates of the energy counter (polled every 2 ms on a
    host thread) and `min_s` seconds: (E_end - E_start) / frames."""
    import torch
    if not nv.ok:
        return {"unavailable": nv.why}
    seen = {"n": 0, "run": True}

    def poll():
        last = nv.read_mj()
        while seen["run"]:
            v = nv.read_mj()
            if v is not None and v != last:
                seen["n"] += 1
                last = v
            time.sleep(0.002)

    th = threading.Thread(target=poll, daemon=True)
    torch.cuda.synchronize(dev)
    th.start()
    e0, t0, steps = nv.read_mj(), time.perf_counter(), 0
    while True:
        for _ in range(50):
            step(steps)
            steps += 1
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        if (el >= min_s and seen["n"] >= min_quanta) or el >= max_s:
            break
    e1 = nv.read_mj()
    seen["run"] = False
    th.join()
    joules = (e1 - e0) / 1e3
    frames = frames_per_step * steps
    return {"joules_per_frame": joules / frames, "frames_per_joule": frames / joules if joules > 0 else None,
            "watts": joules / el, "window_s": el, "counter_updates": seen["n"], "launches": steps,
            "method": "NVML total-energy counter over back-to-back launches (>= 30 counter updates)"}


# --------------------------------------------------------- config legs, sweeps
def time_launches(fn, dev, steps, trials=7, warmup=3):
    """Median over `trials` of the per-launch time (ms) of `steps` back-to-back calls of fn(i)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    for i in range(warmup):
        fn(i)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(trials + 1)]
    ev[0].record(stream)
    i = 0
    for t in range(trials):
        for _ in range(steps):
            fn(i)
            i += 1
        ev[t + 1].record(stream)
    torch.cuda.synchronize(dev)
    return statistics.median(ev[t].elapsed_time(ev[t + 1]) / steps for t in range(trials))


def _gen_levels(first, n):
    from paper_2606_01009_gb300 import inputs as G
    return G.workload("levels_1024x10s", clips=n, first=first)[0]


def levels_clips(workers=16):
    """The 1024 x 10 s precision-sweep clips, generated by a pool of spawned
    processes (generation only; the clips are identical to a serial draw)."""
    import multiprocessing as mp
    n = max(1, min(workers, os.cpu_count() or 1))
    parts = [(i * 1024 // n, (i + 1) * 1024 // n - i * 1024 // n) for i in range(n)]
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.starmap(_gen_levels, parts)
    return [c for part in res for c in part]


def frontend_leg(melt, dev, clips, cfg, precision, n_mfcc=0, steps=10, peaks=None, oracle_clips=0):
    """Launch time, frames/s and roofline fraction of one Frontend on a batch of
    clips (inputs + outputs rotated over copies that exceed L2); with
    oracle_clips > 0, the form's dB error against the FP64 oracle on the first
    oracle_clips clips."""
    import torch
    from paper_2606_01009_gb300 import inputs as G
    pk = G.pack_clips(clips)
    fe = melt.Frontend(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"], fmin=cfg["fmin"],
                       fmax=cfg["fmax"], precision=precision, n_mfcc=n_mfcc)
    T = fe.total_frames(pk.lengths)
    in_b, out_b = pk.wave.nbytes, T * fe.n_out * 4
    copies = max(2, math.ceil(2.5 * L2_BYTES / max(in_b + out_b, 1)))
    waves = [torch.from_numpy(pk.wave).to(dev) for _ in range(copies)]
    outs = [torch.empty((T, fe.n_out), device=dev) for _ in range(copies)]
    ms = time_launches(lambda i: fe(waves[i % copies], pk.offsets, pk.lengths, out=outs[i % copies],
                                    input_ready=True), dev, steps)
    fe.sync()
    alg = algorithmic_bytes(pk.lengths, cfg["n_fft"], cfg["hop"], fe.n_out)
    res = {"precision": precision, "n_mels": cfg["n_mels"], "n_mfcc": n_mfcc, "frames": T, "launch_us": ms * 1e3,
           "frames_per_s": T / (ms / 1e3), "hbm_gbs": alg / (ms / 1e3) / 1e9}
    if peaks:
        if precision == "fp32":
            flops = 2 * cfg["n_fft"] * 2 * cfg["n_mels"] * T
            peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
            res["roofline_frac"], res["bound"] = flops / (ms / 1e3) / peak, "alu"
        else:
            res["roofline_frac"], res["bound"] = res["hbm_gbs"] / peaks["hbm_gbs"], "hbm"
    if oracle_clips:
        from oracle import melt_oracle as O
        spec = O.MelTSpec(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"], fmin=cfg["fmin"],
                          fmax=cfg["fmax"], n_mfcc=n_mfcc)
        ref = np.concatenate([O.melt_clip(c, spec) for c in clips[:oracle_clips]])
        fe(waves[0], pk.offsets, pk.lengths, out=outs[0])
        fe.sync()
        got = outs[0][: ref.shape[0]].cpu().numpy().astype(np.float64)
        err = {"all": O.err_db(got, ref)}
        if not n_mfcc:
            for d in (10.0, 30.0, 60.0, 100.0):
                err[f"within_{int(d)}dB"] = O.err_db(got, ref, O.within_db_of_frame_max(ref, d))
        res["error_db_vs_fp64"] = {k: {"max": v[0], "rms": v[1]} for k, v in err.items()}
        res["error_sample"] = f"first {oracle_clips} clips ({ref.shape[0]} frames)"
    fe.close()
    return res


def config_legs(args, dev, peaks):
    """The other configurations of the workload list, as bench legs: the
    64 x 30 s batch at M = 128 and with the MFCC variant (K = 40), and every
    operand form on the 1024 x 10 s precision sweep (levels -60..0 dBFS)."""
    from paper_2606_01009_gb300 import inputs as G
    from paper_2606_01009_gb300 import melt
    base = dict(sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0)
    out = {}
    rich, _ = G.workload("rich_64x30s")
    out["rich_64x30s_bf16_m128"] = frontend_leg(melt, dev, rich, dict(base, n_mels=128), "bf16", steps=20,
                                               peaks=peaks, oracle_clips=1)
    out["rich_64x30s_bf16_mfcc40"] = frontend_leg(melt, dev, rich, base, "bf16", n_mfcc=40, steps=20, peaks=peaks,
                                                 oracle_clips=1)
    levels = levels_clips()
    sweep = {}
    for prec in ("fp32", "bf16", "bf16x3", "fp8"):
        sweep[prec] = frontend_leg(melt, dev, levels, base, prec, steps=3 if prec == "fp32" else 10, peaks=peaks,
                                   oracle_clips=4)
    out["levels_1024x10s"] = sweep
    return out


def time_fused_stft(W, dev, peaks):
    """The fused STFT + triangular Mel comparator (melt_stft_create: tensor-core
    DFT at N/2 + 1 bins, power, HTK filterbank and log in one kernel) on the
    headline batch, BF16, beside the MelT headline and the torch.stft context."""
    import torch
    from paper_2606_01009_gb300 import melt
    cfg = W.cfg
    fe = melt.StftMelFrontend(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"],
                              fmin=cfg["fmin"], fmax=cfg["fmax"], precision="bf16", scale="htk")
    T = fe.total_frames(W.lens)
    waves, outs, copies = W.device_copies(fe.n_out, T)
    ms = time_launches(lambda i: fe(waves[i % copies], W.offs, W.lens, out=outs[i % copies]), dev, 20)
    fe.sync()
    fe.close()
    alg = algorithmic_bytes(W.lens, cfg["n_fft"], cfg["hop"], cfg["n_mels"])
    bins = cfg["n_fft"] // 2 + 1
    return {"pipeline": f"fused STFT ({bins} DFT bins, BF16 tensor cores) + |X|^2 + HTK triangular Mel + log, "
                        "one kernel (melt_stft_create)",
            "frames_per_step": T, "launch_us": ms * 1e3, "frames_per_s": T / (ms / 1e3),
            "hbm_frac": alg / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "tensor_tflops": 2 * cfg["n_fft"] * 2 * bins * T / (ms / 1e3) / 1e12}


def sweeps(args, dev):
    """Paper's scaling figures on synthetic clips: the batch sweep (1..256 clips
    of 4 s) and the Mel-count sweep (one 160 s clip, M = 40..512, and the
    whole 64 x 30 s batch), MelT (BF16; FP32 up to M = 128 on the 160 s clip)
    against the torch.stft context pipeline on the same GPU."""
    import torch
    from paper_2606_01009_gb300 import inputs as G
    from paper_2606_01009_gb300 import melt
    base = dict(sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0)
    res = {"batch_4s": [], "mels_160s": []}
    clips = [G.rich_clip(4242, i, 64000) for i in range(256)]
    fes = {p: melt.Frontend(precision=p) for p in ("bf16", "fp32")}
    for b in (1, 2, 4, 8, 16, 32, 64, 128, 256):
        pk = G.pack_clips(clips[:b])
        wave = torch.from_numpy(pk.wave).to(dev)
        row = {"batch": b, "frames": fes["bf16"].total_frames(pk.lengths)}
        for p, fe in fes.items():
            out = torch.empty((row["frames"], 80), device=dev)
            ms = time_launches(lambda i: fe(wave, pk.offsets, pk.lengths, out=out, input_ready=True), dev,
                               10 if p == "bf16" else 3)
            row[f"melt_{p}_us"] = ms * 1e3
        x = torch.from_numpy(np.stack([c for c in clips[:b]]))
        row["torch_stft_us"] = time_stft_batch(x, base, dev, steps=10)["ms_per_step"] * 1e3
        row["speedup_bf16_vs_stft"] = row["torch_stft_us"] / row["melt_bf16_us"]
        res["batch_4s"].append(row)
    for fe in fes.values():
        fe.close()
    clip = G.rich_clip(4243, 0, 160 * 16000)
    pk = G.pack_clips([clip])
    wave = torch.from_numpy(pk.wave).to(dev)
    for M in (40, 64, 80, 128, 256, 512):
        cfg = dict(base, n_mels=M)
        row = {"n_mels": M}
        for p in (("bf16", "fp32") if M <= 128 else ("bf16",)):  # FP32 kernels hold M <= 128
            fe = melt.Frontend(precision=p, n_mels=M)
            T = fe.total_frames(pk.lengths)
            out = torch.empty((T, M), device=dev)
            row[f"melt_{p}_us"] = time_launches(lambda i: fe(wave, pk.offsets, pk.lengths, out=out, input_ready=True),
                                                dev, 10 if p == "bf16" else 3) * 1e3
            fe.close()
        row["frames"] = T
        row["torch_stft_us"] = time_stft_batch(torch.from_numpy(clip[None, :].copy()), cfg, dev, steps=10)["ms_per_step"] * 1e3
        row["speedup_bf16_vs_stft"] = row["torch_stft_us"] / row["melt_bf16_us"]
        res["mels_160s"].append(row)
    # the same Mel counts on the whole 64 x 30 s batch, where neither side is
    # launch-bound: inputs rotate over two device copies (246 MB > L2)
    res["mels_64x30s"] = []
    clips64, _ = G.workload("rich_64x30s")
    pk = G.pack_clips(clips64)
    waves = [torch.from_numpy(pk.wave).to(dev) for _ in range(2)]
    x64 = torch.from_numpy(np.stack(clips64))
    for M in (40, 80, 128, 256, 512):
        cfg = dict(base, n_mels=M)
        fe = melt.Frontend(precision="bf16", n_mels=M)
        T = fe.total_frames(pk.lengths)
        outs = [torch.empty((T, M), device=dev) for _ in range(2)]
        us = time_launches(lambda i: fe(waves[i % 2], pk.offsets, pk.lengths, out=outs[i % 2], input_ready=True),
                           dev, 10) * 1e3
        fe.close()
        del outs
        row = {"n_mels": M, "frames": T, "melt_bf16_us": us,
               "torch_stft_us": time_stft_batch(x64, cfg, dev, steps=5)["ms_per_step"] * 1e3}
        row["speedup_bf16_vs_stft"] = row["torch_stft_us"] / row["melt_bf16_us"]
        res["mels_64x30s"].append(row)
    return res


def time_correction(args, W, dev, steps=200, warmup=5):
    """BF16 log-Mel with the per-frame correction MLP (80 -> 256 -> 80) attached:
    plain, fused in the kernel's epilogue, and as a separate FP32 pass after it."""
    import torch
    from paper_2606_01009_gb300 import inputs as G
    from paper_2606_01009_gb300 import melt
    cfg = W.cfg
    fe = melt.Frontend(sr=cfg["sr"], n_fft=cfg["n_fft"], hop=cfg["hop"], n_mels=cfg["n_mels"],
                       fmin=cfg["fmin"], fmax=cfg["fmax"], precision="bf16")
    M, Hd = fe.n_out, 256
    T = fe.total_frames(W.lens)
    waves, outs, copies = W.device_copies(M, T)
    stream = torch.cuda.current_stream(dev)
    fe(waves[0], W.offs, W.lens, out=outs[0], stream=stream)
    mlp = melt.melt_mlp_create(M, Hd, melt.pack_mlp_params(G.xavier_uniform(3, Hd, M, 0), np.zeros(Hd),
                                                            G.xavier_uniform(3, M, Hd, 1), np.zeros(M)))
    melt.melt_mlp_fit_stats(mlp, outs[0], T, stream)

    def timed(fn):
        for i in range(warmup):
            fn(i)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(steps):
            fn(i)
        b.record(stream)
        torch.cuda.synchronize(dev)
        fe.sync(stream)
        return a.elapsed_time(b) / steps * 1e3

    res = {"mlp": f"{M} -> {Hd} -> {M}, GELU", "frames_per_step": T}
    res["plain_us"] = timed(lambda i: fe(waves[i % copies], W.offs, W.lens, out=outs[i % copies], stream=stream))

    def separate(i):
        o = outs[i % copies]
        fe(waves[i % copies], W.offs, W.lens, out=o, stream=stream)
        melt.melt_mlp_forward(mlp, o, o, T, stream)
    res["separate_fp32_pass_us"] = timed(separate)
    melt.melt_basis_set_correction(fe.handle, mlp)
    res["fused_plan"] = melt.melt_plan_get(fe.handle)
    res["fused_bf16_us"] = timed(lambda i: fe(waves[i % copies], W.offs, W.lens, out=outs[i % copies], stream=stream))
    for k in ("plain", "separate_fp32_pass", "fused_bf16"):
        res[k + "_frames_per_s"] = T / (res[k + "_us"] / 1e6)
    melt.melt_basis_set_correction(fe.handle, None)
    fe.close()
    melt.melt_mlp_destroy(mlp)
    return res


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res, default=_jsonable), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    res, W, forms = run_melt(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_oracle_baseline(W.clips, W.cfg, args.mfcc, args.cpu_seconds)
            ok = {k: v for k, v in forms.items() if "error" not in v}
            res["accuracy_db"], res["accuracy_sample"] = accuracy_vs_oracle(W, ok, W.cfg, args.mfcc)
        if args.correction:
            import torch
            try:
                res["correction"] = time_correction(args, W, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
            except Exception as e:  # reported, not fatal: the headline line above stands
                res["correction"] = {"error": str(e)}
        if args.grouped:
            import torch
            try:
                res["grouped"] = time_grouped(args, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
            except Exception as e:  # reported, not fatal: the headline line above stands
                res["grouped"] = {"error": str(e)}
        if args.stft:
            import torch
            try:
                res["torch_stft_context"] = time_torch_stft(
                    W, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
            except Exception as e:  # reported, not fatal: the headline line above stands
                res["torch_stft_context"] = {"error": str(e)}
        if args.stft:
            import torch
            try:
                res["fused_stft_comparator"] = time_fused_stft(
                    W, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))), load_peaks()[0])
            except Exception as e:  # reported, not fatal
                res["fused_stft_comparator"] = {"error": repr(e)}
        if args.configs:
            import torch
            try:
                res["configs"] = config_legs(args, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))),
                                             load_peaks()[0])
            except Exception as e:  # reported, not fatal
                res["configs"] = {"error": repr(e)}
        if args.sweeps:
            import torch
            try:
                res["sweeps"] = sweeps(args, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
            except Exception as e:  # reported, not fatal
                res["sweeps"] = {"error": repr(e)}
        print(json.dumps(res, default=_jsonable), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
