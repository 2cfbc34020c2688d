"""Thin ctypes binding of libmelt (include/melt.h), same names as the C ABI.

Argument marshalling only: every step of the MelT path runs in libmelt's
CUDA kernels.  torch is used for device memory and streams.  If libmelt.so
has not been built, importing this module raises (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmelt.so")

MELT_OK = 0
MELT_ERR_ARG = -1
MELT_ERR_CUDA = -2
MELT_ERR_OOM = -3
MELT_ERR_UNSUPPORTED = -4
MELT_ERR_TIMEOUT = -5
MELT_ERR_NO_DEVICE = -6

MELT_WIN_HANN_PERIODIC = 0
MELT_WIN_HANN_SYMMETRIC = 1

MELT_MAX_GROUPS = 16
MELT_GROUP_NO_GRAPH = 1
MELT_GROUP_SHARED = 2

MELT_FWD_INPUT_READY = 1

MELT_FP32 = 0
MELT_BF16 = 1
MELT_BF16X3 = 2
MELT_FP8E4M3 = 3
PRECISIONS = {"fp32": MELT_FP32, "bf16": MELT_BF16, "bf16x3": MELT_BF16X3, "fp8": MELT_FP8E4M3}

# Every symbol include/melt.h declares, with (restype, argtypes).
_VP = C.c_void_p
_I64P = C.POINTER(C.c_int64)
SIGNATURES = {
    "melt_basis_create": (C.c_int, [C.c_double, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_int, C.POINTER(_VP)]),
    "melt_basis_create_ex": (C.c_int, [C.c_double, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.c_double, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.POINTER(_VP)]),
    "melt_basis_create_freqs": (C.c_int, [C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double),
                                          C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                          C.POINTER(_VP)]),
    "melt_num_frames": (C.c_int64, [_VP, C.c_int64]),
    "melt_num_outputs": (C.c_int, [_VP]),
    "melt_basis_info": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "melt_basis_get_fp64": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "melt_forward": (C.c_int, [_VP, _VP, _I64P, _I64P, C.c_int, _VP, _VP]),
    "melt_forward_ex": (C.c_int, [_VP, _VP, _I64P, _I64P, C.c_int, _VP, _VP, C.c_uint]),
    "melt_group_set_split": (C.c_int, [_VP, C.c_double]),
    "melt_stft_create": (C.c_int, [C.c_double, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                   C.c_int, C.c_int, C.c_double, C.POINTER(_VP)]),
    "melt_forward_components": (C.c_int, [_VP, _VP, _I64P, _I64P, C.c_int, _VP, _VP]),
    "melt_forward_noalloc": (C.c_int, [_VP, _VP, _I64P, _I64P, C.c_int, _VP, _VP]),
    "melt_forward_host": (C.c_int, [_VP, _VP, _I64P, _I64P, C.c_int, _VP, _VP]),
    "melt_pad_reflect": (C.c_int, [_VP, _I64P, _I64P, C.c_int, C.c_int, _VP, _I64P, _VP]),
    "melt_diag_wait_timeout": (C.c_int, [_VP, _VP]),
    "melt_diag_alloc_count": (C.c_longlong, []),
    "melt_diag_gelu": (C.c_int, [_VP, _VP, C.c_int64, _VP]),
    "melt_diag_log": (C.c_int, [_VP, _VP, C.c_int64, _VP]),
    "melt_plan_get": (C.c_int, [_VP, _VP]),
    "melt_plan_set": (C.c_int, [_VP, _VP]),
    "melt_autotune": (C.c_int, [_VP, _VP, _I64P, _I64P, C.c_int, _VP, _VP, C.c_int, _VP]),
    "melt_autotune_file": (C.c_int, [_VP, _VP, _I64P, _I64P, C.c_int, _VP, _VP, C.c_int, C.c_char_p, _VP,
                                     C.POINTER(C.c_int)]),
    "melt_group_create": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_int, C.POINTER(_VP)]),
    "melt_forward_grouped": (C.c_int, [_VP, _VP, _I64P, _I64P, C.POINTER(C.c_int32), C.c_int, _VP, _VP]),
    "melt_group_sync": (C.c_int, [_VP, _VP]),
    "melt_group_autotune": (C.c_int, [_VP, _VP, _I64P, _I64P, C.POINTER(C.c_int32), C.c_int, _VP, _VP, C.c_int,
                                      C.c_char_p, C.POINTER(C.c_int)]),
    "melt_group_destroy": (C.c_int, [_VP]),
    "melt_mlp_num_params": (C.c_int64, [C.c_int, C.c_int]),
    "melt_mlp_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                  C.POINTER(C.c_float), C.POINTER(_VP)]),
    "melt_mlp_fit_stats": (C.c_int, [_VP, _VP, C.c_int64, _VP]),
    "melt_mlp_set_adamw": (C.c_int, [_VP, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]),
    "melt_mlp_grad": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int, _VP, _VP, _VP]),
    "melt_mlp_train_step": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int, _VP, _VP]),
    "melt_mlp_adamw_apply": (C.c_int, [_VP, _VP, _VP]),
    "melt_mlp_forward": (C.c_int, [_VP, _VP, _VP, C.c_int64, _VP]),
    "melt_mlp_get_params": (C.c_int, [_VP, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "melt_mlp_destroy": (C.c_int, [_VP]),
    "melt_basis_set_correction": (C.c_int, [_VP, _VP]),
    "melt_sync": (C.c_int, [_VP, _VP]),
    "melt_destroy": (C.c_int, [_VP]),
    "melt_status_string": (C.c_char_p, [C.c_int]),
    "melt_version": (C.c_char_p, []),
}


class MeltPlan(C.Structure):
    """melt_plan: layout of the tensor-core pipeline in shared memory."""
    _fields_ = [("basis_resident", C.c_int), ("a_buffers", C.c_int), ("prefetch_tiles", C.c_int),
                ("basis_slots", C.c_int), ("ksteps_per_slot", C.c_int),
                ("cta_pair", C.c_int),
                ("schedule", C.c_int)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class MeltError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmelt.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def status_string(status: int) -> str:
    return lib.melt_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != MELT_OK:
        raise MeltError(status, what)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _i64(a):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    return arr, arr.ctypes.data_as(_I64P)


# ------------------------------------------------------------------ C names
def melt_basis_create(sr, n_fft, hop, n_mels, fmin, fmax, window=MELT_WIN_HANN_PERIODIC):
    h = C.c_void_p()
    _check(lib.melt_basis_create(sr, n_fft, hop, n_mels, fmin, fmax, window, C.byref(h)),
           "melt_basis_create")
    return h


def melt_basis_create_ex(sr, n_fft, hop, n_mels, fmin, fmax, window=MELT_WIN_HANN_PERIODIC,
                         precision=MELT_FP32, n_mfcc=0, eps=1e-10):
    h = C.c_void_p()
    _check(lib.melt_basis_create_ex(sr, n_fft, hop, n_mels, fmin, fmax, window, precision, n_mfcc,
                                    eps, C.byref(h)), "melt_basis_create_ex")
    return h


def melt_basis_create_freqs(sr, n_fft, hop, freqs, window=MELT_WIN_HANN_PERIODIC,
                            precision=MELT_FP32, n_mfcc=0, eps=1e-10):
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
    h = C.c_void_p()
    _check(lib.melt_basis_create_freqs(sr, n_fft, hop, f.ctypes.data_as(C.POINTER(C.c_double)),
                                       int(f.shape[0]), window, precision, n_mfcc, eps,
                                       C.byref(h)), "melt_basis_create_freqs")
    return h


def melt_stft_create(sr, n_fft, hop, n_mels, fmin, fmax, window=MELT_WIN_HANN_PERIODIC, precision=MELT_BF16,
                     scale=0, eps=1e-10):
    """The fused STFT + triangular Mel comparator (scale 0: HTK peak-1, 1: Slaney area)."""
    h = C.c_void_p()
    _check(lib.melt_stft_create(sr, n_fft, hop, n_mels, fmin, fmax, window, precision, scale, eps, C.byref(h)),
           "melt_stft_create")
    return h


def melt_num_frames(basis, length) -> int:
    return int(lib.melt_num_frames(basis, int(length)))


def melt_num_outputs(basis) -> int:
    return int(lib.melt_num_outputs(basis))


def melt_basis_info(basis):
    ints = (C.c_int * 6)()
    dbl = (C.c_double * 4)()
    _check(lib.melt_basis_info(basis, ints, dbl), "melt_basis_info")
    keys_i = ["n_fft", "hop", "n_mels", "n_mfcc", "precision", "window"]
    keys_d = ["sr", "fmin", "fmax", "eps"]
    out = {k: int(v) for k, v in zip(keys_i, ints)}
    out.update({k: float(v) for k, v in zip(keys_d, dbl)})
    return out


def melt_basis_get_fp64(basis):
    info = melt_basis_info(basis)
    M, N = info["n_mels"], info["n_fft"]
    freqs = np.zeros(M, np.float64)
    w = np.zeros((2 * M, N), np.float64)
    _check(lib.melt_basis_get_fp64(basis, freqs.ctypes.data_as(C.POINTER(C.c_double)),
                                   w.ctypes.data_as(C.POINTER(C.c_double))), "melt_basis_get_fp64")
    return freqs, w


def melt_forward(basis, wave, offsets, lengths, out, stream=None, batch=None):
    """wave/out: CUDA float32 tensors (or raw device pointers); offsets/lengths: host int64."""
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    b = int(lens.shape[0]) if batch is None else int(batch)
    wp = wave if isinstance(wave, int) else wave.data_ptr()
    outp = out if isinstance(out, int) else out.data_ptr()
    _check(lib.melt_forward(basis, C.c_void_p(wp), op, lp, b, C.c_void_p(outp), _stream_ptr(stream)),
           "melt_forward")


def melt_forward_ex(basis, wave, offsets, lengths, out, flags, stream=None):
    """melt_forward with call flags (MELT_FWD_INPUT_READY: no kernel enqueued on
    the stream since the last host synchronisation writes ``wave``)."""
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    wp = wave if isinstance(wave, int) else wave.data_ptr()
    outp = out if isinstance(out, int) else out.data_ptr()
    _check(lib.melt_forward_ex(basis, C.c_void_p(wp), op, lp, int(lens.shape[0]), C.c_void_p(outp),
                               _stream_ptr(stream), int(flags)), "melt_forward_ex")


def melt_forward_noalloc(basis, wave, offsets, lengths, out, stream=None):
    """melt_forward with its tile list in a fixed device array: allocates nothing."""
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    wp = wave if isinstance(wave, int) else wave.data_ptr()
    outp = out if isinstance(out, int) else out.data_ptr()
    _check(lib.melt_forward_noalloc(basis, C.c_void_p(wp), op, lp, int(lens.shape[0]), C.c_void_p(outp),
                                    _stream_ptr(stream)), "melt_forward_noalloc")


def melt_pad_reflect(wave, offsets, lengths, pad, out, out_offsets=None, stream=None):
    """Reflection-pad every clip by ``pad`` samples at both ends (centred framing)."""
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    oo, oop = _i64(out_offsets)
    wp = wave if isinstance(wave, int) else wave.data_ptr()
    outp = out if isinstance(out, int) else out.data_ptr()
    _check(lib.melt_pad_reflect(C.c_void_p(wp), op, lp, int(lens.shape[0]), int(pad), C.c_void_p(outp), oop,
                                _stream_ptr(stream)), "melt_pad_reflect")


def melt_diag_wait_timeout(basis, stream=None):
    """Run the failure path of the bounded waits: the next melt_sync reports MELT_ERR_TIMEOUT."""
    _check(lib.melt_diag_wait_timeout(basis, _stream_ptr(stream)), "melt_diag_wait_timeout")


def melt_diag_log(x, y, stream=None):
    """The tensor-core epilogues' natural log on device tensors x -> y (float32)."""
    _check(lib.melt_diag_log(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), int(x.numel()), _stream_ptr(stream)),
           "melt_diag_log")


def melt_diag_gelu(h, y, stream=None):
    """The fused correction epilogue's GELU on device tensors h -> y (float32)."""
    _check(lib.melt_diag_gelu(C.c_void_p(h.data_ptr()), C.c_void_p(y.data_ptr()), int(h.numel()), _stream_ptr(stream)),
           "melt_diag_gelu")


def melt_diag_alloc_count() -> int:
    """Device and page-locked host allocations libmelt has made in this process."""
    return int(lib.melt_diag_alloc_count())


def padded_layout(lengths, pad):
    """Lengths, packed offsets and total floats of a batch after melt_pad_reflect."""
    lens = np.asarray(lengths, dtype=np.int64) + 2 * int(pad)
    sizes = (lens + 3) // 4 * 4
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64) if len(lens) else lens
    return lens, offs, int(sizes.sum())


def melt_forward_host(basis, wave, offsets, lengths, out, stream=None):
    """wave/out: host buffers (numpy arrays or CPU torch tensors, pinned for async copies).

    Asynchronous on `stream`: synchronise it before reading `out`."""
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)

    def hptr(a):
        return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()

    if isinstance(out, np.ndarray) and (out.dtype != np.float32 or not out.flags.c_contiguous):
        raise ValueError("out must be a contiguous float32 array")
    _check(lib.melt_forward_host(basis, C.c_void_p(hptr(wave)), op, lp, int(lens.shape[0]),
                                 C.c_void_p(hptr(out)), _stream_ptr(stream)), "melt_forward_host")


def melt_forward_components(basis, wave, offsets, lengths, out, stream=None):
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    _check(lib.melt_forward_components(basis, C.c_void_p(wave.data_ptr()), op, lp, int(lens.shape[0]),
                                       C.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "melt_forward_components")


def melt_plan_get(basis) -> dict:
    pl = MeltPlan()
    _check(lib.melt_plan_get(basis, C.byref(pl)), "melt_plan_get")
    return pl.as_dict()


def melt_plan_set(basis, plan=None):
    """plan: dict with the melt_plan fields, or None for the default layout."""
    if plan is None:
        _check(lib.melt_plan_set(basis, None), "melt_plan_set")
        return
    pl = MeltPlan(**{k: int(v) for k, v in plan.items()})
    _check(lib.melt_plan_set(basis, C.byref(pl)), "melt_plan_set")


def melt_autotune(basis, wave, offsets, lengths, out, stream=None, reps=5) -> dict:
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    pl = MeltPlan()
    _check(lib.melt_autotune(basis, C.c_void_p(wave.data_ptr()), op, lp, int(lens.shape[0]),
                             C.c_void_p(out.data_ptr()), _stream_ptr(stream), int(reps), C.byref(pl)),
           "melt_autotune")
    return pl.as_dict()


def melt_autotune_file(basis, wave, offsets, lengths, out, path, stream=None, reps=5):
    """melt_autotune with the on-disk plan cache at `path`; returns (plan dict, hit)."""
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    pl = MeltPlan()
    hit = C.c_int(0)
    _check(lib.melt_autotune_file(basis, C.c_void_p(wave.data_ptr()), op, lp, int(lens.shape[0]),
                                  C.c_void_p(out.data_ptr()),
                                  _stream_ptr(stream), int(reps), os.fsencode(path), C.byref(pl), C.byref(hit)),
           "melt_autotune_file")
    return pl.as_dict(), bool(hit.value)


def melt_group_create(bases, flags=0):
    """bases: sequence of basis handles (or Frontends)."""
    hs = [b.handle if hasattr(b, "handle") else b for b in bases]
    arr = (_VP * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    g = C.c_void_p()
    _check(lib.melt_group_create(arr, len(hs), int(flags), C.byref(g)), "melt_group_create")
    return g


def melt_group_set_split(group, frac0):
    """First basis's share of the clusters in a two-basis shared launch (0: by work)."""
    _check(lib.melt_group_set_split(group, float(frac0)), "melt_group_set_split")


def melt_forward_grouped(group, wave, offsets, lengths, basis_of, out, stream=None):
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    ids = np.ascontiguousarray(np.asarray(basis_of, dtype=np.int32))
    if ids.shape[0] != lens.shape[0]:
        raise ValueError("basis_of and lengths differ in length")
    wp = wave if isinstance(wave, int) else wave.data_ptr()
    outp = out if isinstance(out, int) else out.data_ptr()
    _check(lib.melt_forward_grouped(group, C.c_void_p(wp), op, lp, ids.ctypes.data_as(C.POINTER(C.c_int32)),
                                    int(lens.shape[0]), C.c_void_p(outp), _stream_ptr(stream)),
           "melt_forward_grouped")


def melt_group_autotune(group, wave, offsets, lengths, basis_of, out, path=None, stream=None, reps=3) -> bool:
    """Tunes the plans of the group's bases on this batch; returns True on a plan-cache hit."""
    lens, lp = _i64(lengths)
    offs, op = _i64(offsets)
    ids = np.ascontiguousarray(np.asarray(basis_of, dtype=np.int32))
    if ids.shape[0] != lens.shape[0]:
        raise ValueError("basis_of and lengths differ in length")
    hit = C.c_int(0)
    _check(lib.melt_group_autotune(group, C.c_void_p(wave.data_ptr()), op, lp,
                                   ids.ctypes.data_as(C.POINTER(C.c_int32)), int(lens.shape[0]),
                                   C.c_void_p(out.data_ptr()), _stream_ptr(stream), int(reps),
                                   None if path is None else os.fsencode(path), C.byref(hit)),
           "melt_group_autotune")
    return bool(hit.value)


def melt_group_sync(group, stream=None):
    _check(lib.melt_group_sync(group, _stream_ptr(stream)), "melt_group_sync")


def melt_group_destroy(group):
    _check(lib.melt_group_destroy(group), "melt_group_destroy")


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _dptr(t):
    """Device pointer of a torch tensor, an int, or None."""
    if t is None:
        return None
    return C.c_void_p(t if isinstance(t, int) else t.data_ptr())


def melt_mlp_num_params(n_in, n_hidden) -> int:
    return int(lib.melt_mlp_num_params(int(n_in), int(n_hidden)))


def melt_mlp_create(n_in, n_hidden, params, mu=None, sd=None):
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    if p.size != melt_mlp_num_params(n_in, n_hidden):
        raise ValueError("params has the wrong size")
    m = None if mu is None else np.ascontiguousarray(np.asarray(mu, dtype=np.float32))
    s = None if sd is None else np.ascontiguousarray(np.asarray(sd, dtype=np.float32))
    h = C.c_void_p()
    _check(lib.melt_mlp_create(int(n_in), int(n_hidden), _fptr(p), None if m is None else _fptr(m),
                               None if s is None else _fptr(s), C.byref(h)), "melt_mlp_create")
    return h


def melt_mlp_fit_stats(mlp, X, n, stream=None):
    _check(lib.melt_mlp_fit_stats(mlp, _dptr(X), int(n), _stream_ptr(stream)), "melt_mlp_fit_stats")


def melt_mlp_set_adamw(mlp, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01):
    _check(lib.melt_mlp_set_adamw(mlp, lr, beta1, beta2, eps, wd), "melt_mlp_set_adamw")


def melt_mlp_grad(mlp, X, target, rows, batch, grads=None, loss=None, stream=None):
    _check(lib.melt_mlp_grad(mlp, _dptr(X), _dptr(target), _dptr(rows), int(batch), _dptr(grads),
                             _dptr(loss), _stream_ptr(stream)), "melt_mlp_grad")


def melt_mlp_train_step(mlp, X, target, rows, batch, loss=None, stream=None):
    _check(lib.melt_mlp_train_step(mlp, _dptr(X), _dptr(target), _dptr(rows), int(batch), _dptr(loss),
                                   _stream_ptr(stream)), "melt_mlp_train_step")


def melt_mlp_adamw_apply(mlp, grads, stream=None):
    _check(lib.melt_mlp_adamw_apply(mlp, _dptr(grads), _stream_ptr(stream)), "melt_mlp_adamw_apply")


def melt_mlp_forward(mlp, X, Y, n, stream=None):
    _check(lib.melt_mlp_forward(mlp, _dptr(X), _dptr(Y), int(n), _stream_ptr(stream)), "melt_mlp_forward")


def melt_mlp_get_params(mlp, n_in, n_hidden):
    """Returns (params, mu, sd) as float32 numpy arrays."""
    p = np.zeros(melt_mlp_num_params(n_in, n_hidden), np.float32)
    m = np.zeros(n_in, np.float32)
    s = np.zeros(n_in, np.float32)
    _check(lib.melt_mlp_get_params(mlp, _fptr(p), _fptr(m), _fptr(s)), "melt_mlp_get_params")
    return p, m, s


def melt_mlp_destroy(mlp):
    _check(lib.melt_mlp_destroy(mlp), "melt_mlp_destroy")


def melt_basis_set_correction(basis, mlp):
    _check(lib.melt_basis_set_correction(basis, mlp), "melt_basis_set_correction")


def pack_mlp_params(W1, b1, W2, b2) -> np.ndarray:
    """Packed parameter vector [W1 | b1 | W2 | b2] (float32)."""
    return np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in (W1, b1, W2, b2)])


def unpack_mlp_params(p, n_in, n_hidden):
    M, H = n_in, n_hidden
    W1 = p[:H * M].reshape(H, M)
    b1 = p[H * M:H * M + H]
    W2 = p[H * M + H:H * M + H + M * H].reshape(M, H)
    b2 = p[H * M + H + M * H:]
    return W1, b1, W2, b2


def melt_sync(basis, stream=None):
    _check(lib.melt_sync(basis, _stream_ptr(stream)), "melt_sync")


def melt_destroy(basis):
    _check(lib.melt_destroy(basis), "melt_destroy")


def melt_status_string(status: int) -> str:
    return status_string(status)


def melt_version() -> str:
    return lib.melt_version().decode()


# ------------------------------------------------------- convenience object
class Frontend:
    """Owns one melt_basis; calls melt_forward on torch tensors.

    ``precision`` is one of "fp32", "bf16", "bf16x3", "fp8".  ``center=True``
    reflection-pads every clip by n_fft // 2 first (melt_pad_reflect), giving
    floor(L / hop) + 1 frames per clip, each centred on sample t * hop.
    """

    def __init__(self, sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0,
                 window=MELT_WIN_HANN_PERIODIC, precision="fp32", n_mfcc=0, eps=1e-10, freqs=None,
                 center=False):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if freqs is None:
            self.handle = melt_basis_create_ex(sr, n_fft, hop, n_mels, fmin, fmax, window, p, n_mfcc, eps)
        else:
            self.handle = melt_basis_create_freqs(sr, n_fft, hop, freqs, window, p, n_mfcc, eps)
        self.n_out = melt_num_outputs(self.handle)
        # centred framing: every clip reflection-padded by n_fft // 2 first
        # (melt_pad_reflect into one buffer the Frontend keeps; calls on one
        # Frontend must then be ordered on one stream)
        self.center = bool(center)
        self.pad = int(n_fft) // 2 if center else 0
        self._pad_buf = None

    def num_frames(self, length) -> int:
        return melt_num_frames(self.handle, int(length) + 2 * self.pad)

    def total_frames(self, lengths) -> int:
        return sum(self.num_frames(int(L)) for L in lengths)

    def __call__(self, wave, offsets, lengths, out=None, stream=None, input_ready=False):
        """Features of a batch.  input_ready=True passes MELT_FWD_INPUT_READY
        (no kernel enqueued on the stream since the last host synchronisation
        writes ``wave``); centred framing pads with a kernel and ignores it."""
        import torch
        if out is None:
            out = torch.empty((self.total_frames(lengths), self.n_out), device=wave.device,
                              dtype=torch.float32)
        if self.center:
            lens, offs, total = padded_layout(lengths, self.pad)
            if self._pad_buf is None or self._pad_buf.numel() < total or self._pad_buf.device != wave.device:
                self._pad_buf = torch.empty(max(total, 4), device=wave.device, dtype=torch.float32)
            melt_pad_reflect(wave, offsets, lengths, self.pad, self._pad_buf, offs, stream)
            melt_forward(self.handle, self._pad_buf, offs, lens, out, stream)
            return out
        if input_ready:
            melt_forward_ex(self.handle, wave, offsets, lengths, out, MELT_FWD_INPUT_READY, stream)
        else:
            melt_forward(self.handle, wave, offsets, lengths, out, stream)
        return out

    def sync(self, stream=None):
        melt_sync(self.handle, stream)

    def close(self):
        if self.handle is not None:
            melt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StftMelFrontend(Frontend):
    """Owns a fused STFT + triangular Mel comparator basis (melt_stft_create):
    log(F |DFT|^2 + eps) per frame, n_mels bands; same call interface as
    Frontend.  ``scale`` is "htk" (peak-1 triangles) or "slaney" (unit area)."""

    def __init__(self, sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0,
                 window=MELT_WIN_HANN_PERIODIC, precision="bf16", scale="htk", eps=1e-10):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        sc = {"htk": 0, "slaney": 1}[scale] if isinstance(scale, str) else int(scale)
        self.handle = melt_stft_create(sr, n_fft, hop, n_mels, fmin, fmax, window, p, sc, eps)
        self.n_out = melt_num_outputs(self.handle)
        self.center = False
        self.pad = 0
        self._pad_buf = None


class GroupedFrontend:
    """Owns one melt_group over several Frontends (which must outlive it)."""

    def __init__(self, frontends, graphs=True, shared_launch=False):
        """shared_launch=True asks for both bases in one persistent launch (MELT_GROUP_SHARED)."""
        self.frontends = list(frontends)
        if any(fe.center for fe in self.frontends):
            raise ValueError("grouped launches frame clips from their first sample (center=False)")
        self.n_out = self.frontends[0].n_out
        flags = (0 if graphs else MELT_GROUP_NO_GRAPH) | (MELT_GROUP_SHARED if shared_launch else 0)
        self.handle = melt_group_create(self.frontends, flags)

    def total_frames(self, lengths, basis_of):
        return sum(self.frontends[int(g)].num_frames(int(L)) for L, g in zip(lengths, basis_of))

    def __call__(self, wave, offsets, lengths, basis_of, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.total_frames(lengths, basis_of), self.n_out), device=wave.device,
                              dtype=torch.float32)
        melt_forward_grouped(self.handle, wave, offsets, lengths, basis_of, out, stream)
        return out

    def autotune(self, wave, offsets, lengths, basis_of, out, path=None, stream=None, reps=3):
        """Plans of every basis tuned on this batch (melt_group_autotune); returns
        (plans per basis, cache hit)."""
        hit = melt_group_autotune(self.handle, wave, offsets, lengths, basis_of, out, path, stream, reps)
        plans = []
        for fe in self.frontends:
            try:
                plans.append(melt_plan_get(fe.handle))
            except MeltError:
                plans.append(None)
        return plans, hit

    def sync(self, stream=None):
        melt_group_sync(self.handle, stream)

    def close(self):
        if self.handle is not None:
            melt_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
