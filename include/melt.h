/*
 * melt.h - C ABI of libmelt, a GB300 (sm_103a) implementation of the MelT /
 * MFCCT audio frontend of arXiv 2606.01009 ("Matmul-Native Mel Frontends").
 *
 * What is computed (paper Sec. III-A):
 *   f_m      M analysis frequencies, uniform on the HTK Mel scale (Eq. 1-2):
 *            the M interior points of M+2 Mel-uniform points on [fmin, fmax]
 *   w[n]     Hann window of length N (periodic or symmetric)
 *   W_r,W_i  window-folded basis  w[n] cos(2 pi f_m n / sr), w[n] sin(...)  (Eq. 5)
 *   frame t  x[tH .. tH+N-1] of a clip, T = floor((L-N)/H)+1 frames (0 if L<N),
 *            no centring or padding
 *   R, I     R = X W_r^T, I = X W_i^T, one GEMM against [W_r; W_i] (Eq. 6)
 *   S        R^2 + I^2 (Eq. 7)
 *   MelT     log(S + eps), natural log, additive eps (Eq. 8)
 *   MFCCT    log(S + eps) D^T, D = first K rows of the orthonormal DCT-II (Eq. 9)
 *
 * Conventions for every entry point:
 *   - Pointers named "device" are CUDA device pointers of the current device;
 *     "host" pointers are ordinary host memory.  The caller owns every buffer
 *     it passes; the library owns what a melt_basis holds (device basis,
 *     workspace, pinned staging, cached plans) and frees it in melt_destroy.
 *   - A `stream` argument is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Forward calls are asynchronous on that stream and do
 *     not allocate once a basis has seen a batch of the same or larger size.
 *   - Errors are returned as negative melt_status values; nothing aborts.
 *     Errors found by a kernel while it runs (a bounded wait that ran out)
 *     are latched in the basis and reported by melt_sync().
 *   - One melt_basis may be used by one host thread at a time.
 */
#ifndef MELT_H_
#define MELT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct melt_basis melt_basis;

typedef enum {
  MELT_OK = 0,
  MELT_ERR_ARG = -1,          /* invalid argument (null pointer, size, alignment) */
  MELT_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  MELT_ERR_OOM = -3,          /* device or pinned host allocation failed */
  MELT_ERR_UNSUPPORTED = -4,  /* valid request this build or device cannot run */
  MELT_ERR_TIMEOUT = -5,      /* a kernel's bounded wait ran out (pipeline stalled) */
  MELT_ERR_NO_DEVICE = -6     /* no CUDA device, or not an sm_103 device */
} melt_status;

typedef enum { MELT_WIN_HANN_PERIODIC = 0, MELT_WIN_HANN_SYMMETRIC = 1 } melt_window;

/*
 * GEMM operand formats (the paper runs FP32/TF32 only; the reduced forms are
 * this library's).  All accumulate in FP32 and take FP32 waveforms.
 *   MELT_FP32    FP32 samples x FP32 basis on CUDA cores (FFMA).
 *   MELT_BF16    BF16 samples x BF16 basis on tcgen05 tensor cores.
 *   MELT_BF16X3  two-term BF16 splits of both operands, three products
 *                (hi*hi + hi*lo + lo*hi) on tcgen05 tensor cores.
 *   MELT_FP8E4M3 e4m3 samples with a per-frame scale amax(|x_t|)/448 and an
 *                e4m3 basis scaled by 448, on tcgen05 tensor cores.
 */
typedef enum { MELT_FP32 = 0, MELT_BF16 = 1, MELT_BF16X3 = 2, MELT_FP8E4M3 = 3 } melt_precision;

/*
 * melt_basis_create - build the FP64 basis of Sec. III-A (Eq. 1, 2, 5) on the
 * host, round it to the operand format and upload it to the current device.
 *   sr          sample rate in Hz (> 0)
 *   n_fft       frame length N (16..4096, multiple of 4)
 *   hop         hop H (1..n_fft, multiple of 4)
 *   n_mels      M (1..128)
 *   fmin, fmax  0 <= fmin < fmax <= sr/2
 *   window      melt_window
 *   out         receives the new basis (host pointer to a handle)
 * Defaults: MELT_FP32, log-Mel output (no MFCC), eps = 1e-10.
 * Returns MELT_ERR_ARG on a bad parameter, MELT_ERR_NO_DEVICE without an
 * sm_103 device, MELT_ERR_OOM/MELT_ERR_CUDA on allocation or copy failure.
 */
melt_status melt_basis_create(double sr, int n_fft, int hop, int n_mels, double fmin,
                              double fmax, int window, melt_basis** out);

/*
 * melt_basis_create_ex - as melt_basis_create, plus:
 *   precision   melt_precision of the projection GEMM
 *   n_mfcc      K > 0 appends the DCT-II of Eq. 9 (K <= n_mels); 0 = log-Mel
 * More than 128 Mel bins (up to 1024) are supported by MELT_BF16 and
 * MELT_BF16X3 log-Mel bases only (MELT_ERR_UNSUPPORTED otherwise).
 *   eps         additive eps of Eq. 8 (>= 0)
 */
melt_status melt_basis_create_ex(double sr, int n_fft, int hop, int n_mels, double fmin,
                                 double fmax, int window, int precision, int n_mfcc,
                                 double eps, melt_basis** out);

/*
 * melt_basis_create_freqs - basis at caller-chosen analysis frequencies
 * (host array freqs[n_freqs], Hz, each in [0, sr/2]) instead of the Mel
 * centres; used to check the projection against a plain DFT (f_k = k sr/N).
 * Other arguments as melt_basis_create_ex.
 */
melt_status melt_basis_create_freqs(double sr, int n_fft, int hop, const double* freqs,
                                    int n_freqs, int window, int precision, int n_mfcc,
                                    double eps, melt_basis** out);

/* Frames of a clip of `length` samples: floor((L-N)/H)+1, or 0 if L < N (or basis NULL). */
int64_t melt_num_frames(const melt_basis* basis, int64_t length);

/* Values per output frame: n_mfcc if MFCC is on, else n_mels; 0 if basis is NULL. */
int melt_num_outputs(const melt_basis* basis);

/*
 * melt_basis_info - copies basis parameters to host ints/doubles (any may be NULL):
 *   ints[6]    = {n_fft, hop, n_mels, n_mfcc, precision, window}
 *   doubles[4] = {sr, fmin, fmax, eps}
 */
melt_status melt_basis_info(const melt_basis* basis, int* ints, double* doubles);

/*
 * melt_basis_get_fp64 - copy the host FP64 basis before rounding (Eq. 5) to
 *   freqs  host double[n_mels]            analysis frequencies f_m in Hz
 *   w      host double[2*n_mels*n_fft]    rows 0..M-1 = W_r, rows M..2M-1 = W_i,
 *                                         row-major (n fastest)
 * Either pointer may be NULL.
 */
melt_status melt_basis_get_fp64(const melt_basis* basis, double* freqs, double* w);

/*
 * Layout of the tensor-core pipeline in shared memory (BF16 / BF16X3 / FP8
 * bases).  The library picks one by default; melt_autotune times the
 * candidates on a real batch and keeps the fastest.
 *   basis_resident   1: the whole basis is loaded once per CTA and kept in
 *                    shared memory; 0: it is streamed from L2 through a ring
 *   a_buffers        MMA A-operand (frame sample) buffers: 1 or 2
 *   prefetch_tiles   0..4: how many tiles ahead of the converters the CTA's
 *                    waveform spans are prefetched into L2 (the converters
 *                    read samples from global memory; no shared memory is
 *                    spent on them)
 *   basis_slots      streamed-basis ring slots (ignored when resident)
 *   ksteps_per_slot  basis K-steps (16 samples each; FP8: 32) per streamed slot
 *   cta_pair         1 (BF16 and FP8): clusters of two CTAs share each MMA
 *                    (tcgen05 cta_group::2, 256 frames); each CTA keeps half
 *                    of the basis resident (basis_resident must be 1) and
 *                    stages its waveform span through a ring of bulk copies
 *                    (as many ~14 KB slots as fit; prefetch_tiles is how many
 *                    tiles ahead the spans are prefetched into L2 besides;
 *                    basis_slots and ksteps_per_slot are ignored).  0: one
 *                    CTA per MMA.
 *   schedule         CTA pairs only.  0: static, cluster c takes pairs c,
 *                    c + C, c + 2C, ... (C clusters).  1: dynamic, cluster c
 *                    takes pair c, then claims each next pair from a
 *                    launch-wide counter one pair ahead, so clusters that
 *                    run faster take more (prefetch_tiles is then ignored).
 *                    The counter lives in the basis (one per launch, 16
 *                    launches of one basis may be in flight at once).
 */
typedef struct {
  int basis_resident;
  int a_buffers;
  int prefetch_tiles;
  int basis_slots;
  int ksteps_per_slot;
  int cta_pair;
  int schedule;
} melt_plan;

/* melt_plan_get - the layout the next forward will use (host struct out).
 * MELT_ERR_UNSUPPORTED for an FP32 (CUDA-core) basis, which has no layout. */
melt_status melt_plan_get(const melt_basis* basis, melt_plan* plan);

/* melt_plan_set - force a layout (plan NULL = back to the default choice).
 * MELT_ERR_UNSUPPORTED if it does not fit in shared memory; the previous
 * layout is then kept. */
melt_status melt_plan_set(melt_basis* basis, const melt_plan* plan);

/*
 * melt_autotune - run melt_forward on the given batch (same arguments, `out`
 * is overwritten) once per candidate layout, `reps` timed runs each after
 * one warm-up, keep the fastest and return it in *best (may be NULL).
 * Synchronises `stream`.  Not for use inside stream capture.
 */
melt_status melt_autotune(melt_basis* basis, const float* wave, const int64_t* offsets,
                          const int64_t* lengths, int batch, float* out, void* stream, int reps,
                          melt_plan* best);

/*
 * melt_autotune_file - melt_autotune with a plan cache on disk, so that a
 *   process tunes a configuration once and later processes reuse the plan.
 *   The file at `path` (text, one line per tuned configuration, created if
 *   missing) is read first.  A line for this GPU (by name), this basis
 *   configuration (n_fft, hop, frequency count, precision, n_mfcc, fused
 *   correction's hidden units, comparator bands) and this batch size class
 *   (log2 of the batch's tile count) that still fits the device sets its plan
 *   without timing (*hit = 1).  Otherwise melt_autotune runs (arguments as
 *   there) and its plan is appended as one line (*hit = 0).  The plan in
 *   effect is returned in *best.  `best` and `hit` may be NULL.
 *   Errors: those of melt_autotune; MELT_ERR_ARG for a NULL path;
 *   MELT_ERR_CUDA if the device name cannot be read.  A file that cannot be
 *   written only skips the append.
 */
melt_status melt_autotune_file(melt_basis* basis, const float* wave, const int64_t* offsets,
                               const int64_t* lengths, int batch, float* out, void* stream, int reps,
                               const char* path, melt_plan* best, int* hit);

/*
 * melt_forward - MelT (Eq. 8) or MFCCT (Eq. 9) features of a batch of clips.
 *   wave     device float[]: clip b occupies wave[offsets[b] .. offsets[b]+lengths[b]);
 *            the whole 4-float-aligned span [offsets[b], offsets[b]+round_up(lengths[b],4))
 *            must be readable (its tail beyond lengths[b] is never used).
 *            wave must be 16-byte aligned.
 *   offsets  host int64[batch], each a multiple of 4 (NULL = clips packed back to
 *            back at 4-float alignment: offsets[b] = sum_{c<b} round_up(lengths[c],4))
 *   lengths  host int64[batch], each >= 0
 *   batch    number of clips (>= 0; 0 is a no-op)
 *   out      device float[sum_b T_b * n_out], 16-byte aligned: clip after clip,
 *            frame-major, n_out = melt_num_outputs(basis) values per frame
 *   stream   cudaStream_t as void*
 * Asynchronous; the host arrays may be reused as soon as it returns.
 * Returns MELT_ERR_ARG for a bad pointer, alignment or length.
 */
melt_status melt_forward(melt_basis* basis, const float* wave, const int64_t* offsets,
                         const int64_t* lengths, int batch, float* out, void* stream);

/* Flags of melt_forward_ex. */
enum { MELT_FWD_INPUT_READY = 1 };

/*
 * melt_forward_ex - melt_forward with call flags; the features are the same
 *   (Eq. 8 / Eq. 9), bit for bit.  Every tensor-core launch may start while
 *   the kernel before it on `stream` is still running (programmatic dependent
 *   launch); by default each of its roles that reads the waveform waits for
 *   that kernel to finish first.
 *   flags  0 or MELT_FWD_INPUT_READY.  With MELT_FWD_INPUT_READY the caller
 *          states that no kernel enqueued on `stream` since the host last
 *          synchronised with it writes `wave` (the samples came from copies,
 *          from work on other streams that `stream` waits for through events,
 *          or from work already synchronised).  The launch then stages and
 *          converts samples, and runs its MMAs, while the preceding kernel
 *          drains; it still stores features only after that kernel has
 *          finished.  A batch produced by a kernel on `stream` (for example
 *          melt_pad_reflect) must not use the flag.  The FP32 form and the
 *          dynamic pair schedule ignore it.
 *   Other arguments and errors as melt_forward; MELT_ERR_ARG for an unknown flag.
 */
melt_status melt_forward_ex(melt_basis* basis, const float* wave, const int64_t* offsets,
                            const int64_t* lengths, int batch, float* out, void* stream, unsigned flags);

/*
 * melt_forward_noalloc - melt_forward without any allocation at call time.
 *   The paper has no counterpart: this entry point exists for callers that
 *   must not allocate device memory once running - a real-time audio thread
 *   (cudaMalloc can block on driver locks and synchronise the device), a
 *   process whose device memory is already reserved by another framework's
 *   caching allocator, or a deployment that fixes its memory footprint at
 *   start-up.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   Arguments, layouts and results are those of melt_forward.
 *   Scratch: the per-call tile list lives in one file-scope device array of
 *     16384 tiles (512 KiB; one tile = up to 128 frames of one clip, so each
 *     clip needs ceil(T_b / 128) tiles), held by every device that loads the
 *     library until the process exits.  A batch that needs more tiles is
 *     rejected with MELT_ERR_ARG before anything is launched.
 *   The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     outside any stream capture.  The basis must belong to the current
 *     device.
 *   All calls share the array, which keeps the previous call's descriptors;
 *     each call rewrites every entry it uses, so nothing needs clearing.
 *     Calls whose work overlaps on the GPU (different streams without
 *     ordering) race on the array: order them on one stream, or wait.
 *   Host-side planning uses a file-scope host array guarded by a mutex; the
 *     plan reaches the device array by a copy from that pageable host array,
 *     which the driver stages before the call returns.  The call may
 *     therefore block until the work already queued on `stream` has
 *     finished, and it holds the mutex meanwhile, so concurrent calls from
 *     other threads wait too.  A pageable copy cannot be replayed by a CUDA
 *     graph: while `stream` is being captured the call returns
 *     MELT_ERR_UNSUPPORTED and enqueues nothing.
 */
melt_status melt_forward_noalloc(melt_basis* basis, const float* wave, const int64_t* offsets,
                                 const int64_t* lengths, int batch, float* out, void* stream);

/*
 * melt_forward_host - melt_forward on a batch held in host memory: the same
 *   features (Eq. 8 / Eq. 9), bit for bit, with the host<->device transfers
 *   done by the library and overlapped with the kernels.  The batch is cut
 *   into chunks of whole clips; each chunk's samples are copied to a device
 *   slot, processed and its features copied back on one of four internal
 *   streams, so the copies of some chunks run while others compute.
 *   wave     host float[], clip b at wave[offsets[b] .. offsets[b]+lengths[b])
 *            (page-locked memory lets the copies run asynchronously; any
 *            host memory is accepted)
 *   offsets  host int64[batch], multiples of 4, non-decreasing (NULL = packed
 *            back to back at 4-float alignment, as for melt_forward)
 *   lengths  host int64[batch]
 *   out      host float[sum_b T_b * n_out]
 *   stream   work already queued on `stream` happens before the copies, and
 *            later work on `stream` happens after every feature is in `out`;
 *            the call returns before that (synchronise `stream` before
 *            reading `out` or reusing `wave`).
 * The basis keeps the device slots, the four streams and the chunk plan of
 * the last batch layout (they grow to the largest chunk seen and are freed
 * by melt_destroy).  The correction MLP, if attached, is applied as in
 * melt_forward.  MELT_ERR_ARG for bad pointers, lengths, unordered offsets or
 * a basis of another device.
 */
melt_status melt_forward_host(melt_basis* basis, const float* wave, const int64_t* offsets,
                              const int64_t* lengths, int batch, float* out, void* stream);

/*
 * melt_pad_reflect - centred framing.  The paper frames each clip from its
 *   first sample (Sec. III-A, Eq. 6: no padding).  Frontends built on a
 *   centred STFT pad each clip with N/2 samples of reflection at both ends,
 *   so that frame t is centred on sample t*H and a clip of L samples gives
 *   floor(L/H) + 1 frames (for even N).  This call writes that padded batch;
 *   melt_forward on it (lengths + 2*pad) gives the centred features.
 *   Clip b of L = lengths[b] samples becomes y[0 .. L + 2 pad) with
 *   y[i] = x[r(i - pad)], r(j) = -j for j < 0, 2 (L-1) - j for j >= L, j
 *   otherwise (reflection without repeating the edge sample).
 *   wave         device float[], clip b at wave[offsets[b] ..] (NULL offsets:
 *                packed at 4-float alignment, as for melt_forward)
 *   lengths      host int64[batch]; every clip needs lengths[b] > pad
 *   pad          samples added at each end (N/2 for centred frames), >= 0
 *   out          device float[], padded clip b at out[out_offsets[b] ..],
 *                lengths[b] + 2 pad floats; it must not overlap wave
 *   out_offsets  host int64[batch] (NULL: packed at 4-float alignment, which
 *                keeps every padded clip's start 16-byte aligned for
 *                melt_forward)
 *   Asynchronous on `stream`; allocates nothing (the clip descriptors travel
 *   in the kernels' parameters, 1000 clips per launch).  Errors:
 *   MELT_ERR_ARG for bad arguments or a clip of at most pad samples (nothing
 *   is launched), MELT_ERR_CUDA for a failed launch.
 */
melt_status melt_pad_reflect(const float* wave, const int64_t* offsets, const int64_t* lengths,
                             int batch, int pad, float* out, const int64_t* out_offsets, void* stream);

/*
 * Conventional STFT + triangular Mel pipeline, fused into one kernel: the
 * comparator the paper names as future work (Sec. "Threats to Validity",
 * baseline and comparison fairness: a fused STFT+Mel kernel as a stronger
 * conventional baseline), built from this library's own parts.
 *
 * melt_stft_create - a basis whose melt_forward computes, per frame,
 *     out[m] = log( sum_k F[m][k] |X_k|^2 + eps ),   m < n_mels,
 *   |X_k|^2 the power of the DFT of the windowed frame at the N/2 + 1 uniform
 *   frequencies k sr / N (k = 0 .. N/2): the projection of Eq. 6 onto the
 *   window-folded cos/sin rows at those frequencies, a tensor-core GEMM with
 *   the power, the filterbank and the log fused in its epilogue.  F is the
 *   triangular filterbank with n_mels bands on n_mels + 2 edges spaced
 *   uniformly between fmin and fmax on the Mel scale chosen by `scale`:
 *     0  HTK scale (Eq. 1), peak-1 triangles
 *     1  Slaney scale (linear below 1 kHz, logarithmic above), triangles of
 *        unit area (weights 2 / (edge[m+2] - edge[m]))
 *   Band m rises from edge m to edge m+1 and falls to edge m+2.
 *   sr, n_fft, hop, window, eps   as melt_basis_create_ex (N/2 + 1 <= 1024)
 *   n_mels      bands, 1..512
 *   precision   MELT_BF16 or MELT_BF16X3
 *   out         receives the basis; melt_num_outputs(basis) = n_mels
 * Framing, batching and the forward entry points (melt_forward and its
 * variants) are those of any basis; a correction MLP cannot be attached.
 * MELT_ERR_UNSUPPORTED for another precision or n_fft; MELT_ERR_ARG for a
 * bad parameter.
 */
melt_status melt_stft_create(double sr, int n_fft, int hop, int n_mels, double fmin, double fmax, int window,
                             int precision, int scale, double eps, melt_basis** out);

/*
 * melt_forward_components - debug form: the raw projection (Eq. 6) for every
 * frame, out = device float[sum_b T_b * 2M]: per frame M values of R then M of I.
 * Only MELT_FP32 bases.  Arguments otherwise as melt_forward.
 */
melt_status melt_forward_components(melt_basis* basis, const float* wave,
                                    const int64_t* offsets, const int64_t* lengths,
                                    int batch, float* out, void* stream);

/*
 * Grouped launch over several bases (batching across configurations, Sec. V).
 *
 * A melt_group holds up to MELT_MAX_GROUPS bases of one device whose outputs
 * have the same width (melt_num_outputs); their frame geometries, precisions
 * and layout plans may differ (e.g. 16 kHz 400/160/80 and 22.05 kHz
 * 1024/256/80).  One call plans a work list of tiles (basis, clip, 128-frame
 * run), copies it to the device once per batch layout, and runs one
 * persistent kernel per basis over its part of the list.  With
 * MELT_GROUP_SHARED, two BF16 log-Mel bases (without a correction, with
 * CTA-pair plans or default plans) share one persistent launch instead: the
 * clusters are split between the bases (melt_group_set_split; by default in
 * proportion to tiles x n_fft) and each cluster runs its basis's layout (a
 * basis whose default plan is single-CTA takes its first CTA-pair plan
 * there; a forced single-CTA plan keeps the per-basis launches).  On the
 * 4096-clip 16 kHz + 22.05 kHz batch the shared launch measured slower
 * (1.05 ms at its best split against 0.81 ms), hence not the default.
 * Unless disabled, the launches of a batch layout are captured once into a
 * CUDA graph and replayed by later calls with the same layout.
 */
#define MELT_MAX_GROUPS 16
#define MELT_GROUP_NO_GRAPH 1   /* melt_group_create flag: launch directly, no graph */
#define MELT_GROUP_SHARED 2     /* melt_group_create flag: two bases in one shared persistent launch */

typedef struct melt_group melt_group;

/*
 * melt_group_create - bundle `n_bases` bases (host array of handles, 1..16,
 * all created on the current device, equal melt_num_outputs).  The group
 * does not own the bases: destroy the group first.  `flags`: 0 or an OR of
 * MELT_GROUP_NO_GRAPH and MELT_GROUP_SHARED.  Returns MELT_ERR_ARG on a bad
 * argument.
 */
melt_status melt_group_create(melt_basis* const* bases, int n_bases, int flags, melt_group** out);

/*
 * melt_forward_grouped - features of a batch whose clips use different bases.
 *   wave       device float[], clips packed as for melt_forward (16-byte aligned starts)
 *   offsets    host int64[batch] start of clip b in wave (floats, multiple of 4),
 *              or NULL for back-to-back packing rounded up to 4 floats
 *   lengths    host int64[batch] samples of clip b
 *   basis_of   host int32[batch] index (0..n_bases-1) of the basis of clip b
 *   out        device float[sum_b T_b * n_out]: the frames of clip b, with
 *              T_b = floor((L_b - N_g)/H_g) + 1 of its basis g, in batch order
 * Asynchronous on `stream`.  A batch layout not seen before (same pointers,
 * offsets, lengths and basis indices) allocates its device work list and,
 * with graphs, captures a graph; the group caches the last 8 layouts.
 * Results equal melt_forward on each clip with its own basis, bit for bit.
 */
melt_status melt_forward_grouped(melt_group* group, const float* wave, const int64_t* offsets,
                                 const int64_t* lengths, const int32_t* basis_of, int batch,
                                 float* out, void* stream);

/*
 * melt_group_autotune - layout plans for the bases of a group, chosen by
 *   timing melt_forward_grouped's launches on the given batch (arguments as
 *   there), so that each basis is tuned as it runs beside the others.  The
 *   bases are tuned one at a time: each of a basis's candidate plans is set
 *   (melt_plan_set), the whole grouped launch runs once as warm-up and then
 *   `reps` times under events, and the fastest candidate stays set before
 *   the next basis is tuned.  FP32 bases have no plans and keep theirs.
 *   The plans stay set on the bases (as melt_plan_set leaves them), and the
 *   group's cached work lists and graphs are dropped, so the next
 *   melt_forward_grouped captures the tuned launches.
 *   path   plan cache file (text, created if missing) or NULL.  A line for this
 *          GPU (by name), these basis configurations and the size class of each
 *          basis's share of the batch (floor(log2) of its tile count) sets its
 *          plans without timing (*hit = 1); after tuning, one line is appended.
 *          A file that cannot be written only skips the append.
 *   hit    may be NULL.
 *   Writes `out` (as the forward would), synchronises `stream`.  Not for use
 *   inside stream capture.  Errors: those of melt_forward_grouped;
 *   MELT_ERR_ARG for reps < 1.
 */
melt_status melt_group_autotune(melt_group* group, const float* wave, const int64_t* offsets,
                                const int64_t* lengths, const int32_t* basis_of, int batch, float* out,
                                void* stream, int reps, const char* path, int* hit);

/*
 * melt_group_set_split - the first basis's share of the clusters in the
 * shared launch of a two-basis group (0 <= frac0 < 1; 0 = in proportion to
 * tiles x n_fft, the default).  Drops the group's recorded graphs.
 * MELT_ERR_ARG outside that range.
 */
melt_status melt_group_set_split(melt_group* group, double frac0);

/* melt_group_sync - melt_sync of every basis of the group; first error wins. */
melt_status melt_group_sync(melt_group* group, void* stream);

/* melt_group_destroy - free the group's work lists and graphs (NULL is a no-op). */
melt_status melt_group_destroy(melt_group* group);

/*
 * Learned per-frame correction (a residual MLP on the log-Mel bands) and its
 * training.  The paper does not evaluate one: Sec. VI-C names a calibration
 * layer as untested, and Sec. IV-H / Sec. V describe the MelT-to-STFT+Mel gap
 * as mostly a per-band affine map.  The model, for a frame x of M log-Mel
 * values:
 *   xh = (x - mu) / sd                        fixed per-band statistics
 *   y  = x + W2 GELU(W1 xh + b1) + b2         W1 [Hd x M], W2 [M x Hd], exact-erf GELU
 * trained on MSE = mean over rows and bands of (y - target)^2 with AdamW
 * (decoupled weight decay on every parameter).  All arithmetic is FP32.
 *
 * Parameters are one packed FP32 vector, row-major blocks in this order:
 *   W1 [Hd][M], b1 [Hd], W2 [M][Hd], b2 [M]   (melt_mlp_num_params floats)
 * Matrices X, target, Y are device float [rows][M], row-major.
 */
typedef struct melt_mlp melt_mlp;

/* Number of floats of the packed parameter vector (0 for bad sizes). */
int64_t melt_mlp_num_params(int n_in, int n_hidden);

/*
 * melt_mlp_create - upload initial parameters (host, packed as above) and the
 * per-band statistics mu, sd (host float[n_in]; NULL = 0 and 1) to the current
 * device.  n_in = M in 1..128; n_hidden = Hd, a multiple of 64 in 64..4096.
 * AdamW defaults: lr 1e-3, betas (0.9, 0.999), eps 1e-8, weight decay 0.01.
 */
melt_status melt_mlp_create(int n_in, int n_hidden, const float* params, const float* mu,
                            const float* sd, melt_mlp** out);

/* Set mu, sd to the population mean and standard deviation (floor 1e-6) of
 * the n rows of X (device).  Asynchronous on `stream`. */
melt_status melt_mlp_fit_stats(melt_mlp* mlp, const float* X, int64_t n, void* stream);

/* AdamW hyper-parameters for later steps (lr >= 0, 0 <= betas < 1, eps > 0, wd >= 0). */
melt_status melt_mlp_set_adamw(melt_mlp* mlp, double lr, double beta1, double beta2, double eps,
                               double wd);

/*
 * melt_mlp_grad - loss gradient over one batch, without updating anything.
 *   X, target  device float[*][M]
 *   rows       device int64[batch]: the batch is rows[0..batch) of X/target;
 *              NULL = rows 0..batch-1
 *   grads      device float[num_params] (packed like the parameters), or NULL
 *              for the internal buffer
 *   loss       device float accumulator: the sum of squared errors over the
 *              batch is ADDED to *loss (divide by batch*M for the MSE), or NULL
 * Asynchronous on `stream`; the workspace grows to the largest batch seen.
 */
melt_status melt_mlp_grad(melt_mlp* mlp, const float* X, const float* target, const int64_t* rows,
                          int batch, float* grads, float* loss, void* stream);

/* melt_mlp_train_step - melt_mlp_grad, then one AdamW update (step count += 1). */
melt_status melt_mlp_train_step(melt_mlp* mlp, const float* X, const float* target,
                                const int64_t* rows, int batch, float* loss, void* stream);

/* melt_mlp_adamw_apply - one AdamW update with caller gradients (device, packed). */
melt_status melt_mlp_adamw_apply(melt_mlp* mlp, const float* grads, void* stream);

/* melt_mlp_forward - y = x + W2 GELU(W1 xh + b1) + b2 for n rows; Y == X allowed. */
melt_status melt_mlp_forward(const melt_mlp* mlp, const float* X, float* Y, int64_t n, void* stream);

/* Copy parameters, mu and sd to host buffers (any may be NULL).  Synchronises the device. */
melt_status melt_mlp_get_params(const melt_mlp* mlp, float* params, float* mu, float* sd);

/* Free the MLP (NULL is a no-op).  Detach it from every basis first.  Synchronises the device. */
melt_status melt_mlp_destroy(melt_mlp* mlp);

/*
 * melt_basis_set_correction - apply `mlp` in place to the output of every
 * later melt_forward / melt_forward_noalloc of this log-Mel basis (NULL
 * detaches).  The basis does not own the MLP.  MELT_ERR_UNSUPPORTED for an
 * MFCC basis; MELT_ERR_ARG if the MLP's band count or device differ.
 * melt_forward_grouped refuses bases with a correction (MELT_ERR_UNSUPPORTED).
 */
melt_status melt_basis_set_correction(melt_basis* basis, const melt_mlp* mlp);

/*
 * melt_sync - wait for `stream`, then report (and clear) any error a kernel of
 * this basis latched while running (MELT_ERR_TIMEOUT), else the stream's own
 * CUDA status.
 */
melt_status melt_sync(melt_basis* basis, void* stream);

/* melt_destroy - free everything the basis owns (NULL is a no-op). Synchronises the device. */
melt_status melt_destroy(melt_basis* basis);

/* Static English text for a status code. */
const char* melt_status_string(int status);

/* Library version string, e.g. "melt 0.1 sm_103a". */
const char* melt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MELT_H_ */
