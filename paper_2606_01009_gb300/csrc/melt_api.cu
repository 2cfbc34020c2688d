// Host side of libmelt: FP64 basis builder, tile planner and the C ABI.
//
// The basis (Sec. III-A, Eq. 1, 2, 5) is built once per configuration in
// FP64 on the host: the phase 2 pi f_m n / sr, its cos/sin and the window
// product are all double precision, and only the finished values are rounded
// to the operand format of the chosen kernel and uploaded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "melt_diag.h"
#include "melt_internal.h"
#include "melt_tc.h"
#include "sm100_ptx.cuh"

using namespace melt;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxFreqs = 1024;  // analysis frequencies of a basis (BF16 forms above 128)
constexpr int kStagingSlots = 4;

// ---- Eq. 1 and Eq. 2: HTK Mel map and its inverse
double hz_to_mel(double f) { return 2595.0 * std::log10(1.0 + f / 700.0); }
double mel_to_hz(double mu) { return 700.0 * (std::pow(10.0, mu / 2595.0) - 1.0); }

struct Staging {
  TileDesc* host = nullptr;    // pinned
  TileDesc* dev = nullptr;
  size_t cap = 0;              // tiles
  size_t n = 0;                // tiles currently held (valid when `key_batch >= 0`)
  cudaEvent_t done = nullptr;  // recorded after the last kernel that read `dev`
  // batch layout the tiles were planned for (plan cache key)
  int key_batch = -1;
  std::vector<int64_t> key_offsets, key_lengths;
  int64_t rows = 0;            // output rows of the batch
};

}  // namespace

struct melt_basis {
  int device = 0;
  int sm_count = 0;
  double sr = 0, fmin = 0, fmax = 0, eps = 1e-10;
  int n_fft = 0, hop = 0, n_mels = 0, n_mfcc = 0, precision = 0, window = 0;
  std::vector<double> freqs;   // [M]
  std::vector<double> w64;     // [2M][N]: W_r rows then W_i rows
  // device data
  int mj = 0, mp = 0;          // SIMT: 16*mj padded mels
  float* d_w32 = nullptr;      // SIMT basis [N][2*mp]
  float* d_dct = nullptr;      // [K][M]
  int* d_err = nullptr;        // latched kernel errors
  TcBasis tc;                  // tensor-core operand images (BF16/FP8 forms)
  Staging staging[kStagingSlots];
  int next_slot = 0;
  std::vector<TileDesc> plan;  // host scratch for planning
  int64_t plan_rows = 0;       // output rows of the planned batch
  const melt_mlp* correction = nullptr;  // applied in place after the log-Mel (not owned)
  // fused STFT + triangular Mel comparator (melt_stft_create): bands per frame
  // and, per DFT bin, {weight of band b0, weight of band b0 + 1, b0 as int bits, 0}
  int stft_bands = 0;
  float4* d_fb = nullptr;
  HostPipe* host_pipe = nullptr;         // melt_forward_host buffers and streams
};

namespace {

melt_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MELT_OK;
  if (e == cudaErrorMemoryAllocation) return MELT_ERR_OOM;
  return MELT_ERR_CUDA;
}

#define MELT_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_status(e_);        \
  } while (0)

void free_basis(melt_basis* b) {
  if (!b) return;
  host_pipe_free(b->host_pipe);
  cudaFree(b->d_w32);
  cudaFree(b->d_dct);
  cudaFree(b->d_err);
  cudaFree(b->d_fb);
  tc_free(&b->tc);
  for (auto& s : b->staging) {
    if (s.done) cudaEventSynchronize(s.done), cudaEventDestroy(s.done);
    cudaFreeHost(s.host);
    cudaFree(s.dev);
  }
  delete b;
}

// Build W_r, W_i (Eq. 5) in FP64.
void build_fp64(melt_basis* b) {
  const int N = b->n_fft, M = b->n_mels;
  const double den = b->window == MELT_WIN_HANN_SYMMETRIC ? (double)(N - 1) : (double)N;
  std::vector<double> w(N);
  for (int n = 0; n < N; ++n) w[n] = 0.5 - 0.5 * std::cos(2.0 * kPi * n / den);
  b->w64.assign((size_t)2 * M * N, 0.0);
  for (int m = 0; m < M; ++m) {
    for (int n = 0; n < N; ++n) {
      const double theta = 2.0 * kPi * b->freqs[m] * (double)n / b->sr;
      b->w64[(size_t)m * N + n] = w[n] * std::cos(theta);
      b->w64[(size_t)(M + m) * N + n] = w[n] * std::sin(theta);
    }
  }
}

melt_status upload_fp32(melt_basis* b) {
  const int N = b->n_fft, M = b->n_mels;
  b->mj = (M + 15) / 16;
  b->mp = 16 * b->mj;
  std::vector<float> h((size_t)N * 2 * b->mp, 0.f);
  for (int n = 0; n < N; ++n)
    for (int m = 0; m < M; ++m) {
      h[(size_t)n * 2 * b->mp + 2 * m] = (float)b->w64[(size_t)m * N + n];
      h[(size_t)n * 2 * b->mp + 2 * m + 1] = (float)b->w64[(size_t)(M + m) * N + n];
    }
  MELT_CUDA(melt::dev_alloc(&b->d_w32, h.size() * sizeof(float)));
  MELT_CUDA(cudaMemcpy(b->d_w32, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
  return MELT_OK;
}

melt_status upload_dct(melt_basis* b) {
  if (b->n_mfcc == 0) return MELT_OK;
  const int K = b->n_mfcc, M = b->n_mels;
  std::vector<float> d((size_t)K * M);
  for (int k = 0; k < K; ++k)
    for (int m = 0; m < M; ++m) {
      double v = std::cos(kPi * k * (2.0 * m + 1.0) / (2.0 * M)) * std::sqrt(2.0 / M);
      if (k == 0) v *= std::sqrt(0.5);
      d[(size_t)k * M + m] = (float)v;
    }
  MELT_CUDA(melt::dev_alloc(&b->d_dct, d.size() * sizeof(float)));
  MELT_CUDA(cudaMemcpy(b->d_dct, d.data(), d.size() * sizeof(float), cudaMemcpyHostToDevice));
  return MELT_OK;
}

melt_status check_device(int* dev, int* sms) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return MELT_ERR_NO_DEVICE;
  MELT_CUDA(cudaGetDevice(dev));
  cudaDeviceProp prop;
  MELT_CUDA(cudaGetDeviceProperties(&prop, *dev));
  if (prop.major != 10 || prop.minor != 3) return MELT_ERR_NO_DEVICE;
  *sms = prop.multiProcessorCount;
  return MELT_OK;
}

melt_status create_common(double sr, int n_fft, int hop, const double* freqs, int n_freqs,
                          double fmin, double fmax, int window, int precision, int n_mfcc,
                          double eps, melt_basis** out, int stft_bands = 0) {
  if (!out) return MELT_ERR_ARG;
  *out = nullptr;
  // more than 128 frequencies: BF16 forms only, log-Mel (the kernels' blocks of 128 bins)
  if (n_freqs > 128 && (precision == MELT_FP32 || precision == MELT_FP8E4M3 || n_mfcc > 0) && n_freqs <= kMaxFreqs &&
      sr > 0 && n_fft >= 16)
    return MELT_ERR_UNSUPPORTED;
  if (!(sr > 0) || n_fft < 16 || n_fft > 4096 || (n_fft & 3) || hop < 1 || hop > n_fft ||
      (hop & 3) || n_freqs < 1 || n_freqs > kMaxFreqs || n_mfcc < 0 || n_mfcc > n_freqs ||
      !(eps >= 0) || (window != MELT_WIN_HANN_PERIODIC && window != MELT_WIN_HANN_SYMMETRIC) ||
      precision < MELT_FP32 || precision > MELT_FP8E4M3)
    return MELT_ERR_ARG;
  for (int m = 0; m < n_freqs; ++m)
    if (!(freqs[m] >= 0.0) || !(freqs[m] <= sr / 2)) return MELT_ERR_ARG;
  int dev = 0, sms = 0;
  melt_status st = check_device(&dev, &sms);
  if (st != MELT_OK) return st;
  melt_basis* b = new (std::nothrow) melt_basis();
  if (!b) return MELT_ERR_OOM;
  b->device = dev;
  b->sm_count = sms;
  b->sr = sr; b->fmin = fmin; b->fmax = fmax; b->eps = eps;
  b->n_fft = n_fft; b->hop = hop; b->n_mels = n_freqs; b->n_mfcc = n_mfcc;
  b->precision = precision; b->window = window;
  b->freqs.assign(freqs, freqs + n_freqs);
  build_fp64(b);
  st = upload_fp32(b);
  if (st == MELT_OK) st = upload_dct(b);
  if (st == MELT_OK && precision != MELT_FP32 && n_mfcc > tc_max_mfcc()) st = MELT_ERR_UNSUPPORTED;
  if (st == MELT_OK && precision != MELT_FP32) {
    TcConfig c{n_fft, hop, n_freqs, precision, n_mfcc, stft_bands};
    st = tc_build(&b->tc, c, b->w64.data());
  }
  if (st == MELT_OK) {
    cudaError_t e = melt::dev_alloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    st = cuda_status(e);
  }
  for (int i = 0; st == MELT_OK && i < kStagingSlots; ++i)
    st = cuda_status(cudaEventCreateWithFlags(&b->staging[i].done, cudaEventDisableTiming));
  if (st != MELT_OK) {
    free_basis(b);
    return st;
  }
  *out = b;
  return MELT_OK;
}

int64_t frames_of(const melt_basis* b, int64_t len) {
  if (len < b->n_fft) return 0;
  return (len - b->n_fft) / b->hop + 1;
}

// The FP32 kernel's CTAs take tiles in list order, round by round, and a
// tile costs it in proportion to its frames (warps past the tile's end
// idle); with the longest tiles first, the last, partly filled round holds
// the short tiles that end clips.  Tiles are independent (each writes its
// own rows), so the order changes no result.
void order_longest_first(TileDesc* t, long long n) {
  std::stable_sort(t, t + n, [](const TileDesc& a, const TileDesc& b) { return a.n_frames > b.n_frames; });
}

// Build the tile list of a batch; returns MELT_ERR_ARG on bad offsets/lengths.
melt_status plan_tiles(melt_basis* b, const int64_t* offsets, const int64_t* lengths, int batch) {
  b->plan.clear();
  int64_t row = 0, off = 0;
  for (int c = 0; c < batch; ++c) {
    const int64_t L = lengths[c];
    if (L < 0) return MELT_ERR_ARG;
    const int64_t o = offsets ? offsets[c] : off;
    if (o < 0 || (o & 3)) return MELT_ERR_ARG;
    off += (L + 3) & ~int64_t(3);
    const int64_t T = frames_of(b, L);
    for (int64_t t0 = 0; t0 < T; t0 += kTileFrames) {
      TileDesc d;
      d.in_off = o + t0 * b->hop;
      d.out_row = row + t0;
      d.n_frames = (int32_t)std::min<int64_t>(kTileFrames, T - t0);
      d.n_samples = (int32_t)std::min<int64_t>(L - t0 * b->hop, INT32_MAX);
      d.group = 0;
      d.clip = c;
      b->plan.push_back(d);
    }
    row += T;
  }
  b->plan_rows = row;
  if (b->precision == MELT_FP32) order_longest_first(b->plan.data(), (long long)b->plan.size());
  return MELT_OK;
}

bool same_layout(const Staging& s, const int64_t* offsets, const int64_t* lengths, int batch) {
  if (s.key_batch != batch) return false;
  if ((offsets == nullptr) != s.key_offsets.empty()) return false;
  if (std::memcmp(s.key_lengths.data(), lengths, sizeof(int64_t) * batch) != 0) return false;
  return !offsets || std::memcmp(s.key_offsets.data(), offsets, sizeof(int64_t) * batch) == 0;
}

// A slot already holding the device tile list of this exact batch layout.
Staging* cached_plan(melt_basis* b, const int64_t* offsets, const int64_t* lengths, int batch) {
  for (auto& s : b->staging)
    if (same_layout(s, offsets, lengths, batch)) return &s;
  return nullptr;
}

// Copy the plan to the device through the next pinned staging slot.
melt_status stage_plan(melt_basis* b, const int64_t* offsets, const int64_t* lengths, int batch,
                       cudaStream_t stream, Staging** slot_out) {
  Staging& s = b->staging[b->next_slot];
  b->next_slot = (b->next_slot + 1) % kStagingSlots;
  MELT_CUDA(cudaEventSynchronize(s.done));  // the previous user of this slot is finished
  s.key_batch = -1;
  const size_t n = std::max<size_t>(b->plan.size(), 1);
  if (n > s.cap) {
    cudaFreeHost(s.host);
    cudaFree(s.dev);
    s.host = nullptr; s.dev = nullptr; s.cap = 0;
    const size_t cap = std::max<size_t>(n, 1024);
    MELT_CUDA(melt::host_alloc_pinned(&s.host, cap * sizeof(TileDesc)));
    MELT_CUDA(melt::dev_alloc(&s.dev, cap * sizeof(TileDesc)));
    s.cap = cap;
  }
  std::memcpy(s.host, b->plan.data(), b->plan.size() * sizeof(TileDesc));
  MELT_CUDA(cudaMemcpyAsync(s.dev, s.host, b->plan.size() * sizeof(TileDesc),
                            cudaMemcpyHostToDevice, stream));
  s.n = b->plan.size();
  s.rows = b->plan_rows;
  s.key_batch = batch;
  s.key_lengths.assign(lengths, lengths + batch);
  if (offsets) s.key_offsets.assign(offsets, offsets + batch); else s.key_offsets.clear();
  *slot_out = &s;
  return MELT_OK;
}

melt_status forward_impl(melt_basis* b, const float* wave, const int64_t* offsets,
                         const int64_t* lengths, int batch, float* out, void* stream_v,
                         int mode, unsigned flags = 0) {
  if (!b || batch < 0 || (batch > 0 && (!lengths || !wave || !out))) return MELT_ERR_ARG;
  if (((uintptr_t)wave & 15) || ((uintptr_t)out & 15)) return MELT_ERR_ARG;
  if (batch == 0) return MELT_OK;
  cudaStream_t stream = (cudaStream_t)stream_v;
  Staging* slot = cached_plan(b, offsets, lengths, batch);
  if (!slot) {
    melt_status st = plan_tiles(b, offsets, lengths, batch);
    if (st != MELT_OK) return st;
    if (b->plan.empty()) return MELT_OK;
    st = stage_plan(b, offsets, lengths, batch, stream, &slot);
    if (st != MELT_OK) return st;
  }
  if (slot->n == 0) return MELT_OK;
  const int n_tiles = (int)slot->n;
  cudaError_t e;
  bool fused = false;  // the kernel applied the correction itself
  if (b->precision == MELT_FP32 || mode == 1) {
    SimtParams p;
    p.wave = wave; p.tiles = slot->dev; p.n_tiles = n_tiles;
    p.w32 = b->d_w32; p.dct = b->d_dct; p.out = out;
    p.n_fft = b->n_fft; p.hop = b->hop; p.n_mels = b->n_mels; p.mp = b->mp;
    p.n_mfcc = b->n_mfcc; p.n_out = b->n_mfcc ? b->n_mfcc : b->n_mels;
    p.eps = (float)b->eps; p.mode = mode;
    e = launch_simt(p, b->mj, b->sm_count, stream);
  } else {
    TcLaunch L;
    L.wave = wave; L.tiles = slot->dev; L.n_tiles = n_tiles; L.out = out;
    L.dct = b->d_dct; L.n_mfcc = b->n_mfcc; L.eps = (float)b->eps; L.err = b->d_err;
    L.sm_count = b->sm_count;
    L.mlp = mode == 0 ? b->correction : nullptr;
    L.early_inputs = (flags & MELT_FWD_INPUT_READY) != 0;
    L.fused = &fused;
    L.fb = b->d_fb;
    L.stft_bands = b->stft_bands;
    e = tc_launch(&b->tc, L, stream);
  }
  if (e != cudaSuccess) return cuda_status(e);
  if (b->correction && mode == 0 && !fused) {
    const melt_status st = mlp_apply(b->correction, out, out, slot->rows, stream);
    if (st != MELT_OK) return st;
  }
  MELT_CUDA(cudaEventRecord(slot->done, stream));
  return MELT_OK;
}

}  // namespace

namespace melt {

static std::atomic<long long> g_alloc_calls{0};  // allocations made by the library

cudaError_t dev_alloc_bytes(void** p, size_t bytes) {
  g_alloc_calls.fetch_add(1, std::memory_order_relaxed);
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc_pinned_bytes(void** p, size_t bytes) {
  g_alloc_calls.fetch_add(1, std::memory_order_relaxed);
  return cudaMallocHost(p, bytes);
}

int64_t basis_frames(const melt_basis* b, int64_t len) { return frames_of(b, len); }

long long plan_clip_tiles(const melt_basis* b, int64_t off, int64_t len, int64_t row, int clip,
                          int group, TileDesc* dst, long long cap) {
  const int64_t T = frames_of(b, len);
  long long n = 0;
  for (int64_t t0 = 0; t0 < T; t0 += kTileFrames) {
    if (n >= cap) return -2;
    TileDesc& d = dst[n++];
    d.in_off = off + t0 * b->hop;
    d.out_row = row + t0;
    d.n_frames = (int32_t)std::min<int64_t>(kTileFrames, T - t0);
    d.n_samples = (int32_t)std::min<int64_t>(len - t0 * b->hop, INT32_MAX);
    d.group = group;
    d.clip = clip;
  }
  return n;
}

long long plan_tiles_into(const melt_basis* b, const int64_t* offsets, const int64_t* lengths,
                          int batch, TileDesc* dst, long long cap) {
  long long n = 0;
  int64_t row = 0, off = 0;
  for (int c = 0; c < batch; ++c) {
    const int64_t L = lengths[c];
    if (L < 0) return -1;
    const int64_t o = offsets ? offsets[c] : off;
    if (o < 0 || (o & 3)) return -1;
    off += (L + 3) & ~int64_t(3);
    const long long k = plan_clip_tiles(b, o, L, row, c, 0, dst + n, cap - n);
    if (k < 0) return k;
    n += k;
    row += frames_of(b, L);
  }
  if (b->precision == MELT_FP32) order_longest_first(dst, n);
  return n;
}

melt_status launch_forward_tiles(melt_basis* b, const float* wave, const TileDesc* d_tiles,
                                 int n_tiles, float* out, int64_t rows, cudaStream_t stream) {
  cudaError_t e;
  bool fused = false;
  if (b->precision == MELT_FP32) {
    SimtParams p;
    p.wave = wave; p.tiles = d_tiles; p.n_tiles = n_tiles;
    p.w32 = b->d_w32; p.dct = b->d_dct; p.out = out;
    p.n_fft = b->n_fft; p.hop = b->hop; p.n_mels = b->n_mels; p.mp = b->mp;
    p.n_mfcc = b->n_mfcc; p.n_out = b->n_mfcc ? b->n_mfcc : b->n_mels;
    p.eps = (float)b->eps; p.mode = 0;
    e = launch_simt(p, b->mj, b->sm_count, stream);
  } else {
    TcLaunch L;
    L.wave = wave; L.tiles = d_tiles; L.n_tiles = n_tiles; L.out = out;
    L.dct = b->d_dct; L.n_mfcc = b->n_mfcc; L.eps = (float)b->eps; L.err = b->d_err;
    L.sm_count = b->sm_count;
    L.mlp = b->correction;
    L.fused = &fused;
    L.fb = b->d_fb;
    L.stft_bands = b->stft_bands;
    e = tc_launch(&b->tc, L, stream);
  }
  if (e != cudaSuccess) return cuda_status(e);
  if (b->correction && !fused) return mlp_apply(b->correction, out, out, rows, stream);
  return MELT_OK;
}

melt_status launch_forward_tiles_pair2(melt_basis* b0, const TileDesc* t0, int n0, melt_basis* b1,
                                       const TileDesc* t1, int n1, const float* wave, float* out, double frac0,
                                       cudaStream_t stream, bool* launched) {
  *launched = false;
  if (b0->precision == MELT_FP32 || b1->precision == MELT_FP32 || b0->correction || b1->correction)
    return MELT_OK;
  TcLaunch L[2];
  melt_basis* bs[2] = {b0, b1};
  const TileDesc* ts[2] = {t0, t1};
  const int ns[2] = {n0, n1};
  for (int k = 0; k < 2; ++k) {
    L[k].wave = wave; L[k].tiles = ts[k]; L[k].n_tiles = ns[k]; L[k].out = out;
    L[k].dct = bs[k]->d_dct; L[k].n_mfcc = bs[k]->n_mfcc; L[k].eps = (float)bs[k]->eps; L[k].err = bs[k]->d_err;
    L[k].sm_count = bs[k]->sm_count;
    L[k].fb = bs[k]->d_fb;
    L[k].stft_bands = bs[k]->stft_bands;
  }
  // clusters in proportion to each basis's tiles x n_fft (the MMA work of a tile)
  const double w0 = (double)n0 * b0->n_fft, w1 = (double)n1 * b1->n_fft;
  const cudaError_t e =
      tc_launch_pair_group(&b0->tc, L[0], &b1->tc, L[1], frac0 > 0.0 ? frac0 : w0 / (w0 + w1), stream, launched);
  return e == cudaSuccess ? MELT_OK : cuda_status(e);
}

int basis_device(const melt_basis* b) { return b->device; }

const melt_mlp* basis_correction(const melt_basis* b) { return b->correction; }

int basis_plan_candidates(const melt_basis* b, melt_plan* out, int cap) {
  if (b->precision == MELT_FP32) return 0;
  return tc_candidates(&b->tc, out, cap);
}

bool device_token(int device, char* buf, size_t n) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return false;
  std::snprintf(buf, n, "%s", prop.name);
  for (char* ch = buf; *ch; ++ch)
    if (*ch == ' ' || *ch == '\t' || *ch == ':') *ch = '_';
  return true;
}

void basis_plan_key(const melt_basis* b, char* buf, size_t n) {
  std::snprintf(buf, n, "%d %d %d %d %d %d %d", b->n_fft, b->hop, b->n_mels, b->precision, b->n_mfcc,
                b->correction ? mlp_hidden(b->correction) : 0, b->stft_bands);
}

int tile_class(long long tiles) {
  int c = 0;
  while (c < 62 && (1ll << (c + 1)) <= tiles) ++c;
  return c;
}

int format_plan(const melt_plan& p, char* buf, size_t n) {
  return std::snprintf(buf, n, "%d %d %d %d %d %d %d", p.basis_resident, p.a_buffers, p.prefetch_tiles,
                       p.basis_slots, p.ksteps_per_slot, p.cta_pair, p.schedule);
}

bool parse_plan(const char* s, melt_plan* p, int* used) {
  int k = 0;
  if (std::sscanf(s, " %d %d %d %d %d %d %d%n", &p->basis_resident, &p->a_buffers, &p->prefetch_tiles,
                  &p->basis_slots, &p->ksteps_per_slot, &p->cta_pair, &p->schedule, &k) != 7)
    return false;
  *used = k;
  return true;
}

bool cache_lookup(const char* path, const char* key, char* rest, size_t n) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[2048];
  const size_t kl = std::strlen(key);
  bool found = false;
  while (!found && std::fgets(line, sizeof(line), f)) {
    if (std::strncmp(line, key, kl) != 0 || std::strncmp(line + kl, " : ", 3) != 0) continue;
    std::snprintf(rest, n, "%s", line + kl + 3);
    found = true;
  }
  std::fclose(f);
  return found;
}

void cache_append(const char* path, const char* key, const char* rest) {
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  char line[2048];
  const int k = std::snprintf(line, sizeof(line), "%s : %s\n", key, rest);
  if (k > 0 && (size_t)k < sizeof(line)) std::fwrite(line, 1, (size_t)k, f);  // one write: appends stay whole lines
  std::fclose(f);
}

HostPipe*& basis_host_pipe(melt_basis* b) { return b->host_pipe; }

}  // namespace melt

namespace {

// HTK Mel scale (Eq. 1) and the Slaney scale (linear, 200/3 Hz per mel, below
// 1 kHz; logarithmic, ln(6.4)/27 per mel, above), and their inverses.
double slaney_mel(double f) {
  const double logstep = std::log(6.4) / 27.0;
  return f >= 1000.0 ? 15.0 + std::log(f / 1000.0) / logstep : f / (200.0 / 3.0);
}
double slaney_hz(double m) {
  const double logstep = std::log(6.4) / 27.0;
  return m >= 15.0 ? 1000.0 * std::exp(logstep * (m - 15.0)) : m * (200.0 / 3.0);
}

// Per DFT bin k (frequency k sr / N): the bin lies between edges e[i] and
// e[i+1] of the n_bands + 2 filterbank edges, in the falling side of band i-1
// (weight (e[i+1] - f) / (e[i+1] - e[i])) and the rising side of band i
// (weight (f - e[i]) / (e[i+1] - e[i])); bands past either end get weight 0.
// Entry {w(band i-1), w(band i), i-1 as int bits, 0}; a bin outside [e[0],
// e[n_bands+1]] gets band index -2 (no band).
std::vector<float4> stft_filterbank(double sr, int n_fft, int n_bands, double fmin, double fmax, int scale) {
  std::vector<double> e(n_bands + 2);
  const double lo = scale ? slaney_mel(fmin) : hz_to_mel(fmin), hi = scale ? slaney_mel(fmax) : hz_to_mel(fmax);
  for (int i = 0; i < n_bands + 2; ++i) {
    const double mu = lo + (hi - lo) * i / (n_bands + 1);
    e[i] = scale ? slaney_hz(mu) : mel_to_hz(mu);
  }
  const int K = n_fft / 2 + 1;
  std::vector<float4> fb(K);
  int prev = -1;  // band c of the epilogue's walk before bin k (the last in-range bin's b0)
  for (int k = 0; k < K; ++k) {
    const double f = (double)k * sr / n_fft;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    int b0 = -2;
    if (f >= e[0] && f <= e[n_bands + 1]) {
      int i = 0;
      while (i < n_bands && f >= e[i + 1]) ++i;  // e[i] <= f < e[i+1] (or the last interval)
      const double span = e[i + 1] - e[i];
      double wfall = span > 0 ? (e[i + 1] - f) / span : 0.0, wrise = span > 0 ? (f - e[i]) / span : 0.0;
      wfall = std::max(0.0, wfall);
      wrise = std::max(0.0, wrise);
      if (scale) {  // unit area: band j scaled by 2 / (e[j+2] - e[j])
        if (i >= 1) wfall *= 2.0 / (e[i + 1] - e[i - 1]);
        if (i < n_bands) wrise *= 2.0 / (e[i + 2] - e[i]);
      }
      v.x = i >= 1 ? (float)wfall : 0.f;
      v.y = i < n_bands ? (float)wrise : 0.f;
      b0 = i - 1;
    }
    // bands completed before this bin's power is added (the walk moves from
    // band prev to b0); bins outside every triangle add zero and complete none
    const int nf = b0 >= -1 ? b0 - prev : 0;
    if (b0 >= -1) prev = b0;
    std::memcpy(&v.z, &b0, sizeof(float));  // the band index's int bits
    std::memcpy(&v.w, &nf, sizeof(float));
    fb[k] = v;
  }
  return fb;
}

}  // namespace

extern "C" {

melt_status melt_basis_create(double sr, int n_fft, int hop, int n_mels, double fmin,
                              double fmax, int window, melt_basis** out) {
  return melt_basis_create_ex(sr, n_fft, hop, n_mels, fmin, fmax, window, MELT_FP32, 0, 1e-10,
                              out);
}

melt_status melt_basis_create_ex(double sr, int n_fft, int hop, int n_mels, double fmin,
                                 double fmax, int window, int precision, int n_mfcc,
                                 double eps, melt_basis** out) {
  if (!out) return MELT_ERR_ARG;
  *out = nullptr;
  if (n_mels < 1 || n_mels > kMaxFreqs || !(sr > 0) || !(fmin >= 0) || !(fmax > fmin) ||
      !(fmax <= sr / 2))
    return MELT_ERR_ARG;
  // M interior points of M+2 points uniform on the Mel scale (Sec. III-A)
  std::vector<double> f(n_mels);
  const double lo = hz_to_mel(fmin), hi = hz_to_mel(fmax);
  for (int m = 0; m < n_mels; ++m) f[m] = mel_to_hz(lo + (hi - lo) * (m + 1) / (n_mels + 1));
  melt_status st = create_common(sr, n_fft, hop, f.data(), n_mels, fmin, fmax, window, precision,
                                 n_mfcc, eps, out);
  return st;
}

melt_status melt_basis_create_freqs(double sr, int n_fft, int hop, const double* freqs,
                                    int n_freqs, int window, int precision, int n_mfcc,
                                    double eps, melt_basis** out) {
  if (!freqs) return MELT_ERR_ARG;
  return create_common(sr, n_fft, hop, freqs, n_freqs, 0.0, sr / 2, window, precision, n_mfcc,
                       eps, out);
}

melt_status melt_stft_create(double sr, int n_fft, int hop, int n_mels, double fmin, double fmax, int window,
                             int precision, int scale, double eps, melt_basis** out) {
  if (!out) return MELT_ERR_ARG;
  *out = nullptr;
  if (n_mels < 1 || n_mels > 512 || !(sr > 0) || !(fmin >= 0) || !(fmax > fmin) || !(fmax <= sr / 2) ||
      (scale != 0 && scale != 1) || n_fft < 16 || n_fft > 4096)
    return MELT_ERR_ARG;
  if ((precision != MELT_BF16 && precision != MELT_BF16X3) || n_fft / 2 + 1 > kMaxFreqs) return MELT_ERR_UNSUPPORTED;
  const int K = n_fft / 2 + 1;
  std::vector<double> f(K);
  for (int k = 0; k < K; ++k) f[k] = (double)k * sr / n_fft;
  // the projection needs more than 128 frequencies: the blocked BF16 path
  melt_basis* b = nullptr;
  melt_status st = create_common(sr, n_fft, hop, f.data(), K, 0.0, sr / 2, window, precision, 0, eps, &b, n_mels);
  if (st != MELT_OK) return st;
  b->fmin = fmin;
  b->fmax = fmax;
  const std::vector<float4> fb = stft_filterbank(sr, n_fft, n_mels, fmin, fmax, scale);
  cudaError_t e = melt::dev_alloc(&b->d_fb, fb.size() * sizeof(float4));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_fb, fb.data(), fb.size() * sizeof(float4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_basis(b);
    return cuda_status(e);
  }
  b->stft_bands = n_mels;
  *out = b;
  return MELT_OK;
}

int64_t melt_num_frames(const melt_basis* basis, int64_t length) {
  if (!basis) return 0;
  return frames_of(basis, length);
}

int melt_num_outputs(const melt_basis* basis) {
  if (!basis) return 0;
  if (basis->stft_bands) return basis->stft_bands;
  return basis->n_mfcc ? basis->n_mfcc : basis->n_mels;
}

melt_status melt_basis_info(const melt_basis* b, int* ints, double* doubles) {
  if (!b) return MELT_ERR_ARG;
  if (ints) {
    ints[0] = b->n_fft; ints[1] = b->hop; ints[2] = b->n_mels;
    ints[3] = b->n_mfcc; ints[4] = b->precision; ints[5] = b->window;
  }
  if (doubles) {
    doubles[0] = b->sr; doubles[1] = b->fmin; doubles[2] = b->fmax; doubles[3] = b->eps;
  }
  return MELT_OK;
}

melt_status melt_basis_get_fp64(const melt_basis* b, double* freqs, double* w) {
  if (!b) return MELT_ERR_ARG;
  if (freqs) std::memcpy(freqs, b->freqs.data(), b->freqs.size() * sizeof(double));
  if (w) std::memcpy(w, b->w64.data(), b->w64.size() * sizeof(double));
  return MELT_OK;
}

melt_status melt_forward(melt_basis* basis, const float* wave, const int64_t* offsets,
                         const int64_t* lengths, int batch, float* out, void* stream) {
  return forward_impl(basis, wave, offsets, lengths, batch, out, stream, 0);
}

melt_status melt_forward_ex(melt_basis* basis, const float* wave, const int64_t* offsets,
                            const int64_t* lengths, int batch, float* out, void* stream, unsigned flags) {
  if (flags & ~(unsigned)MELT_FWD_INPUT_READY) return MELT_ERR_ARG;
  return forward_impl(basis, wave, offsets, lengths, batch, out, stream, 0, flags);
}

melt_status melt_forward_components(melt_basis* basis, const float* wave,
                                    const int64_t* offsets, const int64_t* lengths, int batch,
                                    float* out, void* stream) {
  if (basis && basis->precision != MELT_FP32) return MELT_ERR_UNSUPPORTED;
  return forward_impl(basis, wave, offsets, lengths, batch, out, stream, 1);
}

melt_status melt_plan_get(const melt_basis* b, melt_plan* plan) {
  if (!b || !plan) return MELT_ERR_ARG;
  if (b->precision == MELT_FP32) return MELT_ERR_UNSUPPORTED;
  return tc_current_plan(&b->tc, plan) ? MELT_OK : MELT_ERR_UNSUPPORTED;
}

melt_status melt_plan_set(melt_basis* b, const melt_plan* plan) {
  if (!b) return MELT_ERR_ARG;
  if (b->precision == MELT_FP32) return MELT_ERR_UNSUPPORTED;
  if (!plan) {
    b->tc.forced = false;
    return MELT_OK;
  }
  if (!tc_plan_fits(&b->tc, *plan)) return MELT_ERR_UNSUPPORTED;
  b->tc.plan = *plan;
  b->tc.forced = true;
  return MELT_OK;
}

melt_status melt_autotune(melt_basis* b, const float* wave, const int64_t* offsets,
                          const int64_t* lengths, int batch, float* out, void* stream_v, int reps,
                          melt_plan* best) {
  if (!b || reps < 1) return MELT_ERR_ARG;
  if (b->precision == MELT_FP32) return MELT_ERR_UNSUPPORTED;
  cudaStream_t stream = (cudaStream_t)stream_v;
  melt_plan cands[64];
  const int n = tc_candidates(&b->tc, cands, 64);
  if (n < 1) return MELT_ERR_UNSUPPORTED;
  cudaEvent_t e0, e1;
  MELT_CUDA(cudaEventCreate(&e0));
  MELT_CUDA(cudaEventCreate(&e1));
  const bool had = b->tc.forced;
  const melt_plan prev = b->tc.plan;
  float best_ms = 1e30f;
  int best_i = -1;
  melt_status st = MELT_OK;
  for (int i = 0; i < n && st == MELT_OK; ++i) {
    b->tc.plan = cands[i];
    b->tc.forced = true;
    st = melt_forward(b, wave, offsets, lengths, batch, out, stream);  // warm-up
    if (st != MELT_OK) break;
    cudaEventRecord(e0, stream);
    for (int r = 0; r < reps && st == MELT_OK; ++r)
      st = melt_forward(b, wave, offsets, lengths, batch, out, stream);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = MELT_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (st == MELT_OK && ms < best_ms) {
      best_ms = ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == MELT_OK) st = melt_sync(b, stream);
  if (st != MELT_OK || best_i < 0) {
    b->tc.forced = had;
    b->tc.plan = prev;
    return st != MELT_OK ? st : MELT_ERR_UNSUPPORTED;
  }
  b->tc.plan = cands[best_i];
  b->tc.forced = true;
  if (best) *best = cands[best_i];
  return MELT_OK;
}

melt_status melt_autotune_file(melt_basis* b, const float* wave, const int64_t* offsets,
                               const int64_t* lengths, int batch, float* out, void* stream_v, int reps,
                               const char* path, melt_plan* best, int* hit) {
  if (hit) *hit = 0;
  if (!b || !path || reps < 1 || batch < 0 || (batch > 0 && !lengths)) return MELT_ERR_ARG;
  if (b->precision == MELT_FP32) return MELT_ERR_UNSUPPORTED;
  char gpu[256], cfg[160], key[512], rest[256];
  if (!device_token(b->device, gpu, sizeof(gpu))) return MELT_ERR_CUDA;
  basis_plan_key(b, cfg, sizeof(cfg));
  long long tiles = 0;
  for (int c = 0; c < batch; ++c) tiles += (frames_of(b, lengths[c]) + kTileFrames - 1) / kTileFrames;
  std::snprintf(key, sizeof(key), "melt-plan-v1 %s %s %d", gpu, cfg, tile_class(tiles));
  melt_plan pl;
  int used = 0;
  if (cache_lookup(path, key, rest, sizeof(rest)) && parse_plan(rest, &pl, &used) && tc_plan_fits(&b->tc, pl)) {
    b->tc.plan = pl;
    b->tc.forced = true;
    if (best) *best = pl;
    if (hit) *hit = 1;
    return MELT_OK;
  }
  const melt_status st = melt_autotune(b, wave, offsets, lengths, batch, out, stream_v, reps, &pl);
  if (st != MELT_OK) return st;
  if (best) *best = pl;
  format_plan(pl, rest, sizeof(rest));
  cache_append(path, key, rest);
  return MELT_OK;
}

melt_status melt_basis_set_correction(melt_basis* b, const melt_mlp* mlp) {
  if (!b) return MELT_ERR_ARG;
  if (mlp) {
    if (b->n_mfcc != 0 || b->stft_bands) return MELT_ERR_UNSUPPORTED;  // the correction acts on MelT log-Mel bands
    if (mlp_inputs(mlp) != b->n_mels || mlp_device(mlp) != b->device) return MELT_ERR_ARG;
  }
  // the BF16 image for the fused epilogue is allocated here, so that forward
  // calls (the allocation-free one included) allocate nothing
  if (mlp && b->precision == MELT_BF16 && b->tc.d_b2 && mlp_fused_shape_ok(b->n_mels, mlp_hidden(mlp))) {
    const long long half = mlp_fused_half_bytes(b->n_mels, mlp_hidden(mlp));
    if (!b->tc.d_mlp_img || b->tc.mlp_half != half) {
      MELT_CUDA(cudaDeviceSynchronize());  // no kernel may still read the old image
      cudaFree(b->tc.d_mlp_img);
      b->tc.d_mlp_img = nullptr;
      b->tc.mlp_hd = 0;
      MELT_CUDA(melt::dev_alloc(&b->tc.d_mlp_img, 2 * half));
      b->tc.mlp_half = half;
    }
    b->tc.mlp_hd = mlp_hidden(mlp);
  } else {
    b->tc.mlp_hd = 0;
  }
  b->tc.pair_clusters = -1;  // the pair kernel's shared memory may have changed
  b->correction = mlp;
  return MELT_OK;
}

namespace {

// One thread waits on an mbarrier that nothing arrives on.  The wait is the
// library's bounded one: after its limit it latches the timeout bit in the
// basis's error word, raises the (local) abort flag and returns, and the
// kernel ends; nothing faults and the context stays usable.
__global__ void diag_wait_timeout_kernel(int* err) {
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    const uint32_t a = melt::ptx::smem_u32(&bar);
    melt::ptx::mbar_init(a, 1);
    melt::ptx::fence_mbar_init();
    melt::ptx::mbar_wait(a, 0, &abort_flag, err, kErrTimeout);
  }
}

}  // namespace

melt_status melt_diag_wait_timeout(melt_basis* b, void* stream) {
  if (!b) return MELT_ERR_ARG;
  int dev = -1;
  MELT_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) return MELT_ERR_ARG;
  diag_wait_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(b->d_err);
  MELT_CUDA(cudaGetLastError());
  return MELT_OK;
}

long long melt_diag_alloc_count(void) { return melt::g_alloc_calls.load(std::memory_order_relaxed); }

melt_status melt_sync(melt_basis* b, void* stream) {
  if (!b) return MELT_ERR_ARG;
  MELT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int err = 0;
  MELT_CUDA(cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    MELT_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
    return MELT_ERR_TIMEOUT;
  }
  return MELT_OK;
}

melt_status melt_destroy(melt_basis* b) {
  if (!b) return MELT_OK;
  cudaDeviceSynchronize();
  free_basis(b);
  return MELT_OK;
}

const char* melt_status_string(int s) {
  switch (s) {
    case MELT_OK: return "ok";
    case MELT_ERR_ARG: return "invalid argument";
    case MELT_ERR_CUDA: return "CUDA runtime error";
    case MELT_ERR_OOM: return "out of memory";
    case MELT_ERR_UNSUPPORTED: return "unsupported configuration";
    case MELT_ERR_TIMEOUT: return "kernel wait timed out";
    case MELT_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    default: return "unknown status";
  }
}

const char* melt_version(void) { return "melt 0.1 sm_103a"; }

}  // extern "C"
