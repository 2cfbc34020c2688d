// Tensor-core (tcgen05 / TMEM) MelT kernels: BF16, split-BF16 and FP8 forms.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "melt_internal.h"

namespace melt {

struct TcConfig {
  int n_fft, hop, n_mels, precision, n_mfcc;
  int stft_bands;  // > 0: the fused STFT + Mel comparator's epilogue (n_mels = DFT bins)
};

// Device-resident operand images of one basis for the tensor-core kernels.
struct TcBasis {
  int precision = 0;
  int n_fft = 0, hop = 0, n_mels = 0;
  int J = 0;            // polyphase slices ceil(N / H)
  int ksteps = 0;       // MMA K-steps over all slices
  int kstep_k = 0;      // K per MMA instruction (16 for BF16, 32 for FP8)
  int n_cols = 0;       // UMMA N = 2M rounded up to a multiple of 16
  size_t kstep_bytes = 0;  // bytes of one K-step block of the B operand
  void* d_b = nullptr;     // B operand blocks, one per K-step (BF16x3: hi and lo parts)
  void* d_b2 = nullptr;    // CTA-pair image: W_r rows' blocks, then W_i rows' blocks (BF16x3: hi, lo per block)
  int n_mfcc = 0;
  int stft_bands = 0;      // fused STFT + Mel comparator: bands per frame (its table sits in shared memory)
  int pair_clusters = -1;  // co-resident 2-CTA clusters of the pair kernel (-1: not queried)
  int pair_smem = 0;       // shared memory size that count was queried for
  // correction MLP fused in the CTA-pair kernel's epilogue (0 hidden units: none)
  int mlp_hd = 0;
  void* d_mlp_img = nullptr;  // BF16 weight image, two halves of mlp_half bytes
  long long mlp_half = 0;
  // dynamic pair schedule: kSchedWords counter/done word pairs; launch i uses pair i % kSchedWords
  unsigned long long* d_sched = nullptr;
  unsigned sched_next = 0;
  bool forced = false;         // plan below was set explicitly (melt_plan_set / autotune)
  melt_plan plan = {};         // forced layout
};

// Candidate layouts that fit shared memory, best-guess first.
int tc_candidates(const TcBasis* tb, melt_plan* out, int cap);
// Layout the launch will use (forced one if set, else the first candidate).
bool tc_current_plan(const TcBasis* tb, melt_plan* out);
// true if the layout fits shared memory for this basis.
bool tc_plan_fits(const TcBasis* tb, const melt_plan& plan);

struct TcLaunch {
  const float* wave;
  const TileDesc* tiles;
  int n_tiles;
  float* out;
  const float* dct;   // [n_mfcc][n_mels] or nullptr
  int n_mfcc;
  float eps;
  int* err;
  int sm_count;
  bool pdl = true;    // launch with programmatic stream serialisation
  bool early_inputs = false;  // MELT_FWD_INPUT_READY: waveform readers need not wait (not with the dynamic schedule)
  const melt_mlp* mlp = nullptr;  // correction attached to the basis (fused when the layout allows)
  const float4* fb = nullptr;     // fused STFT + Mel comparator: per-bin filterbank entries (device)
  int stft_bands = 0;
  bool* fused = nullptr;          // out: true when the kernel applied `mlp` itself
};

melt_status tc_build(TcBasis* tb, const TcConfig& c, const double* w64);
// Two BF16 log-Mel bases in one persistent CTA-pair launch (the grouped
// call): a fraction frac0 of the clusters works through L0's tiles, the rest
// through L1's.  Each basis runs its own plan when that is a CTA-pair plan;
// a basis without a forced plan whose default is single-CTA runs the first
// streamed-half-basis pair layout that fits.  *launched is false (and
// nothing is enqueued) when a basis cannot run that way.
cudaError_t tc_launch_pair_group(const TcBasis* tb0, const TcLaunch& L0, const TcBasis* tb1, const TcLaunch& L1,
                                 double frac0, cudaStream_t stream, bool* launched);
int tc_max_mfcc();  // largest n_mfcc the tensor-core epilogue supports
void tc_free(TcBasis* tb);
cudaError_t tc_launch(const TcBasis* tb, const TcLaunch& L, cudaStream_t stream);

}  // namespace melt
