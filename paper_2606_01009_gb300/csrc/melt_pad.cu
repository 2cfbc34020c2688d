// melt_pad_reflect: centred framing by reflection padding.
//
// The paper frames a clip from its first sample with no padding (Sec. III-A,
// the matrix X of Eq. 6).  Speech frontends built on a centred STFT (Whisper's,
// or torch.stft with center=True) instead pad each clip by N/2 samples of
// reflection at both ends, so that frame t is centred on sample t H and a clip
// of L samples gives floor(L / H) + 1 frames.  This call builds that padded
// batch; melt_forward then runs unchanged on it.
//
// Reflection without repeating the edge sample: for a clip x[0 .. L), the
// padded clip y[0 .. L + 2p) is y[i] = x[r(i - p)] with r(j) = -j for j < 0,
// r(j) = 2 (L - 1) - j for j >= L, and r(j) = j otherwise; it needs p < L.
//
// The clip descriptors travel by value in the kernel's parameters (up to
// kPadChunk clips per launch), so the call allocates nothing and calls on
// different streams share no state.
#include <cuda_runtime.h>

#include <algorithm>

#include "melt_internal.h"

namespace {

constexpr int kPadChunk = 1000;  // clips per launch: 24 KB of descriptors in the parameters

struct PadClip {
  int64_t src;  // float index of the clip in the input
  int64_t dst;  // float index of the padded clip in the output
  int64_t len;  // samples of the clip (> pad)
};

struct PadBatch {
  const float* wave;
  float* out;
  int64_t pad;
  int n;
  PadClip c[kPadChunk];
};

// Block row y pads clip y of the chunk; the x blocks stride over its padded samples.
__global__ void __launch_bounds__(256) pad_reflect_kernel(const __grid_constant__ PadBatch b) {
  const PadClip cl = b.c[blockIdx.y];
  const int64_t total = cl.len + 2 * b.pad;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
    int64_t j = i - b.pad;
    j = j < 0 ? -j : (j >= cl.len ? 2 * (cl.len - 1) - j : j);
    b.out[cl.dst + i] = b.wave[cl.src + j];
  }
}

}  // namespace

extern "C" melt_status melt_pad_reflect(const float* wave, const int64_t* offsets, const int64_t* lengths,
                                        int batch, int pad, float* out, const int64_t* out_offsets,
                                        void* stream_v) {
  if (batch < 0 || pad < 0 || (batch > 0 && (!lengths || !wave || !out))) return MELT_ERR_ARG;
  if (batch == 0) return MELT_OK;
  // validate everything before the first launch
  int64_t src = 0, dst = 0, max_total = 0;
  for (int c = 0; c < batch; ++c) {
    const int64_t L = lengths[c];
    if (L <= pad) return MELT_ERR_ARG;  // reflection needs pad + 1 samples
    const int64_t s = offsets ? offsets[c] : src;
    const int64_t d = out_offsets ? out_offsets[c] : dst;
    if (s < 0 || d < 0) return MELT_ERR_ARG;
    src += (L + 3) & ~int64_t(3);
    dst += (L + 2 * pad + 3) & ~int64_t(3);
    max_total = std::max(max_total, L + 2 * pad);
  }
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  PadBatch b;
  b.wave = wave;
  b.out = out;
  b.pad = pad;
  src = 0;
  dst = 0;
  const unsigned gx = (unsigned)std::min<int64_t>((max_total + 255) / 256, 64);
  for (int c0 = 0; c0 < batch; c0 += kPadChunk) {
    b.n = std::min(kPadChunk, batch - c0);
    for (int i = 0; i < b.n; ++i) {
      const int c = c0 + i;
      const int64_t L = lengths[c];
      b.c[i].src = offsets ? offsets[c] : src;
      b.c[i].dst = out_offsets ? out_offsets[c] : dst;
      b.c[i].len = L;
      src += (L + 3) & ~int64_t(3);
      dst += (L + 2 * pad + 3) & ~int64_t(3);
    }
    pad_reflect_kernel<<<dim3(gx, (unsigned)b.n), 256, 0, stream>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MELT_ERR_OOM : MELT_ERR_CUDA;
  }
  return MELT_OK;
}
