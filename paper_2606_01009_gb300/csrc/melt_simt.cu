// Plain FP32 MelT on CUDA cores (FFMA, FP32 accumulate).
//
// Computes the projection of Sec. III-A, Eq. 6 ([R | I] = X [W_r; W_i]^T)
// with implicit framing: frame f of a tile is read straight from the packed
// waveform at in_off + f*H, never materialised in global memory.  The power
// (Eq. 7), log (Eq. 8) and optional DCT-II (Eq. 9) are fused in the epilogue.
//
// CTA tile: 128 frames x all 2M basis rows; 256 threads as 16 (frame groups
// of 8) x 16 (mel lanes); thread (ty, tx) owns frames 8ty..8ty+7 and mels
// tx + 16j, j < MJ, for both R and I (16*MJ FP32 accumulators).
// K loop in chunks of 32 samples: the chunk of the frame matrix is
// transposed into shared memory (Xs[k][f]) by asynchronous copies with
// coalesced reads, the basis chunk (row-major [k][2*mp], R/I interleaved) is
// copied beside it; the next chunk's copies are in flight while the current
// one is computed.
#include <algorithm>

#include "melt_internal.h"

namespace melt {

namespace {

constexpr int kF = kTileFrames;  // 128
constexpr int kKC = 32;          // samples per K chunk
constexpr int kXPad = 4;         // Xs row padding (keeps float4 alignment)
constexpr int kThreads = 256;

// K chunks are double-buffered with asynchronous copies (cp.async): the
// copies of chunk c + 1 are issued into the other shared-memory buffer before
// chunk c is computed, so their latency hides behind the FFMAs and no
// registers hold them in flight.  That leaves room for two CTAs per SM (four
// warps per scheduler) where the accumulators allow (MJ <= 5).
template <int MJ>
struct SimtChunk {
  static constexpr int kXq = kF * kKC / kThreads;        // frame samples per thread (16)
  static constexpr int kWq = (kKC * 2 * 16 * MJ / 4 + kThreads - 1) / kThreads;  // basis float4s per thread
};

static __device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

static __device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until at most one group (the newest) of this thread is in flight.
static __device__ __forceinline__ void cp_async_wait_all_but_newest() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// Copies of K chunk [k0, k0 + kKC) of a tile: the frame chunk transposed into
// Xs[k][f] (4-byte copies; lanes take consecutive samples of a frame, so the
// global reads coalesce), the basis chunk into Ws[k][2 mp] (16-byte copies).
// Samples past the tile's frames or past N, and basis rows past N, are
// zero-filled (source size 0; the source address stays inside the buffer).
template <int MJ>
static __device__ __forceinline__ void simt_copy_chunk(const SimtParams& p, const TileDesc& td, int k0, int tid,
                                                       float* Xs, float* Ws) {
  const int N = p.n_fft, H = p.hop;
  constexpr int W2 = 32 * MJ, row4 = W2 / 4;  // 2 mp basis values per sample (mp = 16 MJ)
#pragma unroll
  for (int i = 0; i < SimtChunk<MJ>::kXq; ++i) {
    const int idx = tid + i * kThreads;
    const int k = idx % kKC, f = idx / kKC;
    const int n = k0 + k;
    const bool ok = f < td.n_frames && n < N;
    cp_async4(Xs + k * (kF + kXPad) + f, p.wave + (ok ? td.in_off + (int64_t)f * H + n : td.in_off), ok);
  }
#pragma unroll
  for (int i = 0; i < SimtChunk<MJ>::kWq; ++i) {
    const int idx = tid + i * kThreads;
    if (idx < kKC * row4) {
      const int k = idx / row4, c4 = idx - k * row4;
      const bool ok = k0 + k < N;
      cp_async16(Ws + k * W2 + 4 * c4, p.w32 + (size_t)(ok ? k0 + k : 0) * W2 + 4 * c4, ok);
    }
  }
}

template <int MJ>
__global__ void __launch_bounds__(kThreads, MJ <= 5 ? 2 : 1) melt_simt_kernel(SimtParams p) {
  extern __shared__ __align__(16) float smem[];
  constexpr int kXs = kKC * (kF + kXPad);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int N = p.n_fft, M = p.n_mels;
  // compile-time strides (mp = 16 MJ): every shared-memory offset of the
  // unrolled K loop is an immediate
  constexpr int W2 = 32 * MJ;
  constexpr int kWs = kKC * W2;
  // chunk buffer b: the frame chunk [kKC][kF + kXPad] at smem + b (kXs + kWs),
  // the basis chunk [kKC][2 mp] after it (addressed arithmetically: an array
  // of pointers indexed by b would live in local memory)
  constexpr int kBuf = kXs + kWs;

  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x) {
    const TileDesc td = p.tiles[tile];
    const bool busy = (tid >> 5) * 16 < td.n_frames;  // warp w owns frames 16 w .. 16 w + 15
    float acc[8][MJ][2];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < MJ; ++j) acc[i][j][0] = acc[i][j][1] = 0.f;

    __syncthreads();  // the previous tile's readers of both buffers (and the MFCC staging) are done
    simt_copy_chunk<MJ>(p, td, 0, tid, smem, smem + kXs);
    cp_async_commit();
    int b = 0;
    for (int k0 = 0; k0 < N; k0 += kKC, b ^= 1) {
      // the next chunk's copies go to the other buffer, whose last readers
      // passed the barrier at the end of the previous chunk
      if (k0 + kKC < N) simt_copy_chunk<MJ>(p, td, k0 + kKC, tid, smem + (b ^ 1) * kBuf, smem + (b ^ 1) * kBuf + kXs);
      cp_async_commit();  // (an empty group after the last chunk)
      cp_async_wait_all_but_newest();
      __syncthreads();    // every thread's copies of this chunk have landed
      const float* Xs = smem + b * kBuf;
      const float* Ws = Xs + kXs;
      // every chunk runs all kKC samples: past N both operands were
      // zero-filled, so those products add exact zeros (a compile-time
      // trip count lets every shared-memory offset be an immediate).  A warp
      // whose 16 frames all lie past the tile's end skips the FFMAs (it
      // still copies and meets the barriers), leaving its issue slots to
      // the SM's other warps.
#pragma unroll 8
      for (int k = 0; k < (busy ? kKC : 0); ++k) {
        const float4 xa = *reinterpret_cast<const float4*>(Xs + k * (kF + kXPad) + ty * 8);
        const float4 xb = *reinterpret_cast<const float4*>(Xs + k * (kF + kXPad) + ty * 8 + 4);
        const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
        for (int j = 0; j < MJ; ++j) {
          const float2 w = *reinterpret_cast<const float2*>(Ws + k * W2 + 2 * (tx + 16 * j));
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            acc[i][j][0] = fmaf(xv[i], w.x, acc[i][j][0]);
            acc[i][j][1] = fmaf(xv[i], w.y, acc[i][j][1]);
          }
        }
      }
      __syncthreads();  // this buffer's readers are done before it is refilled
    }

    // ---- epilogue: power (Eq. 7), log (Eq. 8), optional DCT-II (Eq. 9)
    if (p.mode == 1) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int f = ty * 8 + i;
        if (f >= td.n_frames) continue;
        float* orow = p.out + (size_t)(td.out_row + f) * (2 * M);
#pragma unroll
        for (int j = 0; j < MJ; ++j) {
          const int m = tx + 16 * j;
          if (m < M) { orow[m] = acc[i][j][0]; orow[M + m] = acc[i][j][1]; }
        }
      }
      continue;
    }
    if (p.n_mfcc == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int f = ty * 8 + i;
        if (f >= td.n_frames) continue;
        float* orow = p.out + (size_t)(td.out_row + f) * p.n_out;
#pragma unroll
        for (int j = 0; j < MJ; ++j) {
          const int m = tx + 16 * j;
          const float s = fmaf(acc[i][j][0], acc[i][j][0], acc[i][j][1] * acc[i][j][1]);
          if (m < M) orow[m] = __logf(s + p.eps);
        }
      }
      continue;
    }
    // MFCC: stage the tile's log-Mel rows in shared memory, then apply D.
    __syncthreads();  // every thread is done reading the chunk buffers
    float* L = smem;  // [kF][M]
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int f = ty * 8 + i;
#pragma unroll
      for (int j = 0; j < MJ; ++j) {
        const int m = tx + 16 * j;
        const float s = fmaf(acc[i][j][0], acc[i][j][0], acc[i][j][1] * acc[i][j][1]);
        if (m < M) L[f * M + m] = __logf(s + p.eps);
      }
    }
    __syncthreads();
    const int K = p.n_mfcc;
    for (int i = 0; i < 8; ++i) {
      const int f = ty * 8 + i;
      if (f >= td.n_frames) continue;
      for (int k = tx; k < K; k += 16) {
        const float* drow = p.dct + (size_t)k * M;
        float c = 0.f;
        for (int m = 0; m < M; ++m) c = fmaf(L[f * M + m], __ldg(drow + m), c);
        p.out[(size_t)(td.out_row + f) * K + k] = c;
      }
    }
  }
}

}  // namespace

int simt_smem_bytes(int mj, int n_mels, int n_mfcc) {
  const int mp = 16 * mj;
  int bytes = 2 * (kKC * (kF + kXPad) + kKC * 2 * mp) * (int)sizeof(float);  // two chunk buffers
  if (n_mfcc > 0) {
    const int l = kF * n_mels * (int)sizeof(float);
    if (l > bytes) bytes = l;
  }
  return bytes;
}

template <int MJ>
static cudaError_t launch_mj(const SimtParams& p, int sm_count, cudaStream_t stream) {
  const int smem = simt_smem_bytes(MJ, p.n_mels, p.n_mfcc);
  cudaError_t e = cudaFuncSetAttribute(melt_simt_kernel<MJ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;  // persistent: as many CTAs as can be resident at once
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, melt_simt_kernel<MJ>, kThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(p.n_tiles, std::max(1, per_sm) * sm_count);
  melt_simt_kernel<MJ><<<grid, kThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_simt(const SimtParams& p, int mj, int sm_count, cudaStream_t stream) {
  switch (mj) {
    case 1: return launch_mj<1>(p, sm_count, stream);
    case 2: return launch_mj<2>(p, sm_count, stream);
    case 3: return launch_mj<3>(p, sm_count, stream);
    case 4: return launch_mj<4>(p, sm_count, stream);
    case 5: return launch_mj<5>(p, sm_count, stream);
    case 6: return launch_mj<6>(p, sm_count, stream);
    case 7: return launch_mj<7>(p, sm_count, stream);
    case 8: return launch_mj<8>(p, sm_count, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace melt
