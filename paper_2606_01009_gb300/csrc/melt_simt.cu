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
// transposed into shared memory (Xs[k][f]) with coalesced loads, the basis
// chunk (row-major [k][2*mp], R/I interleaved) is copied beside it; the next
// chunk's loads are in flight while the current one is computed.
#include "melt_internal.h"

namespace melt {

namespace {

constexpr int kF = kTileFrames;  // 128
constexpr int kKC = 32;          // samples per K chunk
constexpr int kXPad = 4;         // Xs row padding (keeps float4 alignment)
constexpr int kThreads = 256;

// K chunks are double-buffered: the global loads of chunk c + 1 are issued
// into registers before chunk c is computed and stored into the other
// shared-memory buffer after it, so one barrier per chunk separates them and
// the loads' latency hides behind the FFMAs.
template <int MJ>
struct SimtChunk {
  static constexpr int kXq = kF * kKC / kThreads;        // frame samples per thread (16)
  static constexpr int kWq = (kKC * 2 * 16 * MJ / 4 + kThreads - 1) / kThreads;  // basis float4s per thread
  float x[kXq];
  float4 w[kWq];
};

template <int MJ>
static __device__ __forceinline__ void simt_load_chunk(const SimtParams& p, const TileDesc& td, int k0, int tid,
                                                       SimtChunk<MJ>& c) {
  const int N = p.n_fft, H = p.hop, W2 = 2 * p.mp, row4 = W2 / 4;
#pragma unroll
  for (int i = 0; i < SimtChunk<MJ>::kXq; ++i) {
    const int idx = tid + i * kThreads;
    const int k = idx % kKC, f = idx / kKC;
    const int n = k0 + k;
    c.x[i] = (f < td.n_frames && n < N) ? __ldg(p.wave + td.in_off + (int64_t)f * H + n) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < SimtChunk<MJ>::kWq; ++i) {
    const int idx = tid + i * kThreads;
    const int k = idx / row4, c4 = idx - k * row4;
    c.w[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx < kKC * row4 && k0 + k < N) c.w[i] = __ldg(reinterpret_cast<const float4*>(p.w32 + (size_t)(k0 + k) * W2) + c4);
  }
}

template <int MJ>
static __device__ __forceinline__ void simt_store_chunk(const SimtParams& p, int tid, const SimtChunk<MJ>& c,
                                                        float* Xs, float* Ws) {
  const int W2 = 2 * p.mp, row4 = W2 / 4;
#pragma unroll
  for (int i = 0; i < SimtChunk<MJ>::kXq; ++i) {
    const int idx = tid + i * kThreads;
    Xs[(idx % kKC) * (kF + kXPad) + idx / kKC] = c.x[i];
  }
#pragma unroll
  for (int i = 0; i < SimtChunk<MJ>::kWq; ++i) {
    const int idx = tid + i * kThreads;
    if (idx < kKC * row4) {
      const int k = idx / row4, c4 = idx - k * row4;
      reinterpret_cast<float4*>(Ws + k * W2)[c4] = c.w[i];
    }
  }
}

template <int MJ>
__global__ void __launch_bounds__(kThreads, 1) melt_simt_kernel(SimtParams p) {
  extern __shared__ __align__(16) float smem[];
  constexpr int kXs = kKC * (kF + kXPad);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int N = p.n_fft, M = p.n_mels, W2 = 2 * p.mp;
  const int kWs = kKC * W2;
  float* Xbuf[2] = {smem, smem + kXs + kWs};          // [kKC][kF + kXPad], then the basis chunk [kKC][2 mp]
  float* Wbuf[2] = {smem + kXs, smem + 2 * kXs + kWs};

  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x) {
    const TileDesc td = p.tiles[tile];
    float acc[8][MJ][2];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < MJ; ++j) acc[i][j][0] = acc[i][j][1] = 0.f;

    SimtChunk<MJ> nxt;
    simt_load_chunk<MJ>(p, td, 0, tid, nxt);
    __syncthreads();  // the previous tile's readers of both buffers (and the MFCC staging) are done
    simt_store_chunk<MJ>(p, tid, nxt, Xbuf[0], Wbuf[0]);
    __syncthreads();
    int b = 0;
    for (int k0 = 0; k0 < N; k0 += kKC, b ^= 1) {
      const bool more = k0 + kKC < N;
      if (more) simt_load_chunk<MJ>(p, td, k0 + kKC, tid, nxt);
      const float* Xs = Xbuf[b];
      const float* Ws = Wbuf[b];
      const int kn = min(kKC, N - k0);
#pragma unroll 4
      for (int k = 0; k < kn; ++k) {
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
      if (more) {
        simt_store_chunk<MJ>(p, tid, nxt, Xbuf[b ^ 1], Wbuf[b ^ 1]);  // its last readers finished a chunk ago
        __syncthreads();
      }
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
static cudaError_t launch_mj(const SimtParams& p, int grid, cudaStream_t stream) {
  const int smem = simt_smem_bytes(MJ, p.n_mels, p.n_mfcc);
  cudaError_t e = cudaFuncSetAttribute(melt_simt_kernel<MJ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  melt_simt_kernel<MJ><<<grid, kThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_simt(const SimtParams& p, int mj, int grid, cudaStream_t stream) {
  switch (mj) {
    case 1: return launch_mj<1>(p, grid, stream);
    case 2: return launch_mj<2>(p, grid, stream);
    case 3: return launch_mj<3>(p, grid, stream);
    case 4: return launch_mj<4>(p, grid, stream);
    case 5: return launch_mj<5>(p, grid, stream);
    case 6: return launch_mj<6>(p, grid, stream);
    case 7: return launch_mj<7>(p, grid, stream);
    case 8: return launch_mj<8>(p, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace melt
