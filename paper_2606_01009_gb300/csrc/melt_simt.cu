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
// chunk (row-major [k][2*mp], R/I interleaved) is copied beside it.
#include "melt_internal.h"

namespace melt {

namespace {

constexpr int kF = kTileFrames;  // 128
constexpr int kKC = 32;          // samples per K chunk
constexpr int kXPad = 4;         // Xs row padding (keeps float4 alignment)
constexpr int kThreads = 256;

template <int MJ>
__global__ void __launch_bounds__(kThreads, 1) melt_simt_kernel(SimtParams p) {
  extern __shared__ __align__(16) float smem[];
  constexpr int kXs = kKC * (kF + kXPad);
  float* Xs = smem;             // [kKC][kF + kXPad]
  float* Ws = smem + kXs;       // [kKC][2*mp]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int N = p.n_fft, H = p.hop, M = p.n_mels, W2 = 2 * p.mp;

  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x) {
    const TileDesc td = p.tiles[tile];
    float acc[8][MJ][2];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < MJ; ++j) acc[i][j][0] = acc[i][j][1] = 0.f;

    for (int k0 = 0; k0 < N; k0 += kKC) {
      __syncthreads();
      // Frame chunk, transposed: Xs[k][f] = x[in_off + f*H + k0 + k]
#pragma unroll 4
      for (int i = 0; i < kF * kKC / kThreads; ++i) {
        const int idx = tid + i * kThreads;
        const int k = idx % kKC, f = idx / kKC;
        const int n = k0 + k;
        float v = 0.f;
        if (f < td.n_frames && n < N) v = __ldg(p.wave + td.in_off + (int64_t)f * H + n);
        Xs[k * (kF + kXPad) + f] = v;
      }
      // Basis chunk: rows k0..k0+31 of w32 (zero past N)
      const int row4 = W2 / 4;
      for (int idx = tid; idx < kKC * row4; idx += kThreads) {
        const int k = idx / row4, c4 = idx - k * row4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k0 + k < N) v = __ldg(reinterpret_cast<const float4*>(p.w32 + (size_t)(k0 + k) * W2) + c4);
        reinterpret_cast<float4*>(Ws + k * W2)[c4] = v;
      }
      __syncthreads();
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
    __syncthreads();
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
  int bytes = (kKC * (kF + kXPad) + kKC * 2 * mp) * (int)sizeof(float);
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
