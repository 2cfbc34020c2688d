// Learned per-frame correction of MelT features (a residual MLP) and its
// training step.  The paper does not evaluate such a layer: Sec. VI-C names a
// calibration layer as future work, and Sec. IV-H / Sec. V describe the
// MelT-to-STFT+Mel gap as mostly a per-band affine map.  The model:
//
//   xh = (x - mu) / sd                  per-band standardisation (fixed stats)
//   h  = xh W1^T + b1                   W1 [Hd x M]
//   a  = GELU(h) = 0.5 h (1 + erf(h / sqrt 2))
//   y  = x + a W2^T + b2                W2 [M x Hd], residual output
//   L  = mean over the batch and the M bands of (y - target)^2
//
// and AdamW with decoupled weight decay on every parameter.  Everything runs
// in FP32 on CUDA cores: one training step is a few hundred MFLOP, far too
// small to be worth tensor-core tiles, and FP32 keeps the gradients close
// enough to the FP64 definition to check them element by element.
//
// Kernels of one step (B = batch rows gathered through `rows`):
//   1. H = Xh W1^T + b1, A = GELU(H)                  [B x Hd]
//   2. Y = X + A W2^T + b2, dY = 2 (Y - T) / (B M), loss partial sums
//   3. dH = (dY W2) * GELU'(H)                        [B x Hd]
//   4. dW2 = dY^T A, dW1 = dH^T Xh                    (sums over the batch)
//   5. db1, db2 = column sums of dH, dY
//   6. AdamW over the packed parameter vector
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "melt_internal.h"

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;
constexpr int kMaxIn = 128;       // M (bands) limit of the fused apply kernel
constexpr int kApplyFrames = 64;  // frames per CTA of the fused apply kernel
constexpr int kApplyChunk = 64;   // hidden units per chunk of the fused apply kernel

__device__ __forceinline__ float gelu_f(float h) {
  return 0.5f * h * (1.0f + erff(h * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float h) {
  return 0.5f * (1.0f + erff(h * 0.70710678118654752f)) +
         h * 0.39894228040143268f * expf(-0.5f * h * h);
}

// ---- operand loaders: (i, k) -> element of op(A) [rows i, inner k]
struct LoadRowK {            // p[i * ld + k]
  const float* p;
  long long ld;
  static constexpr bool kMajorK = true;
  __device__ float operator()(long long i, long long k) const { return p[i * ld + k]; }
};
struct LoadColK {            // p[k * ld + i]
  const float* p;
  long long ld;
  static constexpr bool kMajorK = false;
  __device__ float operator()(long long i, long long k) const { return p[k * ld + i]; }
};
struct LoadStdX {            // standardised x of gathered row i, band k
  const float* x;
  const int64_t* rows;
  const float* mu;
  const float* sd;
  int M;
  static constexpr bool kMajorK = true;
  __device__ float operator()(long long i, long long k) const {
    const long long r = rows ? rows[i] : i;
    return (x[r * M + k] - mu[k]) / sd[k];
  }
};
struct LoadStdXT {           // transposed: (band i, row k)
  LoadStdX s;
  static constexpr bool kMajorK = false;
  __device__ float operator()(long long i, long long k) const { return s(k, i); }
};

// ---- epilogues: called once per output element (i, j) with the dot product
struct EpiHidden {           // H = acc + b1, A = GELU(H)
  const float* b1;
  float* H;
  float* A;
  int Hd;
  __device__ void operator()(long long i, long long j, float acc) const {
    const float h = acc + b1[j];
    H[i * Hd + j] = h;
    A[i * Hd + j] = gelu_f(h);
  }
};
struct EpiOutGrad {          // Y = X + acc + b2; dY = 2 (Y - T) / (B M); loss partial
  const float* x;
  const float* t;
  const int64_t* rows;
  const float* b2;
  float* dY;
  float* loss_acc;           // per-thread partial, summed by the caller
  int M;
  float scale;               // 2 / (B M)
  __device__ void operator()(long long i, long long j, float acc) const {
    const long long r = rows ? rows[i] : i;
    const float y = x[r * M + j] + acc + b2[j];
    const float d = y - t[r * M + j];
    dY[i * M + j] = scale * d;
    *loss_acc += d * d;
  }
};
struct EpiBackHidden {       // dH = acc * GELU'(H)
  const float* H;
  float* dH;
  int Hd;
  __device__ void operator()(long long i, long long j, float acc) const {
    dH[i * Hd + j] = acc * gelu_grad_f(H[i * Hd + j]);
  }
};
struct EpiStore {            // G[i * ld + j] = acc
  float* g;
  long long ld;
  __device__ void operator()(long long i, long long j, float acc) const { g[i * ld + j] = acc; }
};

// C[i, j] = sum_k opA(i, k) opB(j, k), 64 x 64 tiles, 4 x 4 outputs per thread.
template <class LA, class LB, class EPI>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(long long nr, long long nc, long long K,
                                                            LA la, LB lb, EPI epi, float* loss) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long long i0 = (long long)blockIdx.y * kBM, j0 = (long long)blockIdx.x * kBN;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  for (long long k0 = 0; k0 < K; k0 += kBK) {
    for (int e = threadIdx.x; e < kBM * kBK; e += kGemmThreads) {
      const int ii = LA::kMajorK ? e / kBK : e % kBM;
      const int kk = LA::kMajorK ? e % kBK : e / kBM;
      As[kk][ii] = (i0 + ii < nr && k0 + kk < K) ? la(i0 + ii, k0 + kk) : 0.f;
    }
    for (int e = threadIdx.x; e < kBN * kBK; e += kGemmThreads) {
      const int jj = LB::kMajorK ? e / kBK : e % kBN;
      const int kk = LB::kMajorK ? e % kBK : e / kBN;
      Bs[kk][jj] = (j0 + jj < nc && k0 + kk < K) ? lb(j0 + jj, k0 + kk) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  float part = 0.f;
  EPI e = epi;
  if constexpr (std::is_same<EPI, EpiOutGrad>::value) e.loss_acc = &part;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const long long i = i0 + ty * 4 + r, j = j0 + tx * 4 + c;
      if (i < nr && j < nc) e(i, j, acc[r][c]);
    }
  if constexpr (std::is_same<EPI, EpiOutGrad>::value) {
    if (loss) atomicAdd(loss, part);
  }
}

template <class LA, class LB, class EPI>
cudaError_t gemm(long long nr, long long nc, long long K, LA la, LB lb, EPI epi, float* loss,
                 cudaStream_t s) {
  const dim3 grid((unsigned)((nc + kBN - 1) / kBN), (unsigned)((nr + kBM - 1) / kBM));
  gemm_kernel<LA, LB, EPI><<<grid, kGemmThreads, 0, s>>>(nr, nc, K, la, lb, epi, loss);
  return cudaGetLastError();
}

// db1[j] = sum_b dH[b, j] (j < Hd), db2[m] = sum_b dY[b, m]
__global__ void colsum_kernel(const float* dH, const float* dY, int B, int Hd, int M, float* db1,
                              float* db2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Hd + M) return;
  float s = 0.f;
  if (c < Hd) {
    for (int b = 0; b < B; ++b) s += dH[(long long)b * Hd + c];
    db1[c] = s;
  } else {
    const int m = c - Hd;
    for (int b = 0; b < B; ++b) s += dY[(long long)b * M + m];
    db2[m] = s;
  }
}

__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, long long n, float lr,
                             float b1, float b2, float eps, float wd, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] = p[i] * (1.f - lr * wd) - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Per-band population mean and standard deviation (two passes, one thread per band).
__global__ void stats_kernel(const float* x, long long n, int M, float* mu, float* sd) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (long long r = 0; r < n; ++r) s += x[r * M + m];
  const double mean = n > 0 ? s / (double)n : 0.0;
  double q = 0.0;
  for (long long r = 0; r < n; ++r) {
    const double d = x[r * M + m] - mean;
    q += d * d;
  }
  mu[m] = (float)mean;
  sd[m] = (float)fmax(sqrt(n > 0 ? q / (double)n : 0.0), 1e-6);
}

// Fused forward for inference: y = x + W2 GELU(W1 xh + b1) + b2 over kApplyFrames
// frames per CTA; the hidden layer is formed kApplyChunk units at a time in
// shared memory and never leaves the SM.  In place (y == x) is allowed: each
// output element is read and then written by the same thread.
// Dynamic shared memory: xs [F][M+1], w1c [C][M+1], w2c [M][C+1], ac [F][C+1].
int apply_smem_bytes(int M) {
  return 4 * (kApplyFrames * (M + 1) + kApplyChunk * (M + 1) + M * (kApplyChunk + 1) +
              kApplyFrames * (kApplyChunk + 1));
}

__global__ void __launch_bounds__(256) apply_kernel(const float* x, float* y, long long n,
                                                    const float* W1, const float* b1,
                                                    const float* W2, const float* b2,
                                                    const float* mu, const float* sd, int M,
                                                    int Hd) {
  extern __shared__ float sm[];
  const int ldx = M + 1, ldc = kApplyChunk + 1;
  float* xs = sm;                              // [kApplyFrames][ldx]
  float* w1c = xs + kApplyFrames * ldx;        // [kApplyChunk][ldx]
  float* w2c = w1c + kApplyChunk * ldx;        // [M][ldc]
  float* ac = w2c + M * ldc;                   // [kApplyFrames][ldc]
  const int t = threadIdx.x;
  const long long f0 = (long long)blockIdx.x * kApplyFrames;
  for (int e = t; e < kApplyFrames * M; e += 256) {
    const int f = e / M, m = e - f * M;
    xs[f * ldx + m] = (f0 + f < n) ? (x[(f0 + f) * M + m] - mu[m]) / sd[m] : 0.f;
  }
  // output accumulators: frames fy*4 .. +3, bands ox + 16 q
  const int fy = t >> 4, ox = t & 15;
  const int nq = (M + 15) >> 4;
  float acc[4][kMaxIn / 16];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < kMaxIn / 16; ++q) acc[r][q] = 0.f;
  for (int h0 = 0; h0 < Hd; h0 += kApplyChunk) {
    __syncthreads();  // previous chunk fully consumed (and xs written, first time)
    for (int e = t; e < kApplyChunk * M; e += 256) {
      const int j = e / M, m = e - j * M;
      w1c[j * ldx + m] = W1[(long long)(h0 + j) * M + m];
    }
    for (int e = t; e < M * kApplyChunk; e += 256) {
      const int o = e / kApplyChunk, j = e - o * kApplyChunk;
      w2c[o * ldc + j] = W2[(long long)o * Hd + h0 + j];
    }
    __syncthreads();
    // hidden chunk: ac[f][j] = GELU(b1 + xs[f] . w1c[j]); thread: frames fy*4.., units ox*4..
    {
      float hacc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) hacc[r][c] = 0.f;
      for (int m = 0; m < M; ++m) {
        float a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = xs[(fy * 4 + r) * ldx + m];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = w1c[(ox * 4 + c) * ldx + m];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) hacc[r][c] = fmaf(a[r], b[c], hacc[r][c]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          ac[(fy * 4 + r) * ldc + ox * 4 + c] = gelu_f(hacc[r][c] + b1[h0 + ox * 4 + c]);
    }
    __syncthreads();
    for (int j = 0; j < kApplyChunk; ++j) {
      float a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = ac[(fy * 4 + r) * ldc + j];
#pragma unroll
      for (int q = 0; q < kMaxIn / 16; ++q) {
        const int o = ox + 16 * q;
        if (q < nq && o < M) {
          const float w = w2c[o * ldc + j];
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[r][q] = fmaf(a[r], w, acc[r][q]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const long long f = f0 + fy * 4 + r;
    if (f >= n) continue;
#pragma unroll
    for (int q = 0; q < kMaxIn / 16; ++q) {
      const int o = ox + 16 * q;
      if (q < nq && o < M) y[f * M + o] = x[f * M + o] + acc[r][q] + b2[o];
    }
  }
}

}  // namespace

struct melt_mlp {
  int device = 0;
  int M = 0, Hd = 0;
  long long n_params = 0;
  float* d_params = nullptr;  // [W1 | b1 | W2 | b2]
  float* d_grads = nullptr;   // same packing
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_mu = nullptr;
  float* d_sd = nullptr;
  long long t = 0;            // AdamW steps taken
  double lr = 1e-3, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, wd = 0.01;
  int cap = 0;                // batch rows the workspace holds
  float* d_H = nullptr;
  float* d_A = nullptr;
  float* d_dY = nullptr;
  float* d_dH = nullptr;
};

namespace {

long long param_count(int M, int Hd) { return 2LL * M * Hd + Hd + M; }

void free_ws(melt_mlp* p) {
  cudaFree(p->d_H);
  cudaFree(p->d_A);
  cudaFree(p->d_dY);
  cudaFree(p->d_dH);
  p->d_H = p->d_A = p->d_dY = p->d_dH = nullptr;
  p->cap = 0;
}

melt_status ensure_ws(melt_mlp* p, int batch) {
  if (batch <= p->cap) return MELT_OK;
  free_ws(p);
  const size_t h = (size_t)batch * p->Hd * sizeof(float), o = (size_t)batch * p->M * sizeof(float);
  if (melt::dev_alloc(&p->d_H, h) != cudaSuccess || melt::dev_alloc(&p->d_A, h) != cudaSuccess ||
      melt::dev_alloc(&p->d_dY, o) != cudaSuccess || melt::dev_alloc(&p->d_dH, h) != cudaSuccess) {
    free_ws(p);
    return MELT_ERR_OOM;
  }
  p->cap = batch;
  return MELT_OK;
}

melt_status grad_impl(melt_mlp* p, const float* X, const float* T, const int64_t* rows, int B,
                      float* grads, float* loss, cudaStream_t s) {
  const int M = p->M, Hd = p->Hd;
  const float* W1 = p->d_params;
  const float* b1 = W1 + (long long)Hd * M;
  const float* W2 = b1 + Hd;
  const float* b2 = W2 + (long long)M * Hd;
  float* gW1 = grads;
  float* gb1 = gW1 + (long long)Hd * M;
  float* gW2 = gb1 + Hd;
  float* gb2 = gW2 + (long long)M * Hd;
  const LoadStdX sx{X, rows, p->d_mu, p->d_sd, M};
  cudaError_t e;
  // 1. H = Xh W1^T + b1, A = GELU(H)
  e = gemm(B, Hd, M, sx, LoadRowK{W1, M}, EpiHidden{b1, p->d_H, p->d_A, Hd}, nullptr, s);
  if (e != cudaSuccess) return MELT_ERR_CUDA;
  // 2. Y = X + A W2^T + b2 -> dY, loss
  e = gemm(B, M, Hd, LoadRowK{p->d_A, Hd}, LoadRowK{W2, Hd},
           EpiOutGrad{X, T, rows, b2, p->d_dY, nullptr, M, 2.f / ((float)B * (float)M)}, loss, s);
  if (e != cudaSuccess) return MELT_ERR_CUDA;
  // 3. dH = (dY W2) * GELU'(H):  op(B)(j, m) = W2[m, j]
  e = gemm(B, Hd, M, LoadRowK{p->d_dY, M}, LoadColK{W2, Hd}, EpiBackHidden{p->d_H, p->d_dH, Hd},
           nullptr, s);
  if (e != cudaSuccess) return MELT_ERR_CUDA;
  // 4. dW2[m, j] = sum_b dY[b, m] A[b, j];  dW1[j, m] = sum_b dH[b, j] Xh[b, m]
  e = gemm(M, Hd, B, LoadColK{p->d_dY, M}, LoadColK{p->d_A, Hd}, EpiStore{gW2, Hd}, nullptr, s);
  if (e != cudaSuccess) return MELT_ERR_CUDA;
  e = gemm(Hd, M, B, LoadColK{p->d_dH, Hd}, LoadStdXT{sx}, EpiStore{gW1, M}, nullptr, s);
  if (e != cudaSuccess) return MELT_ERR_CUDA;
  // 5. bias gradients
  colsum_kernel<<<(Hd + M + 127) / 128, 128, 0, s>>>(p->d_dH, p->d_dY, B, Hd, M, gb1, gb2);
  if (cudaGetLastError() != cudaSuccess) return MELT_ERR_CUDA;
  return MELT_OK;
}

melt_status check_batch(const melt_mlp* p, const float* X, const float* T, int batch) {
  if (!p || !X || !T || batch < 1) return MELT_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MELT_ERR_CUDA;
  return dev == p->device ? MELT_OK : MELT_ERR_ARG;
}

}  // namespace

namespace melt {

// ---- image of the MLP for the CTA-pair kernel's fused epilogue
// Two halves, one per CTA of a pair; each half is
//   W1 blocks  MP/16 K-steps x [2 core columns][Hd/2 rows][8 bf16]   rows n of W1
//              from r*Hd/2 (hidden units), K = bands (zero past M)
//   W2 blocks  Hd/16 K-steps x [2 core columns][MP/2 rows][8 bf16]   rows o of W2
//              from r*MP/2 (bands, zero past M), K = hidden units
//   vectors    FP32 b1[Hd], b2[MP], mu[MP], 1/sd[MP] (zero past M), padded to 128 B
// The blocks are the no-swizzle K-major core-matrix layout of the tcgen05
// B operand (rows 16 B apart, the two core columns of a K-step Hd/2*16 or
// MP/2*16 bytes apart).
bool mlp_fused_shape_ok(int M, int Hd) {
  const int MP = (M + 15) / 16 * 16;
  return M >= 1 && MP <= 80 && Hd >= 64 && Hd <= 256 && Hd % 32 == 0 && MP <= Hd / 2 &&
         (MP / 2) % 8 == 0;
}

long long mlp_fused_half_bytes(int M, int Hd) {
  const int MP = (M + 15) / 16 * 16;
  const long long w1 = (long long)(MP / 16) * 2 * (Hd / 2) * 16;
  const long long w2 = (long long)(Hd / 16) * 2 * (MP / 2) * 16;
  const long long vec = ((long long)(Hd + 3 * MP) * 4 + 127) / 128 * 128;
  return w1 + w2 + vec;
}

__global__ void fused_image_kernel(const float* prm, const float* mu, const float* sd, int M, int Hd,
                                   uint8_t* img, long long half) {
  const int MP = (M + 15) / 16 * 16;
  const long long w1b = (long long)(MP / 16) * 2 * (Hd / 2) * 8;  // bf16 elements
  const long long w2b = (long long)(Hd / 16) * 2 * (MP / 2) * 8;
  const int nvec = Hd + 3 * MP;
  const long long per_half = w1b + w2b + nvec;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * per_half) return;
  const int r = (int)(i / per_half);
  long long e = i - (long long)r * per_half;
  uint8_t* base = img + (long long)r * half;
  const float* W1 = prm;
  const float* b1 = W1 + (long long)Hd * M;
  const float* W2 = b1 + Hd;
  const float* b2 = W2 + (long long)M * Hd;
  if (e < w1b) {
    const int rows = Hd / 2;
    const int s = (int)(e / (2 * rows * 8));
    const int rem = (int)(e - (long long)s * 2 * rows * 8);
    const int cc = rem / (rows * 8), row = (rem / 8) % rows, q = rem % 8;
    const int n = r * rows + row, k = 16 * s + 8 * cc + q;
    const float v = k < M ? W1[(long long)n * M + k] : 0.f;
    reinterpret_cast<__nv_bfloat16*>(base)[e] = __float2bfloat16_rn(v);
    return;
  }
  e -= w1b;
  if (e < w2b) {
    const int rows = MP / 2;
    const int s = (int)(e / (2 * rows * 8));
    const int rem = (int)(e - (long long)s * 2 * rows * 8);
    const int cc = rem / (rows * 8), row = (rem / 8) % rows, q = rem % 8;
    const int o = r * rows + row, k = 16 * s + 8 * cc + q;
    const float v = o < M ? W2[(long long)o * Hd + k] : 0.f;
    reinterpret_cast<__nv_bfloat16*>(base + w1b * 2)[e] = __float2bfloat16_rn(v);
    return;
  }
  e -= w2b;
  float* vec = reinterpret_cast<float*>(base + (w1b + w2b) * 2);
  const int j = (int)e;
  float v;
  if (j < Hd) v = b1[j];
  else if (j < Hd + MP) v = (j - Hd < M) ? b2[j - Hd] : 0.f;
  else if (j < Hd + 2 * MP) v = (j - Hd - MP < M) ? mu[j - Hd - MP] : 0.f;
  else v = (j - Hd - 2 * MP < M) ? 1.f / sd[j - Hd - 2 * MP] : 0.f;
  vec[j] = v;
}

melt_status mlp_apply(const melt_mlp* p, const float* x, float* y, long long n, cudaStream_t s) {
  if (n <= 0) return MELT_OK;
  const float* W1 = p->d_params;
  const float* b1 = W1 + (long long)p->Hd * p->M;
  const float* W2 = b1 + p->Hd;
  const float* b2 = W2 + (long long)p->M * p->Hd;
  const long long blocks = (n + kApplyFrames - 1) / kApplyFrames;
  if (blocks > 0x7fffffffLL) return MELT_ERR_ARG;
  const int smem = apply_smem_bytes(p->M);
  if (cudaFuncSetAttribute(apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return MELT_ERR_CUDA;
  apply_kernel<<<(unsigned)blocks, 256, smem, s>>>(x, y, n, W1, b1, W2, b2, p->d_mu, p->d_sd, p->M,
                                                   p->Hd);
  return cudaGetLastError() == cudaSuccess ? MELT_OK : MELT_ERR_CUDA;
}

int mlp_inputs(const melt_mlp* p) { return p->M; }

melt_status mlp_fused_image(const melt_mlp* p, void* d_img, cudaStream_t s) {
  const int MP = (p->M + 15) / 16 * 16;
  const long long per_half = (long long)(MP / 16) * 2 * (p->Hd / 2) * 8 +
                             (long long)(p->Hd / 16) * 2 * (MP / 2) * 8 + p->Hd + 3 * MP;
  const long long n = 2 * per_half;
  fused_image_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      p->d_params, p->d_mu, p->d_sd, p->M, p->Hd, static_cast<uint8_t*>(d_img),
      mlp_fused_half_bytes(p->M, p->Hd));
  return cudaGetLastError() == cudaSuccess ? MELT_OK : MELT_ERR_CUDA;
}

int mlp_hidden(const melt_mlp* p) { return p->Hd; }

int mlp_device(const melt_mlp* p) { return p->device; }

}  // namespace melt

extern "C" {

int64_t melt_mlp_num_params(int n_in, int n_hidden) {
  if (n_in < 1 || n_hidden < 1) return 0;
  return param_count(n_in, n_hidden);
}

melt_status melt_mlp_create(int n_in, int n_hidden, const float* params, const float* mu,
                            const float* sd, melt_mlp** out) {
  if (!out || !params || n_in < 1 || n_in > kMaxIn || n_hidden < kApplyChunk ||
      n_hidden % kApplyChunk != 0 || n_hidden > 4096)
    return MELT_ERR_ARG;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MELT_ERR_NO_DEVICE;
  melt_mlp* p = new (std::nothrow) melt_mlp;
  if (!p) return MELT_ERR_OOM;
  p->device = dev;
  p->M = n_in;
  p->Hd = n_hidden;
  p->n_params = param_count(n_in, n_hidden);
  const size_t pb = (size_t)p->n_params * sizeof(float);
  bool ok = melt::dev_alloc(&p->d_params, pb) == cudaSuccess && melt::dev_alloc(&p->d_grads, pb) == cudaSuccess &&
            melt::dev_alloc(&p->d_m, pb) == cudaSuccess && melt::dev_alloc(&p->d_v, pb) == cudaSuccess &&
            melt::dev_alloc(&p->d_mu, n_in * sizeof(float)) == cudaSuccess &&
            melt::dev_alloc(&p->d_sd, n_in * sizeof(float)) == cudaSuccess;
  if (ok) {
    std::vector<float> m0(n_in, 0.f), s0(n_in, 1.f);
    ok = cudaMemcpy(p->d_params, params, pb, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(p->d_grads, 0, pb) == cudaSuccess && cudaMemset(p->d_m, 0, pb) == cudaSuccess &&
         cudaMemset(p->d_v, 0, pb) == cudaSuccess &&
         cudaMemcpy(p->d_mu, mu ? mu : m0.data(), n_in * sizeof(float), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(p->d_sd, sd ? sd : s0.data(), n_in * sizeof(float), cudaMemcpyHostToDevice) ==
             cudaSuccess;
  }
  if (!ok) {
    melt_mlp_destroy(p);
    return MELT_ERR_OOM;
  }
  *out = p;
  return MELT_OK;
}

melt_status melt_mlp_fit_stats(melt_mlp* p, const float* X, int64_t n, void* stream) {
  if (!p || !X || n < 1) return MELT_ERR_ARG;
  stats_kernel<<<(p->M + 63) / 64, 64, 0, (cudaStream_t)stream>>>(X, n, p->M, p->d_mu, p->d_sd);
  return cudaGetLastError() == cudaSuccess ? MELT_OK : MELT_ERR_CUDA;
}

melt_status melt_mlp_set_adamw(melt_mlp* p, double lr, double beta1, double beta2, double eps,
                               double wd) {
  if (!p || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0) ||
      !(wd >= 0))
    return MELT_ERR_ARG;
  p->lr = lr;
  p->beta1 = beta1;
  p->beta2 = beta2;
  p->eps = eps;
  p->wd = wd;
  return MELT_OK;
}

melt_status melt_mlp_grad(melt_mlp* p, const float* X, const float* target, const int64_t* rows,
                          int batch, float* grads, float* loss, void* stream) {
  melt_status st = check_batch(p, X, target, batch);
  if (st != MELT_OK) return st;
  if ((st = ensure_ws(p, batch)) != MELT_OK) return st;
  return grad_impl(p, X, target, rows, batch, grads ? grads : p->d_grads, loss, (cudaStream_t)stream);
}

melt_status melt_mlp_train_step(melt_mlp* p, const float* X, const float* target,
                                const int64_t* rows, int batch, float* loss, void* stream) {
  melt_status st = check_batch(p, X, target, batch);
  if (st != MELT_OK) return st;
  if ((st = ensure_ws(p, batch)) != MELT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = grad_impl(p, X, target, rows, batch, p->d_grads, loss, s)) != MELT_OK) return st;
  p->t += 1;
  const float c1 = (float)(1.0 / (1.0 - std::pow(p->beta1, (double)p->t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(p->beta2, (double)p->t)));
  const long long n = p->n_params;
  adamw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->d_params, p->d_grads, p->d_m, p->d_v, n,
                                                          (float)p->lr, (float)p->beta1,
                                                          (float)p->beta2, (float)p->eps,
                                                          (float)p->wd, c1, c2);
  return cudaGetLastError() == cudaSuccess ? MELT_OK : MELT_ERR_CUDA;
}

melt_status melt_mlp_adamw_apply(melt_mlp* p, const float* grads, void* stream) {
  if (!p || !grads) return MELT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(p->d_grads, grads, (size_t)p->n_params * sizeof(float),
                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return MELT_ERR_CUDA;
  p->t += 1;
  const float c1 = (float)(1.0 / (1.0 - std::pow(p->beta1, (double)p->t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(p->beta2, (double)p->t)));
  const long long n = p->n_params;
  adamw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->d_params, p->d_grads, p->d_m, p->d_v, n,
                                                          (float)p->lr, (float)p->beta1,
                                                          (float)p->beta2, (float)p->eps,
                                                          (float)p->wd, c1, c2);
  return cudaGetLastError() == cudaSuccess ? MELT_OK : MELT_ERR_CUDA;
}

melt_status melt_mlp_forward(const melt_mlp* p, const float* X, float* Y, int64_t n, void* stream) {
  if (!p || n < 0 || (n > 0 && (!X || !Y))) return MELT_ERR_ARG;
  return melt::mlp_apply(p, X, Y, n, (cudaStream_t)stream);
}

melt_status melt_mlp_get_params(const melt_mlp* p, float* params, float* mu, float* sd) {
  if (!p) return MELT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return MELT_ERR_CUDA;
  if (params && cudaMemcpy(params, p->d_params, (size_t)p->n_params * sizeof(float),
                           cudaMemcpyDeviceToHost) != cudaSuccess)
    return MELT_ERR_CUDA;
  if (mu && cudaMemcpy(mu, p->d_mu, p->M * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MELT_ERR_CUDA;
  if (sd && cudaMemcpy(sd, p->d_sd, p->M * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MELT_ERR_CUDA;
  return MELT_OK;
}

melt_status melt_mlp_destroy(melt_mlp* p) {
  if (!p) return MELT_OK;
  cudaDeviceSynchronize();
  free_ws(p);
  cudaFree(p->d_params);
  cudaFree(p->d_grads);
  cudaFree(p->d_m);
  cudaFree(p->d_v);
  cudaFree(p->d_mu);
  cudaFree(p->d_sd);
  delete p;
  return MELT_OK;
}

}  // extern "C"
