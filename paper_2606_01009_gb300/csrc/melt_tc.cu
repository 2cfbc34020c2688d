// Host side of the tensor-core MelT kernels: basis operand images, the
// shared-memory plan and the launch.  The device code is in melt_tc_kernel.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "melt_tc_kernel.cuh"

namespace melt {

using namespace tc;

namespace {

// Round-to-nearest-even of an exact double to bfloat16 (8 significant bits).
uint16_t bf16_bits(double v) {
  if (v == 0.0) return std::signbit(v) ? 0x8000 : 0;
  int e;
  std::frexp(v, &e);
  if (e < -125) e = -125;
  const double q = std::nearbyint(std::ldexp(v, 8 - e));
  const float f = (float)std::ldexp(q, e - 8);
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  return (uint16_t)(bits >> 16);
}

double bf16_value(uint16_t b) {
  const uint32_t bits = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &bits, 4);
  return f;
}

// Round-to-nearest-even of an exact double to FP8 e4m3 (saturating at 448).
uint8_t e4m3_bits(double v) {
  const uint8_t sign = std::signbit(v) ? 0x80 : 0;
  double a = std::fabs(v);
  if (a == 0.0) return sign;
  int e;
  std::frexp(a, &e);
  if (e < -5) e = -5;
  double r = std::ldexp(std::nearbyint(std::ldexp(a, 4 - e)), e - 4);
  if (r > 448.0) r = 448.0;
  if (r < 0.015625) return sign | (uint8_t)(r * 512.0);  // subnormal: r = m 2^-9
  int ee;
  const double mm = std::frexp(r, &ee);  // r = mm 2^ee, mm in [0.5, 1)
  const int ef = ee - 1 + 7;
  const int mant = (int)((mm * 2.0 - 1.0) * 8.0);
  return sign | (uint8_t)(ef << 3) | (uint8_t)mant;
}

constexpr uint32_t kSmemLimit = 227 * 1024;

uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// Shared-memory plan for one basis; false if it cannot fit.
bool plan_smem(const TcBasis* tb, TcParams& p, int n_mfcc) {
  const int P = tb->precision;
  p.N = tb->n_fft;
  p.H = tb->hop;
  p.M = tb->n_mels;
  p.MP = (p.M + 15) / 16 * 16;
  p.NC = 2 * p.MP;
  p.J = tb->J;
  p.KS = tb->ksteps;
  p.zrows = kF + p.J - 1;
  p.items = p.zrows * (p.H / 8);
  p.inv_h8 = 8.0f / (float)p.H;
  p.kstep_bytes = (uint32_t)tb->kstep_bytes;
  const int parts = P == MELT_BF16X3 ? 2 : 1;
  p.bslot_bytes = p.kstep_bytes * parts;
  if (P == MELT_FP8E4M3) {
    p.lbo_a = kF * 16 + 16;                    // 128 rows x 16 B, +16 B spreads banks
    p.a_bytes = p.lbo_a * (uint32_t)(p.KS * 2);
  } else {
    int zr = p.zrows;
    while ((zr & 7) != 1) ++zr;                // rows % 8 == 1: converter stores spread banks
    p.lbo_a = (uint32_t)zr * 16;
    p.a_bytes = p.lbo_a * (uint32_t)(p.H / 8);
  }
  p.abuf_bytes = p.a_bytes * parts;
  // The tile's FP32 span is staged in chunks of whole Z rows, ~16 KB each
  // (the FP8 form holds the whole span at once).
  const uint32_t row_bytes = (uint32_t)p.H * 4;
  const uint32_t span_bytes = row_bytes * p.zrows;
  p.NCHUNK = (int)((span_bytes + 16383) / 16384);
  p.CH = (p.zrows + p.NCHUNK - 1) / p.NCHUNK;
  // a converter thread handles at most kQuadsPerThread float4s of a chunk
  const int max_rows = kQuadsPerThread * kCvtThreads * 4 / p.H;
  if (p.CH > max_rows) p.CH = std::max(1, max_rows);
  p.NCHUNK = (p.zrows + p.CH - 1) / p.CH;
  p.st_bytes = row_bytes * p.CH;  // slots back to back: the FP8 form reads the span contiguously
  // Layout candidates, best first: the whole basis resident in shared memory
  // (loaded once per CTA), then a streamed basis ring; two A buffers before one.
  struct Cand { int resident, zb, nb, ns; };
  std::vector<Cand> cands;
  for (int ns = 4; ns >= 3; --ns)
    for (int zb = 2; zb >= 1; --zb) cands.push_back({1, zb, p.KS, ns});
  for (int zb = 2; zb >= 1; --zb)
    for (int nb = std::min(p.KS, 24); nb >= 4; --nb) cands.push_back({0, zb, nb, 3});
  for (int zb = 2; zb >= 1; --zb)
    for (int nb = 3; nb >= 2; --nb)
      for (int ns = 3; ns >= 2; --ns) cands.push_back({0, zb, nb, ns});
  for (const Cand& c : cands) {
    p.b_resident = c.resident;
    p.ZB = c.zb;
    p.NB = c.nb;
    p.NS = (P == MELT_FP8E4M3) ? p.NCHUNK : c.ns;
    const Bars B(p.NS, p.ZB, p.NB);
    uint32_t off = 0;
    p.off_a = off;
    off += align_up(p.abuf_bytes * p.ZB, 128);
    p.off_st = off;
    off += align_up(p.st_bytes * p.NS, 128);
    p.off_b = off;
    off += align_up(p.bslot_bytes * p.NB, 128);
    p.off_bar = off;
    off += align_up(8 * B.total, 128);
    p.off_tab = off;
    off += align_up(8 * p.KS, 128);
    p.off_misc = off;
    off += 128;
    p.off_scale = off;
    off += (P == MELT_FP8E4M3) ? kScaleRing * kF * 4 : 0;
    p.off_rowmax = off;
    off += (P == MELT_FP8E4M3) ? align_up((2 * p.zrows + kF) * 4, 128) : 0;
    p.off_dct = off;
    off += align_up(4 * n_mfcc * p.MP, 128);
    if (off + 128 <= kSmemLimit) {
      p.smem_total = off + 128;
      p.tmem_cols = p.NC <= 32 ? 64 : p.NC <= 64 ? 128 : p.NC <= 128 ? 256 : 512;
      p.acc_stride = p.tmem_cols / 2;
      p.idesc = idesc_f32acc(P == MELT_FP8E4M3 ? 0u : 1u, kF, p.NC);
      p.desc_hi = (128u >> 4) | (1u << 14);  // SBO = 128 B; version bit (descriptor bit 46)
      return true;
    }
  }
  return false;
}

}  // namespace

melt_status tc_build(TcBasis* tb, const TcConfig& c, const double* w64) {
  const int N = c.n_fft, H = c.hop, M = c.n_mels, P = c.precision;
  if (P != MELT_BF16 && P != MELT_BF16X3 && P != MELT_FP8E4M3) return MELT_ERR_ARG;
  if (P != MELT_FP8E4M3 && (H % 16) != 0) return MELT_ERR_UNSUPPORTED;
  if (M > 128) return MELT_ERR_UNSUPPORTED;
  const int MP = (M + 15) / 16 * 16, NC = 2 * MP;
  const int J = (N + H - 1) / H;
  int KS = 0;
  std::vector<std::pair<int, int>> steps;  // BF16 forms: (j, first column r0)
  if (P == MELT_FP8E4M3) {
    KS = (N + 31) / 32;
  } else {
    for (int j = 0; j < J; ++j) {
      const int kj = std::min(H, N - j * H);
      for (int kk = 0; kk < (kj + 15) / 16; ++kk) steps.push_back({j, 16 * kk});
    }
    KS = (int)steps.size();
  }
  const size_t kstep_bytes = (size_t)NC * 32;  // 2 core columns x NC rows x 16 B
  const int parts = (P == MELT_BF16X3) ? 2 : 1;
  std::vector<uint8_t> img((size_t)KS * parts * kstep_bytes, 0);
  auto wval = [&](int row, int n) -> double {  // row of the stacked, padded basis
    if (n < 0 || n >= N) return 0.0;
    if (row < MP) return row < M ? w64[(size_t)row * N + n] : 0.0;
    const int m = row - MP;
    return m < M ? w64[(size_t)(M + m) * N + n] : 0.0;
  };
  for (int s = 0; s < KS; ++s) {
    uint8_t* blk = img.data() + (size_t)s * parts * kstep_bytes;
    for (int cc = 0; cc < 2; ++cc)
      for (int row = 0; row < NC; ++row) {
        if (P == MELT_FP8E4M3) {
          for (int e = 0; e < 16; ++e) {
            const int n = 32 * s + 16 * cc + e;
            blk[(size_t)cc * NC * 16 + row * 16 + e] = e4m3_bits(wval(row, n) * 448.0);
          }
        } else {
          const int j = steps[s].first, r0 = steps[s].second;
          for (int e = 0; e < 8; ++e) {
            const int r = r0 + 8 * cc + e;
            const double w = (r < H) ? wval(row, j * H + r) : 0.0;
            const uint16_t hi = bf16_bits(w);
            std::memcpy(blk + (size_t)cc * NC * 16 + row * 16 + e * 2, &hi, 2);
            if (P == MELT_BF16X3) {
              const uint16_t lo = bf16_bits(w - bf16_value(hi));
              std::memcpy(blk + kstep_bytes + (size_t)cc * NC * 16 + row * 16 + e * 2, &lo, 2);
            }
          }
        }
      }
  }
  tb->precision = P;
  tb->n_fft = N;
  tb->hop = H;
  tb->n_mels = M;
  tb->J = J;
  tb->ksteps = KS;
  tb->kstep_k = P == MELT_FP8E4M3 ? 32 : 16;
  tb->n_cols = NC;
  tb->kstep_bytes = kstep_bytes;
  {
    TcParams probe;
    std::memset(&probe, 0, sizeof(probe));
    if (!plan_smem(tb, probe, c.n_mfcc)) return MELT_ERR_UNSUPPORTED;  // operands do not fit shared memory
  }
  if (cudaMalloc(&tb->d_b, img.size()) != cudaSuccess) return MELT_ERR_OOM;
  if (cudaMemcpy(tb->d_b, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return MELT_ERR_CUDA;
  return MELT_OK;
}

void tc_free(TcBasis* tb) {
  cudaFree(tb->d_b);
  cudaFree(tb->d_b_lo);
  cudaFree(tb->d_kmap);
  tb->d_b = tb->d_b_lo = nullptr;
  tb->d_kmap = nullptr;
}

int tc_max_mfcc() { return kMaxMfccTc; }

cudaError_t tc_launch(const TcBasis* tb, const TcLaunch& L, cudaStream_t stream) {
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  if (!plan_smem(tb, p, L.n_mfcc)) return cudaErrorInvalidConfiguration;
  if (L.n_mfcc > kMaxMfccTc) return cudaErrorInvalidValue;
  p.wave = L.wave;
  p.tiles = L.tiles;
  p.n_tiles = L.n_tiles;
  p.bimg = static_cast<const uint8_t*>(tb->d_b);
  p.dct = L.dct;
  p.out = L.out;
  p.err = L.err;
  p.eps = L.eps;
  p.n_mfcc = L.n_mfcc;
  p.n_out = L.n_mfcc ? L.n_mfcc : tb->n_mels;
  KernelFn fn = L.n_mfcc ? kernel_for_mfcc(tb->precision, p.MP / 16)
                        : kernel_for_plain(tb->precision, p.MP / 16);
  if (!fn) return cudaErrorInvalidValue;
  const int smem = (int)p.smem_total;
  static thread_local KernelFn last_fn = nullptr;
  static thread_local int last_smem = 0;
  if (fn != last_fn || smem > last_smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    last_fn = fn;
    last_smem = smem;
  }
  const int grid = std::min(L.n_tiles, L.sm_count);
  fn<<<grid, kThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace melt
