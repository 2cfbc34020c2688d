// Tensor-core MelT kernels for sm_103a: BF16, split-BF16 (three products)
// and FP8 e4m3 forms of the projection of Sec. III-A (Eq. 6), with power
// (Eq. 7), log (Eq. 8) and the optional DCT-II (Eq. 9) fused in the epilogue.
//
// One persistent CTA per SM walks a static round-robin list of tiles
// (128 consecutive frames of one clip).  Warp roles:
//   warps 0-3   epilogue: TMEM -> registers, R^2 + I^2, log, (DCT), store
//   warp  4     waveform producer: bulk async copies (TMA engine) of the
//               tile's contiguous FP32 sample span into a ring of chunks
//   warp  5     TMEM allocator + single-thread tcgen05.mma issuer
//   warp  6     basis producer: bulk copies of the basis K-step blocks
//   warps 7-10  converters: FP32 span -> MMA A operand in shared memory
//
// Implicit framing (no im2col in HBM).  Frames overlap (N > H), so the A
// operand's rows would be H samples apart, which a UMMA shared-memory
// descriptor cannot express.  The BF16 forms therefore use a polyphase
// split of the frame: with n = jH + r (0 <= r < H, j < J = ceil(N/H)) and
// Z[u][r] = x[(t0+u)H + r],
//     [R|I][t] = sum_j Z[t+j][:] . B_j^T,   B_j[c][r] = W[c][jH + r]
// so each sample is converted once into Z (rows of H samples, K-major
// canonical layout with rows 16 B apart) and the j-shift is a 16-byte
// offset of the A descriptor's start address.  The J slices accumulate
// into the same TMEM tile.  FP8 needs a per-frame scale, which differs
// between the frames that share a Z row, so the FP8 form writes each frame
// row (im2col inside shared memory only), scaled by 448/amax(frame).
//
// Accumulators: two TMEM tiles of 128 lanes x NC columns (NC = 2*MP, MP =
// M rounded up to 16): columns [0, MP) hold R, [MP, 2MP) hold I.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "melt_tc.h"
#include "sm100_ptx.cuh"

namespace melt {

namespace {

using namespace ptx;

constexpr int kEpiWarps = 4;
constexpr int kProdWarp = 4;
constexpr int kMmaWarp = 5;
constexpr int kBWarp = 6;
constexpr int kCvtWarp0 = 7;
constexpr int kCvtWarps = 4;
constexpr int kThreads = 32 * (kCvtWarp0 + kCvtWarps);  // 352
constexpr int kCvtThreads = 32 * kCvtWarps;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kF = kTileFrames;  // 128 = UMMA M
constexpr int kScaleRing = 4;    // FP8 per-frame scale buffers in flight

struct TcParams {
  const float* wave;
  const TileDesc* tiles;
  int n_tiles;
  const uint8_t* bimg;   // KS blocks of bslot_bytes
  const float* dct;      // [n_mfcc][M] or null
  float* out;
  int* err;
  float eps;
  int N, H, M, MP, NC, J, KS;
  int zrows;             // Z rows (BF16 forms: 128 + J - 1); FP8: rows of the staged span
  int n_out, n_mfcc;
  uint32_t kstep_bytes;  // one B part of one K-step
  uint32_t bslot_bytes;  // one ring slot (BF16X3: hi + lo parts)
  uint32_t lbo_a;        // A operand: bytes between K-adjacent core matrices
  uint32_t a_bytes;      // one A part
  uint32_t abuf_bytes;   // one A buffer (BF16X3: hi + lo parts)
  int ZB;                // A buffers
  int NS, CH, NCHUNK;    // staging slots, Z rows per chunk, chunks per tile
  uint32_t st_bytes;     // bytes per staging slot
  int NB;                // basis ring slots (resident mode: NB == KS, loaded once)
  int b_resident;        // 1: the whole basis stays in shared memory for the CTA's life
  uint32_t tmem_cols, acc_stride, idesc;
  uint32_t off_a, off_st, off_b, off_bar, off_misc, off_scale, off_rowmax;
  uint32_t smem_total;   // dynamic shared memory bytes (incl. alignment slack)
};

// barrier indices
struct Bars {
  int s_full, s_empty, z_full, z_empty, b_full, b_empty, t_full, t_empty, sc_full, drain, total;
  __host__ __device__ Bars(int NS, int ZB, int NB) {
    s_full = 0;
    s_empty = s_full + NS;
    z_full = s_empty + NS;
    z_empty = z_full + ZB;
    b_full = z_empty + ZB;
    b_empty = b_full + NB;
    t_full = b_empty + NB;
    t_empty = t_full + 2;
    sc_full = t_empty + 2;
    drain = sc_full + kScaleRing;
    total = drain + 1;
  }
};

__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          int* err) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort, err, kErrTimeout);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// Wait that ignores the abort flag (used to drain copies in flight).
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, int* err) {
  volatile int never = 0;
  mbar_wait(bar, parity, &never, err, kErrTimeout);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a -> low half
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

// ----------------------------------------------------------------- roles
template <int PREC>
__device__ void role_wave_producer(const TcParams& p, uint32_t sbase, const Bars& B,
                                   volatile int* abort) {
  const uint64_t pol = policy_evict_first();
  int g = 0;
  bool ok = true;
  for (int tile = blockIdx.x; ok && tile < p.n_tiles; tile += gridDim.x) {
    const TileDesc td = p.tiles[tile];
    const long long span = (long long)p.zrows * p.H;
    const long long avail = min(((long long)td.n_samples + 3) & ~3ll, span);
    for (int c = 0; c < p.NCHUNK; ++c, ++g) {
      const int slot = g % p.NS;
      const uint32_t full = sbase + p.off_bar + 8 * (B.s_full + slot);
      const uint32_t empty = sbase + p.off_bar + 8 * (B.s_empty + slot);
      if (!mbar_wait(empty, ((g / p.NS) & 1) ^ 1, abort, p.err, kErrTimeout)) {
        ok = false;
        break;
      }
      const long long f0 = (long long)c * p.CH * p.H;
      const long long nf = max(0ll, min((long long)p.CH * p.H, avail - f0));
      if (nf > 0) {
        mbar_arrive_expect_tx(full, (uint32_t)(nf * 4));
        bulk_g2s_hint(sbase + p.off_st + slot * p.st_bytes, p.wave + td.in_off + f0,
                      (uint32_t)(nf * 4), full, pol);
      } else {
        mbar_arrive(full);
      }
    }
  }
  // drain: every issued copy has landed before the CTA can exit
  for (int k = max(0, g - p.NS); k < g; ++k)
    drain_wait(sbase + p.off_bar + 8 * (B.s_full + k % p.NS), (k / p.NS) & 1, p.err);
}

__device__ void role_basis_producer(const TcParams& p, uint32_t sbase, const Bars& B,
                                    volatile int* abort) {
  const uint64_t pol = policy_evict_last();
  if (p.b_resident) {
    // every K-step block once, each to its own slot; consumers never release them
    for (int s = 0; s < p.KS; ++s) {
      const uint32_t full = sbase + p.off_bar + 8 * (B.b_full + s);
      mbar_arrive_expect_tx(full, p.bslot_bytes);
      bulk_g2s_hint(sbase + p.off_b + s * p.bslot_bytes, p.bimg + (size_t)s * p.bslot_bytes,
                    p.bslot_bytes, full, pol);
    }
    for (int s = 0; s < p.KS; ++s) drain_wait(sbase + p.off_bar + 8 * (B.b_full + s), 0, p.err);
    return;
  }
  int g = 0;
  bool ok = true;
  for (int tile = blockIdx.x; ok && tile < p.n_tiles; tile += gridDim.x) {
    for (int s = 0; s < p.KS; ++s, ++g) {
      const int slot = g % p.NB;
      const uint32_t full = sbase + p.off_bar + 8 * (B.b_full + slot);
      const uint32_t empty = sbase + p.off_bar + 8 * (B.b_empty + slot);
      if (!mbar_wait(empty, ((g / p.NB) & 1) ^ 1, abort, p.err, kErrTimeout)) {
        ok = false;
        break;
      }
      mbar_arrive_expect_tx(full, p.bslot_bytes);
      bulk_g2s_hint(sbase + p.off_b + slot * p.bslot_bytes, p.bimg + (size_t)s * p.bslot_bytes,
                    p.bslot_bytes, full, pol);
    }
  }
  for (int k = max(0, g - p.NB); k < g; ++k)
    drain_wait(sbase + p.off_bar + 8 * (B.b_full + k % p.NB), (k / p.NB) & 1, p.err);
}

template <int PREC>
__device__ void role_mma(const TcParams& p, uint32_t sbase, const Bars& B, uint32_t tmem_base,
                         volatile int* abort) {
  int g = 0;
  int k = 0;
  const uint32_t lbo_b = (uint32_t)p.NC * 16;
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int zb = k % p.ZB;
    const int acc = k & 1;
    if (!mbar_wait(sbase + p.off_bar + 8 * (B.z_full + zb), (k / p.ZB) & 1, abort, p.err,
                   kErrTimeout))
      break;
    if (!mbar_wait(sbase + p.off_bar + 8 * (B.t_empty + acc), ((k >> 1) & 1) ^ 1, abort, p.err,
                   kErrTimeout))
      break;
    tc_fence_after();
    const uint32_t d = tmem_base + acc * p.acc_stride;
    const uint32_t a0 = sbase + p.off_a + zb * p.abuf_bytes;
    bool ok = true;
    int s = 0;
    if constexpr (PREC == MELT_FP8E4M3) {
      for (int ks = 0; ks < p.KS; ++ks, ++g, ++s) {
        const int slot = p.b_resident ? ks : g % p.NB;
        const uint32_t par = p.b_resident ? 0u : (uint32_t)((g / p.NB) & 1);
        if (!mbar_wait(sbase + p.off_bar + 8 * (B.b_full + slot), par, abort, p.err,
                       kErrTimeout)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = sdesc_noswz(a0 + 2u * ks * p.lbo_a, p.lbo_a, 128);
        const uint64_t bd = sdesc_noswz(sbase + p.off_b + slot * p.bslot_bytes, lbo_b, 128);
        mma_f8(d, ad, bd, p.idesc, s > 0);
        if (!p.b_resident) mma_commit(sbase + p.off_bar + 8 * (B.b_empty + slot));
      }
    } else {
      for (int j = 0; ok && j < p.J; ++j) {
        const int kj = min(p.H, p.N - j * p.H);
        const int steps = (kj + 15) / 16;
        for (int kk = 0; kk < steps; ++kk, ++g, ++s) {
          const int slot = p.b_resident ? s : g % p.NB;
          const uint32_t par = p.b_resident ? 0u : (uint32_t)((g / p.NB) & 1);
          if (!mbar_wait(sbase + p.off_bar + 8 * (B.b_full + slot), par, abort, p.err,
                         kErrTimeout)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aoff = 2u * kk * p.lbo_a + 16u * j;
          const uint32_t bslot = sbase + p.off_b + slot * p.bslot_bytes;
          const uint64_t ad = sdesc_noswz(a0 + aoff, p.lbo_a, 128);
          const uint64_t bd = sdesc_noswz(bslot, lbo_b, 128);
          mma_f16(d, ad, bd, p.idesc, s > 0);
          if constexpr (PREC == MELT_BF16X3) {
            const uint64_t bd_lo = sdesc_noswz(bslot + p.kstep_bytes, lbo_b, 128);
            const uint64_t ad_lo = sdesc_noswz(a0 + p.a_bytes + aoff, p.lbo_a, 128);
            mma_f16(d, ad, bd_lo, p.idesc, 1);
            mma_f16(d, ad_lo, bd, p.idesc, 1);
          }
          if (!p.b_resident) mma_commit(sbase + p.off_bar + 8 * (B.b_empty + slot));
        }
      }
    }
    if (!ok) break;
    mma_commit(sbase + p.off_bar + 8 * (B.z_empty + zb));
    mma_commit(sbase + p.off_bar + 8 * (B.t_full + acc));
  }
  // no MMA may still be running when TMEM is released
  mma_commit(sbase + p.off_bar + 8 * B.drain);
  drain_wait(sbase + p.off_bar + 8 * B.drain, 0, p.err);
}

// BF16 / BF16X3 converter: FP32 span chunks -> Z rows (bf16 hi [, lo]).
template <int PREC>
__device__ void role_convert_poly(const TcParams& p, uint8_t* gbase, uint32_t sbase,
                                  const Bars& B, volatile int* abort) {
  const int ct = threadIdx.x - 32 * kCvtWarp0;
  const int H8 = p.H >> 3;
  int g = 0;
  int k = 0;
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int zb = k % p.ZB;
    if (!warp_wait(sbase + p.off_bar + 8 * (B.z_empty + zb), ((k / p.ZB) & 1) ^ 1, abort, p.err))
      break;
    const int nsamp = p.tiles[tile].n_samples;
    const uint32_t zhi = sbase + p.off_a + zb * p.abuf_bytes;
    bool ok = true;
    for (int c = 0; c < p.NCHUNK; ++c, ++g) {
      const int slot = g % p.NS;
      if (!warp_wait(sbase + p.off_bar + 8 * (B.s_full + slot), (g / p.NS) & 1, abort, p.err)) {
        ok = false;
        break;
      }
      const float* st = reinterpret_cast<const float*>(gbase + p.off_st + slot * p.st_bytes);
      const int rows = min(p.CH, p.zrows - c * p.CH);
      // item it = ul * H8 + kc; walk it = ct, ct + 128, ... without dividing in the loop
      int ul = ct / H8, kc = ct - (ct / H8) * H8;
      const int dul = kCvtThreads / H8, dkc = kCvtThreads - dul * H8;
      for (; ul < rows; ul += dul, kc += dkc) {
        if (kc >= H8) {
          kc -= H8;
          ++ul;
          if (ul >= rows) break;
        }
        const int u = c * p.CH + ul;
        const float4 a = *reinterpret_cast<const float4*>(st + ul * p.H + kc * 8);
        const float4 b = *reinterpret_cast<const float4*>(st + ul * p.H + kc * 8 + 4);
        float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const int s0 = u * p.H + kc * 8;
        if (s0 + 8 > nsamp) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (s0 + e >= nsamp) x[e] = 0.f;
        }
        uint4 hv;
        hv.x = pack_bf16(x[0], x[1]);
        hv.y = pack_bf16(x[2], x[3]);
        hv.z = pack_bf16(x[4], x[5]);
        hv.w = pack_bf16(x[6], x[7]);
        const uint32_t zoff = kc * p.lbo_a + u * 16;
        sts128(zhi + zoff, hv);
        if constexpr (PREC == MELT_BF16X3) {
          const uint32_t h[4] = {hv.x, hv.y, hv.z, hv.w};
          float r[8];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            r[2 * e] = x[2 * e] - __uint_as_float(h[e] << 16);
            r[2 * e + 1] = x[2 * e + 1] - __uint_as_float(h[e] & 0xffff0000u);
          }
          uint4 lv;
          lv.x = pack_bf16(r[0], r[1]);
          lv.y = pack_bf16(r[2], r[3]);
          lv.z = pack_bf16(r[4], r[5]);
          lv.w = pack_bf16(r[6], r[7]);
          sts128(zhi + p.a_bytes + zoff, lv);
        }
      }
      mbar_arrive(sbase + p.off_bar + 8 * (B.s_empty + slot));
    }
    if (!ok) break;
    fence_proxy_async();
    mbar_arrive(sbase + p.off_bar + 8 * (B.z_full + zb));
  }
}

// FP8 converter: whole span staged; per-frame amax scale; frame rows (im2col in smem).
__device__ void role_convert_fp8(const TcParams& p, uint8_t* gbase, uint32_t sbase,
                                 const Bars& B, volatile int* abort) {
  const int ct = threadIdx.x - 32 * kCvtWarp0;
  const int cw = ct >> 5, lane = threadIdx.x & 31;
  const int KL = p.N - (p.J - 1) * p.H;  // samples of the last slice of a frame
  const int G = (p.KS * 32) / 16;        // 16-byte groups per frame row
  float* rowmax = reinterpret_cast<float*>(gbase + p.off_rowmax);
  float* rowpre = rowmax + p.zrows;
  float* inv_s = rowpre + p.zrows;
  float* scales = reinterpret_cast<float*>(gbase + p.off_scale);
  const float* span = reinterpret_cast<const float*>(gbase + p.off_st);
  int g = 0;
  int k = 0;
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int zb = k % p.ZB;
    bool ok = warp_wait(sbase + p.off_bar + 8 * (B.z_empty + zb), ((k / p.ZB) & 1) ^ 1, abort, p.err);
    for (int c = 0; ok && c < p.NCHUNK; ++c)
      ok = warp_wait(sbase + p.off_bar + 8 * (B.s_full + c), ((g + c) / p.NS) & 1, abort, p.err);
    // all four converter warps take the same decision before any named barrier
    if (!named_barrier_and(1, kCvtThreads, ok)) break;
    const int nsamp = p.tiles[tile].n_samples;
    // 1. per Z row: max |x| over the row and over its first KL samples
    for (int u = cw; u < p.zrows; u += kCvtWarps) {
      float mf = 0.f, mp = 0.f;
      for (int r = lane; r < p.H; r += 32) {
        const int s = u * p.H + r;
        const float v = s < nsamp ? fabsf(span[s]) : 0.f;
        mf = fmaxf(mf, v);
        if (r < KL) mp = fmaxf(mp, v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
        mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, o));
      }
      if (lane == 0) {
        rowmax[u] = mf;
        rowpre[u] = mp;
      }
    }
    named_barrier(1, kCvtThreads);
    // 2. frame scale: s_t = amax/448, quantiser multiplier 448/amax (1 for silent frames)
    {
      const int f = ct;  // kCvtThreads == kF
      float amax = rowpre[f + p.J - 1];
      for (int j = 0; j < p.J - 1; ++j) amax = fmaxf(amax, rowmax[f + j]);
      const bool pos = amax > 0.f;
      inv_s[f] = pos ? 448.f / amax : 1.f;
      const float st = pos ? amax / 448.f : 1.f;
      scales[(k % kScaleRing) * kF + f] = st / 448.f;
    }
    named_barrier(1, kCvtThreads);
    // 3. quantised frame rows, K-major canonical layout (16-byte core rows)
    const uint32_t abase = sbase + p.off_a + zb * p.abuf_bytes;
    for (int it = ct; it < kF * G; it += kCvtThreads) {
      const int f = it / G;
      const int gq = it - f * G;
      const float inv = inv_s[f];
      const int n0 = gq * 16;
      float x[16];
#pragma unroll
      for (int e = 0; e < 16; e += 4) {
        const int n = n0 + e;
        const int s = f * p.H + n;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n + 3 < p.N && s + 3 < nsamp) {
          v = *reinterpret_cast<const float4*>(span + s);
        } else {
          float t[4] = {0.f, 0.f, 0.f, 0.f};
          for (int q = 0; q < 4; ++q)
            if (n + q < p.N && s + q < nsamp) t[q] = span[s + q];
          v = make_float4(t[0], t[1], t[2], t[3]);
        }
        x[e] = v.x * inv;
        x[e + 1] = v.y * inv;
        x[e + 2] = v.z * inv;
        x[e + 3] = v.w * inv;
      }
      uint4 q;
      q.x = pack_e4m3x4(x[0], x[1], x[2], x[3]);
      q.y = pack_e4m3x4(x[4], x[5], x[6], x[7]);
      q.z = pack_e4m3x4(x[8], x[9], x[10], x[11]);
      q.w = pack_e4m3x4(x[12], x[13], x[14], x[15]);
      sts128(abase + gq * p.lbo_a + f * 16, q);
    }
    fence_proxy_async();
    mbar_arrive(sbase + p.off_bar + 8 * (B.z_full + zb));
    mbar_arrive(sbase + p.off_bar + 8 * (B.sc_full + (k % kScaleRing)));
    for (int c = 0; c < p.NCHUNK; ++c) mbar_arrive(sbase + p.off_bar + 8 * (B.s_empty + c));
    g += p.NCHUNK;
  }
}

template <int PREC, int NCH>
__device__ void role_epilogue(const TcParams& p, uint8_t* gbase, uint32_t sbase, const Bars& B,
                              uint32_t tmem_base, volatile int* abort) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * warp + lane;
  const float* scales = reinterpret_cast<const float*>(gbase + p.off_scale);
  const bool vec = (p.n_out & 3) == 0;
  int k = 0;
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int acc = k & 1;
    if (!warp_wait(sbase + p.off_bar + 8 * (B.t_full + acc), (k >> 1) & 1, abort, p.err)) break;
    float sc = 1.f;
    if constexpr (PREC == MELT_FP8E4M3) {
      if (!warp_wait(sbase + p.off_bar + 8 * (B.sc_full + (k % kScaleRing)), (k / kScaleRing) & 1,
                     abort, p.err))
        break;
      sc = scales[(k % kScaleRing) * kF + row];
    }
    tc_fence_after();
    const TileDesc td = p.tiles[tile];
    const bool valid = row < td.n_frames;
    const uint32_t t0 = tmem_base + ((uint32_t)(32 * warp) << 16) + acc * p.acc_stride;
    float* orow = p.out + (size_t)(td.out_row + row) * p.n_out;
    if (p.n_mfcc == 0) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        float re[16], im[16], v[16];
        tmem_ld16(t0 + 16 * c, re);
        tmem_ld16(t0 + 16 * NCH + 16 * c, im);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float r = re[e] * sc, i = im[e] * sc;
          v[e] = __logf(fmaf(r, r, i * i) + p.eps);
        }
        if (valid) {
          if (vec && 16 * c + 16 <= p.M) {
            float4* o4 = reinterpret_cast<float4*>(orow + 16 * c);
#pragma unroll
            for (int e = 0; e < 4; ++e)
              o4[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (16 * c + e < p.M) orow[16 * c + e] = v[e];
          }
        }
      }
    } else {
      float lm[16 * NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        float re[16], im[16];
        tmem_ld16(t0 + 16 * c, re);
        tmem_ld16(t0 + 16 * NCH + 16 * c, im);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float r = re[e] * sc, i = im[e] * sc;
          lm[16 * c + e] = __logf(fmaf(r, r, i * i) + p.eps);
        }
      }
      if (valid) {
        for (int kk = 0; kk < p.n_mfcc; ++kk) {
          const float* drow = p.dct + (size_t)kk * p.M;
          float a = 0.f;
#pragma unroll
          for (int m = 0; m < 16 * NCH; ++m)
            if (m < p.M) a = fmaf(lm[m], __ldg(drow + m), a);
          orow[kk] = a;
        }
      }
    }
    tc_fence_before();
    mbar_arrive(sbase + p.off_bar + 8 * (B.t_empty + acc));
  }
}

template <int PREC, int NCH>
__global__ void __launch_bounds__(kThreads, 1) melt_tc_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 127u) & ~127u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Bars B(p.NS, p.ZB, p.NB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + p.off_misc);
  volatile int* abort = reinterpret_cast<volatile int*>(gbase + p.off_misc + 4);

  if (threadIdx.x == 0) {
    auto bar = [&](int i) { return sbase + p.off_bar + 8 * i; };
    for (int i = 0; i < p.NS; ++i) {
      mbar_init(bar(B.s_full + i), 1);
      mbar_init(bar(B.s_empty + i), kCvtThreads);
    }
    for (int i = 0; i < p.ZB; ++i) {
      mbar_init(bar(B.z_full + i), kCvtThreads);
      mbar_init(bar(B.z_empty + i), 1);
    }
    for (int i = 0; i < p.NB; ++i) {
      mbar_init(bar(B.b_full + i), 1);
      mbar_init(bar(B.b_empty + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(B.t_full + i), 1);
      mbar_init(bar(B.t_empty + i), kEpiThreads);
    }
    for (int i = 0; i < kScaleRing; ++i) mbar_init(bar(B.sc_full + i), kCvtThreads);
    mbar_init(bar(B.drain), 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(tmem_slot), p.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kProdWarp) {
    if (lane == 0) role_wave_producer<PREC>(p, sbase, B, abort);
    __syncwarp();
  } else if (warp == kBWarp) {
    if (lane == 0) role_basis_producer(p, sbase, B, abort);
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0) role_mma<PREC>(p, sbase, B, tmem_base, abort);
    __syncwarp();
  } else if (warp >= kCvtWarp0) {
    if constexpr (PREC == MELT_FP8E4M3)
      role_convert_fp8(p, gbase, sbase, B, abort);
    else
      role_convert_poly<PREC>(p, gbase, sbase, B, abort);
    __syncwarp();
  } else {
    role_epilogue<PREC, NCH>(p, gbase, sbase, B, tmem_base, abort);
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem_base, p.tmem_cols);
  }
}

// ------------------------------------------------------------ host side
using KernelFn = void (*)(TcParams);

template <int PREC>
KernelFn pick_kernel(int nch) {
  switch (nch) {
    case 1: return melt_tc_kernel<PREC, 1>;
    case 2: return melt_tc_kernel<PREC, 2>;
    case 3: return melt_tc_kernel<PREC, 3>;
    case 4: return melt_tc_kernel<PREC, 4>;
    case 5: return melt_tc_kernel<PREC, 5>;
    case 6: return melt_tc_kernel<PREC, 6>;
    case 7: return melt_tc_kernel<PREC, 7>;
    case 8: return melt_tc_kernel<PREC, 8>;
    default: return nullptr;
  }
}

KernelFn kernel_for(int prec, int nch) {
  switch (prec) {
    case MELT_BF16: return pick_kernel<MELT_BF16>(nch);
    case MELT_BF16X3: return pick_kernel<MELT_BF16X3>(nch);
    case MELT_FP8E4M3: return pick_kernel<MELT_FP8E4M3>(nch);
    default: return nullptr;
  }
}

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

bool plan_smem(const TcBasis* tb, TcParams& p);

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
    if (!plan_smem(tb, probe)) return MELT_ERR_UNSUPPORTED;  // operands do not fit shared memory
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

namespace {

constexpr uint32_t kSmemLimit = 227 * 1024;

uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// Shared-memory plan for one basis; false if it cannot fit.
bool plan_smem(const TcBasis* tb, TcParams& p) {
  const int P = tb->precision;
  p.N = tb->n_fft;
  p.H = tb->hop;
  p.M = tb->n_mels;
  p.MP = (p.M + 15) / 16 * 16;
  p.NC = 2 * p.MP;
  p.J = tb->J;
  p.KS = tb->ksteps;
  p.zrows = kF + p.J - 1;
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
  // staging chunks of ~12 KB of Z rows
  const uint32_t row_bytes = (uint32_t)p.H * 4;
  const uint32_t span_bytes = row_bytes * p.zrows;
  p.NCHUNK = (int)((span_bytes + 12287) / 12288);
  p.CH = (p.zrows + p.NCHUNK - 1) / p.NCHUNK;
  p.NCHUNK = (p.zrows + p.CH - 1) / p.CH;
  p.st_bytes = row_bytes * p.CH;  // slots back to back: the FP8 form reads the span contiguously
  // Layout candidates, best first: the whole basis resident in shared memory
  // (loaded once per CTA) with two then one A buffers, else a streamed basis ring.
  struct Cand { int resident, zb, nb, ns; };
  std::vector<Cand> cands;
  for (int zb = 2; zb >= 1; --zb)
    for (int ns = 4; ns >= 3; --ns) cands.push_back({1, zb, p.KS, ns});
  for (int zb = 2; zb >= 1; --zb)
    for (int nb = 8; nb >= 2; --nb)
      for (int ns = 4; ns >= 2; --ns) cands.push_back({0, zb, nb, ns});
  for (const Cand& c : cands) {
    p.b_resident = c.resident;
    p.ZB = c.zb;
    p.NB = c.nb;
    p.NS = (P == MELT_FP8E4M3) ? p.NCHUNK : c.ns;  // FP8 stages the whole span
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
    p.off_misc = off;
    off += 128;
    p.off_scale = off;
    off += (P == MELT_FP8E4M3) ? kScaleRing * kF * 4 : 0;
    p.off_rowmax = off;
    off += (P == MELT_FP8E4M3) ? align_up((2 * p.zrows + kF) * 4, 128) : 0;
    if (off + 128 <= kSmemLimit) {
      p.smem_total = off + 128;
      p.tmem_cols = p.NC <= 32 ? 64 : p.NC <= 64 ? 128 : p.NC <= 128 ? 256 : 512;
      p.acc_stride = p.tmem_cols / 2;
      p.idesc = idesc_f32acc(P == MELT_FP8E4M3 ? 0u : 1u, kF, p.NC);
      return true;
    }
  }
  return false;
}

}  // namespace

cudaError_t tc_launch(const TcBasis* tb, const TcLaunch& L, cudaStream_t stream) {
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  if (!plan_smem(tb, p)) return cudaErrorInvalidConfiguration;
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
  KernelFn fn = kernel_for(tb->precision, p.MP / 16);
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
