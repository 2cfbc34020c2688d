// Device side of the tensor-core MelT kernels (included by the two
// instantiation units melt_tc_plain.cu and melt_tc_mfcc.cu).
#pragma once
// Tensor-core MelT kernels for sm_103a: BF16, split-BF16 (three products)
// and FP8 e4m3 forms of the projection of Sec. III-A (Eq. 6), with power
// (Eq. 7), log (Eq. 8) and the optional DCT-II (Eq. 9) fused in the epilogue.
//
// One persistent CTA per SM walks a static round-robin list of tiles
// (128 consecutive frames of one clip).  Warp roles (11 warps):
//   warps 0-3   epilogue: TMEM -> registers, R^2 + I^2, log, (DCT), store
//   warp  4     TMEM allocator + single-thread tcgen05.mma issuer
//   warp  5     basis producer: bulk async copies (TMA engine) of the basis
//               K-step blocks, once per CTA when the basis fits in shared
//               memory, else streamed through a ring
//   warp  6     waveform producer: bulk async copies of the tile's FP32
//               sample span in chunks of ~16 KB into a ring
//   warps 7-10  converters: staged FP32 samples -> MMA A operand in shared memory
//
// Implicit framing (no im2col in HBM).  Frames overlap (N > H), so the A
// operand's rows would be H samples apart, which a UMMA shared-memory
// descriptor cannot express.  The BF16 forms use a polyphase split of the
// frame: with n = jH + r (0 <= r < H, j < J = ceil(N/H)) and
// Z[u][r] = x[(t0+u)H + r],
//     [R|I][t] = sum_j Z[t+j][:] . B_j^T,   B_j[c][r] = W[c][jH + r]
// so each sample is loaded and converted once into Z (rows of H samples,
// K-major canonical layout with rows 16 B apart) and the j-shift is a
// 16-byte offset of the A descriptor's start address.  The J slices
// accumulate into the same TMEM tile.  Keeping HBM busy takes >= 16 KB bulk
// copies and >= ~48 KB in flight per SM, so the span is staged by the TMA
// engine; when the basis is resident the tile has one Z buffer (conversion
// and MMA of a tile then run back to back, both well inside the tile's HBM
// time).
// FP8 needs a per-frame scale, which differs between the frames that share
// a Z row, so the FP8 form stages the tile's span with bulk copies and
// writes each frame row (im2col inside shared memory only), scaled by
// 448/amax(frame).
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
namespace tc {

using namespace ptx;

constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kBWarp = 5;
constexpr int kProdWarp = 6;
constexpr int kCvtWarp0 = 7;
constexpr int kCvtWarps = 4;
constexpr int kThreads = 32 * (kCvtWarp0 + kCvtWarps);  // 352
constexpr int kCvtThreads = 32 * kCvtWarps;             // 128
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kF = kTileFrames;  // 128 = UMMA M
constexpr int kScaleRing = 4;    // FP8 per-frame scale buffers in flight
constexpr int kQuadsPerThread = 8;  // float4s per converter thread per staged chunk (<= 16 KB)
constexpr int kEarlyChunks = 5;  // log-Mel rows of up to 80 values are held in registers
constexpr int kMaxMfccTc = 128;  // DCT outputs of the tensor-core epilogue (matrix in shared memory)

struct TcParams {
  const float* wave;
  const TileDesc* tiles;
  int n_tiles;
  const uint8_t* bimg;   // KS blocks of step_bytes
  const float* dct;      // [n_mfcc][M] or null
  float* out;
  int* err;
  float eps;
  int N, H, M, MP, NC, J, KS;
  int zrows;             // Z rows: 128 + J - 1
  int items;             // BF16 forms: 8-sample items per tile (zrows * H / 8)
  float inv_h8;          // 1 / (H / 8)
  int n_out, n_mfcc;
  uint32_t kstep_bytes;  // one B part of one K-step
  uint32_t step_bytes;   // one K-step of the basis (BF16X3: hi + lo parts)
  uint32_t bslot_bytes;  // one basis slot: kps K-steps (resident: one K-step)
  int kps;               // K-steps per streamed basis slot
  uint32_t lbo_a;        // A operand: bytes between K-adjacent core matrices
  uint32_t a_bytes;      // one A part
  uint32_t abuf_bytes;   // one A buffer (BF16X3: hi + lo parts)
  int ZB;                // A buffers
  int NS, CH, NCHUNK;    // FP8: staging slots, Z rows per chunk, chunks per tile
  uint32_t st_bytes;     // FP8: bytes per staging slot
  int NB;                // basis slots (resident: NB == KS)
  int b_resident;        // 1: the whole basis stays in shared memory for the CTA's life
  uint32_t tmem_cols, acc_stride, idesc;
  uint32_t desc_hi;      // high word of every operand descriptor (SBO = 128 B, version)
  uint32_t off_a, off_st, off_b, off_bar, off_misc, off_scale, off_rowmax, off_tab, off_dct;
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

static __device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          int* err) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort, err, kErrTimeout);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// One arrival per warp: the warp's threads finish their own work (and any
// proxy fence) first; lane 0 then arrives on behalf of the warp.  Barriers
// that warps arrive on are initialised with the number of arriving warps.
static __device__ __forceinline__ void warp_arrive(uint32_t bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// Wait that ignores the abort flag (used to drain copies in flight).
static __device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, int* err) {
  volatile int never = 0;
  mbar_wait(bar, parity, &never, err, kErrTimeout);
}

static __device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a -> low half
  return *reinterpret_cast<uint32_t*>(&h);
}

static __device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

// 32-byte store: one full sector per thread (address 32-byte aligned).
static __device__ __forceinline__ void stg256(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}

static __device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

// Streaming read of 4 samples: read once, keep out of L1.
static __device__ __forceinline__ float4 ldg_stream(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// ----------------------------------------------------------------- roles
static __device__ void role_wave_producer(const TcParams& p, uint32_t sbase, const Bars& B,
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

static __device__ void role_basis_producer(const TcParams& p, uint32_t sbase, const Bars& B,
                                    volatile int* abort) {
  const uint64_t pol = policy_evict_last();
  if (p.b_resident) {
    // every K-step block once, each to its own slot; consumers never release them
    for (int s = 0; s < p.KS; ++s) {
      const uint32_t full = sbase + p.off_bar + 8 * (B.b_full + s);
      mbar_arrive_expect_tx(full, p.step_bytes);
      bulk_g2s_hint(sbase + p.off_b + s * p.step_bytes, p.bimg + (size_t)s * p.step_bytes,
                    p.step_bytes, full, pol);
    }
    for (int s = 0; s < p.KS; ++s) drain_wait(sbase + p.off_bar + 8 * (B.b_full + s), 0, p.err);
    return;
  }
  // streamed: slots of kps consecutive K-steps (contiguous in the basis image)
  int slot = 0;
  uint32_t phase = 0;
  int issued = 0;
  bool ok = true;
  for (int tile = blockIdx.x; ok && tile < p.n_tiles; tile += gridDim.x) {
    for (int s0 = 0; s0 < p.KS; s0 += p.kps) {
      const uint32_t full = sbase + p.off_bar + 8 * (B.b_full + slot);
      const uint32_t empty = sbase + p.off_bar + 8 * (B.b_empty + slot);
      if (!mbar_wait(empty, phase ^ 1, abort, p.err, kErrTimeout)) {
        ok = false;
        break;
      }
      const uint32_t bytes = (uint32_t)min(p.kps, p.KS - s0) * p.step_bytes;
      mbar_arrive_expect_tx(full, bytes);
      bulk_g2s_hint(sbase + p.off_b + slot * p.bslot_bytes, p.bimg + (size_t)s0 * p.step_bytes,
                    bytes, full, pol);
      ++issued;
      if (++slot == p.NB) {
        slot = 0;
        phase ^= 1;
      }
    }
  }
  for (int k = max(0, issued - p.NB); k < issued; ++k)
    drain_wait(sbase + p.off_bar + 8 * (B.b_full + k % p.NB), (k / p.NB) & 1, p.err);
}

template <int PREC>
__device__ void role_mma(const TcParams& p, uint8_t* gbase, uint32_t sbase, const Bars& B,
                         uint32_t tmem_base, volatile int* abort) {
  // per K-step: x = A start offset / 16 within a buffer, y = B descriptor low word (resident)
  const uint2* tab = reinterpret_cast<const uint2*>(gbase + p.off_tab);
  const uint64_t hi = (uint64_t)p.desc_hi << 32;
  const uint32_t a_lo0 = ((sbase + p.off_a) >> 4) | ((p.lbo_a >> 4) << 16);
  const uint32_t b_lo0 = ((sbase + p.off_b) >> 4) | (((uint32_t)p.NC * 16 >> 4) << 16);
  const uint32_t abuf16 = p.abuf_bytes >> 4, apart16 = p.a_bytes >> 4;
  const uint32_t bslot16 = p.bslot_bytes >> 4, bpart16 = p.kstep_bytes >> 4;
  int bslot = 0;
  uint32_t bphase = 0;
  int k = 0;
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int zb = p.ZB == 2 ? (k & 1) : 0;
    const int acc = k & 1;
    if (!mbar_wait(sbase + p.off_bar + 8 * (B.z_full + zb), (p.ZB == 2 ? (k >> 1) : k) & 1,
                   abort, p.err, kErrTimeout))
      break;
    if (!mbar_wait(sbase + p.off_bar + 8 * (B.t_empty + acc), ((k >> 1) & 1) ^ 1, abort, p.err,
                   kErrTimeout))
      break;
    bool ok = true;
    if (p.b_resident && k == 0)
      for (int s = 0; ok && s < p.KS; ++s)
        ok = mbar_wait(sbase + p.off_bar + 8 * (B.b_full + s), 0, abort, p.err, kErrTimeout);
    if (!ok) break;
    tc_fence_after();
    const uint32_t d = tmem_base + acc * p.acc_stride;
    const uint32_t alo = a_lo0 + zb * abuf16;
    if (p.b_resident) {
      // descriptors from the K-step table, eight at a time: the loads are issued
      // ahead of the MMAs so that the issue loop is not latency bound
      const uint32_t tab_s = smem_u32(tab);
#pragma unroll 1
      for (int s0 = 0; s0 < p.KS; s0 += 8) {
        uint32_t tx[8], ty[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                       : "=r"(tx[u]), "=r"(ty[u])
                       : "r"(tab_s + 8u * min(s0 + u, p.KS - 1)));
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int s = s0 + u;
          if (s < p.KS) {
            const uint64_t ad = hi | (alo + tx[u]);
            const uint64_t bd = hi | ty[u];
            if constexpr (PREC == MELT_FP8E4M3) {
              mma_f8(d, ad, bd, p.idesc, s > 0);
            } else {
              mma_f16(d, ad, bd, p.idesc, s > 0);
              if constexpr (PREC == MELT_BF16X3) {
                mma_f16(d, ad, hi | (ty[u] + bpart16), p.idesc, 1);
                mma_f16(d, hi | (alo + tx[u] + apart16), bd, p.idesc, 1);
              }
            }
          }
        }
      }
    } else {
      const uint32_t step16 = p.step_bytes >> 4;
      for (int s0 = 0; s0 < p.KS && ok; s0 += p.kps) {
        if (!mbar_wait(sbase + p.off_bar + 8 * (B.b_full + bslot), bphase, abort, p.err,
                       kErrTimeout)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t blo0 = b_lo0 + bslot * bslot16;
        const int n = min(p.kps, p.KS - s0);
        for (int u = 0; u < n; ++u) {
          const int s = s0 + u;
          const uint2 t = tab[s];
          const uint32_t blo = blo0 + u * step16;
          const uint64_t ad = hi | (alo + t.x);
          const uint64_t bd = hi | blo;
          if constexpr (PREC == MELT_FP8E4M3) {
            mma_f8(d, ad, bd, p.idesc, s > 0);
          } else {
            mma_f16(d, ad, bd, p.idesc, s > 0);
            if constexpr (PREC == MELT_BF16X3) {
              mma_f16(d, ad, hi | (blo + bpart16), p.idesc, 1);
              mma_f16(d, hi | (alo + t.x + apart16), bd, p.idesc, 1);
            }
          }
        }
        mma_commit(sbase + p.off_bar + 8 * (B.b_empty + bslot));
        if (++bslot == p.NB) {
          bslot = 0;
          bphase ^= 1;
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

// BF16 / BF16X3 converter: staged FP32 span chunks -> Z rows (bf16 hi [, lo]).
//
// Chunk c of a tile holds Z rows [c*CH, c*CH + rows) as contiguous FP32
// samples.  It is read as float4 "quads" (lanes read consecutive quads:
// conflict-free), and quad hq is the low or high half (hq & 1) of the Z row
// segment (row ul, 8-sample group kc) with 8 * (hq >> 1) = (ul - c*CH) H + 8 kc.
template <int PREC>
static __device__ void role_convert_staged(const TcParams& p, uint8_t* gbase, uint32_t sbase,
                                           const Bars& B, volatile int* abort) {
  const int ct = threadIdx.x - 32 * kCvtWarp0;
  const int H8 = p.H >> 3;
  // Every chunk has the same geometry (the last one may have fewer rows), so
  // this thread's quads and their Z offsets relative to the chunk's first row
  // are computed once.
  const int nq_full = p.CH * (p.H >> 2);
  uint32_t qoff[kQuadsPerThread];
  int qrow[kQuadsPerThread];
#pragma unroll
  for (int q = 0; q < kQuadsPerThread; ++q) {
    const int hq = ct + q * kCvtThreads;
    const int il = hq >> 1;
    const int ull = il / H8;
    const int kc = il - ull * H8;
    qrow[q] = hq < nq_full ? ull : 1 << 30;
    qoff[q] = kc * p.lbo_a + ull * 16 + (hq & 1) * 8;
  }
  const uint32_t st0 = sbase + p.off_st;
  int slot = 0;
  uint32_t sphase = 0;
  int k = 0;
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int zb = p.ZB == 2 ? (k & 1) : 0;
    if (!warp_wait(sbase + p.off_bar + 8 * (B.z_empty + zb), ((p.ZB == 2 ? (k >> 1) : k) & 1) ^ 1,
                   abort, p.err))
      break;
    const int nsamp = p.tiles[tile].n_samples;
    const uint32_t zaddr = sbase + p.off_a + zb * p.abuf_bytes;
    bool ok = true;
    for (int c = 0; c < p.NCHUNK; ++c) {
      if (!warp_wait(sbase + p.off_bar + 8 * (B.s_full + slot), sphase, abort, p.err)) {
        ok = false;
        break;
      }
      const int rows = min(p.CH, p.zrows - c * p.CH);
      const uint32_t st = st0 + slot * p.st_bytes;
      const int s_base = c * p.CH * p.H;
      const uint32_t zrow0 = zaddr + c * p.CH * 16;
      const bool tail = s_base + rows * p.H > nsamp;  // chunk reaches past the clip's end
      float4 x[kQuadsPerThread];
#pragma unroll
      for (int q = 0; q < kQuadsPerThread; ++q)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(x[q].x), "=f"(x[q].y), "=f"(x[q].z), "=f"(x[q].w)
                     : "r"(st + 16u * min(ct + q * kCvtThreads, nq_full - 1)));  // stay inside the slot
      if (tail) {
#pragma unroll
        for (int q = 0; q < kQuadsPerThread; ++q) {
          const int s0 = s_base + 4 * (ct + q * kCvtThreads);
          x[q].x = s0 < nsamp ? x[q].x : 0.f;
          x[q].y = s0 + 1 < nsamp ? x[q].y : 0.f;
          x[q].z = s0 + 2 < nsamp ? x[q].z : 0.f;
          x[q].w = s0 + 3 < nsamp ? x[q].w : 0.f;
        }
      }
      uint32_t hw[kQuadsPerThread][2];
#pragma unroll
      for (int q = 0; q < kQuadsPerThread; ++q) {
        hw[q][0] = pack_bf16(x[q].x, x[q].y);
        hw[q][1] = pack_bf16(x[q].z, x[q].w);
      }
#pragma unroll
      for (int q = 0; q < kQuadsPerThread; ++q)
        if (qrow[q] < rows)
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(zrow0 + qoff[q]), "r"(hw[q][0]),
                       "r"(hw[q][1]));
      if constexpr (PREC == MELT_BF16X3) {
#pragma unroll
        for (int q = 0; q < kQuadsPerThread; ++q) {
          const uint32_t l0 = pack_bf16(x[q].x - __uint_as_float(hw[q][0] << 16),
                                        x[q].y - __uint_as_float(hw[q][0] & 0xffff0000u));
          const uint32_t l1 = pack_bf16(x[q].z - __uint_as_float(hw[q][1] << 16),
                                        x[q].w - __uint_as_float(hw[q][1] & 0xffff0000u));
          if (qrow[q] < rows)
            asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(zrow0 + qoff[q] + p.a_bytes),
                         "r"(l0), "r"(l1));
        }
      }
      warp_arrive(sbase + p.off_bar + 8 * (B.s_empty + slot));
      if (++slot == p.NS) {
        slot = 0;
        sphase ^= 1;
      }
    }
    if (!ok) break;
    fence_proxy_async();
    warp_arrive(sbase + p.off_bar + 8 * (B.z_full + zb));
  }
}

// FP8 converter: whole span staged; per-frame amax scale; frame rows (im2col in smem).
static __device__ void role_convert_fp8(const TcParams& p, uint8_t* gbase, uint32_t sbase,
                                 const Bars& B, volatile int* abort) {
  const int ct = threadIdx.x - 32 * kCvtWarp0;
  const int cw = ct >> 5, lane = threadIdx.x & 31;
  const int KL = p.N - (p.J - 1) * p.H;  // samples of the last slice of a frame
  const int G = 2 * p.KS;                // 16-byte groups per frame row
  float* rowmax = reinterpret_cast<float*>(gbase + p.off_rowmax);
  float* rowpre = rowmax + p.zrows;
  float* inv_s = rowpre + p.zrows;
  float* scales = reinterpret_cast<float*>(gbase + p.off_scale);
  const float* span = reinterpret_cast<const float*>(gbase + p.off_st);
  int g = 0;
  int k = 0;
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int zb = p.ZB == 2 ? (k & 1) : 0;
    bool ok = warp_wait(sbase + p.off_bar + 8 * (B.z_empty + zb),
                        ((p.ZB == 2 ? (k >> 1) : k) & 1) ^ 1, abort, p.err);
    for (int c = 0; ok && c < p.NCHUNK; ++c)
      ok = warp_wait(sbase + p.off_bar + 8 * (B.s_full + c), ((g + c) / p.NS) & 1, abort, p.err);
    // all converter warps take the same decision before any named barrier
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
    if (ct < kF) {
      const int f = ct;
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
    warp_arrive(sbase + p.off_bar + 8 * (B.z_full + zb));
    warp_arrive(sbase + p.off_bar + 8 * (B.sc_full + (k % kScaleRing)));
    for (int c = 0; c < p.NCHUNK; ++c) warp_arrive(sbase + p.off_bar + 8 * (B.s_empty + c));
    g += p.NCHUNK;
  }
}

template <int PREC, int NCH, bool MFCC>
__device__ void role_epilogue(const TcParams& p, uint8_t* gbase, uint32_t sbase, const Bars& B,
                              uint32_t tmem_base, volatile int* abort) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * warp + lane;
  const float* scales = reinterpret_cast<const float*>(gbase + p.off_scale);
  const float* dct = reinterpret_cast<const float*>(gbase + p.off_dct);  // [n_mfcc][dct_ld]
  const bool vec8 = ((p.n_out & 7) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 31) == 0);
  const int nch = p.MP >> 4;
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
    if constexpr (!MFCC) {
      if (nch <= kEarlyChunks) {
        // every value of the row into registers, TMEM released before the stores
        float v[16 * kEarlyChunks];
#pragma unroll
        for (int c = 0; c < kEarlyChunks; ++c) {
          if (c < nch) {
            float re[16], im[16];
            tmem_ld16(t0 + 16 * c, re);
            tmem_ld16(t0 + p.MP + 16 * c, im);
            tmem_ld_wait(re, im);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float r = re[e] * sc, i = im[e] * sc;
              v[16 * c + e] = __logf(fmaf(r, r, fmaf(i, i, p.eps)));
            }
          }
        }
        tc_fence_before();
        warp_arrive(sbase + p.off_bar + 8 * (B.t_empty + acc));
        if (valid) {
#pragma unroll
          for (int c = 0; c < kEarlyChunks; ++c) {
            if (c < nch) {
              if (vec8 && 16 * c + 16 <= p.M) {
                stg256(orow + 16 * c, v + 16 * c);
                stg256(orow + 16 * c + 8, v + 16 * c + 8);
              } else {
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (16 * c + e < p.M) orow[16 * c + e] = v[16 * c + e];
              }
            }
          }
        }
        continue;
      }
      // longer rows: chunk by chunk, the next chunk's TMEM load overlapping this one's math
      float re[2][16], im[2][16];
      tmem_ld16(t0, re[0]);
      tmem_ld16(t0 + p.MP, im[0]);
      for (int c = 0; c < nch; c += 2) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int cc = c + half;
          if (cc >= nch) break;
          tmem_ld_wait(re[half], im[half]);
          if (cc + 1 < nch) {
            tmem_ld16(t0 + 16 * (cc + 1), re[half ^ 1]);
            tmem_ld16(t0 + p.MP + 16 * (cc + 1), im[half ^ 1]);
          }
          float v[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float r = re[half][e] * sc, i = im[half][e] * sc;
            v[e] = __logf(fmaf(r, r, fmaf(i, i, p.eps)));
          }
          if (valid) {
            if (vec8 && 16 * cc + 16 <= p.M) {
              stg256(orow + 16 * cc, v);
              stg256(orow + 16 * cc + 8, v + 8);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (16 * cc + e < p.M) orow[16 * cc + e] = v[e];
            }
          }
        }
      }
      tmem_ld_wait();
    } else {
      // MFCC: the frame's log-Mel row stays in registers; C[k] = sum_m lm[m] D[k][m]
      float lm[16 * NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        float re[16], im[16];
        tmem_ld16(t0 + 16 * c, re);
        tmem_ld16(t0 + 16 * NCH + 16 * c, im);
        tmem_ld_wait(re, im);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float r = re[e] * sc, i = im[e] * sc;
          lm[16 * c + e] = (16 * c + e < p.M) ? __logf(fmaf(r, r, i * i) + p.eps) : 0.f;
        }
      }
#pragma unroll 1
      for (int kk = 0; kk < p.n_mfcc; ++kk) {
        const float4* d4 = reinterpret_cast<const float4*>(dct + kk * 16 * NCH);
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int q = 0; q < 4 * NCH; ++q) {
          const float4 d = d4[q];  // zero past n_mels
          a0 = fmaf(lm[4 * q], d.x, a0);
          a1 = fmaf(lm[4 * q + 1], d.y, a1);
          a0 = fmaf(lm[4 * q + 2], d.z, a0);
          a1 = fmaf(lm[4 * q + 3], d.w, a1);
        }
        if (valid) orow[kk] = a0 + a1;
      }
    }
    tc_fence_before();
    warp_arrive(sbase + p.off_bar + 8 * (B.t_empty + acc));
  }
}

template <int PREC, int NCH, bool MFCC>
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
      mbar_init(bar(B.s_empty + i), kCvtWarps);
    }
    for (int i = 0; i < p.ZB; ++i) {
      mbar_init(bar(B.z_full + i), kCvtWarps);
      mbar_init(bar(B.z_empty + i), 1);
    }
    for (int i = 0; i < p.NB; ++i) {
      mbar_init(bar(B.b_full + i), 1);
      mbar_init(bar(B.b_empty + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(B.t_full + i), 1);
      mbar_init(bar(B.t_empty + i), kEpiWarps);
    }
    for (int i = 0; i < kScaleRing; ++i) mbar_init(bar(B.sc_full + i), kCvtWarps);
    mbar_init(bar(B.drain), 1);
    *abort = 0;
    fence_mbar_init();
  }
  // K-step descriptor table: A start offset (16-byte units) and resident B low word
  if (warp == kBWarp) {
    uint2* tab = reinterpret_cast<uint2*>(gbase + p.off_tab);
    const uint32_t b_lo0 = ((sbase + p.off_b) >> 4) | (((uint32_t)p.NC * 16 >> 4) << 16);
    const uint32_t bslot16 = p.step_bytes >> 4;
    if constexpr (PREC == MELT_FP8E4M3) {
      for (int s = lane; s < p.KS; s += 32)
        tab[s] = make_uint2((2u * s * p.lbo_a) >> 4, b_lo0 + s * bslot16);
    } else {
      // steps in (slice j, 16-column group kk) order, the order of the basis image
      for (int j = 0, s0 = 0; j < p.J; ++j) {
        const int steps = (min(p.H, p.N - j * p.H) + 15) / 16;
        for (int kk = lane; kk < steps; kk += 32)
          tab[s0 + kk] = make_uint2((2u * kk * p.lbo_a + 16u * j) >> 4, b_lo0 + (s0 + kk) * bslot16);
        s0 += steps;
      }
    }
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(tmem_slot), p.tmem_cols);
    tmem_relinquish();
  }
  if constexpr (MFCC) {
    // DCT-II rows padded with zeros to MP columns (16-byte aligned rows)
    if (warp < kEpiWarps) {
      float* dct = reinterpret_cast<float*>(gbase + p.off_dct);
      for (int i = threadIdx.x; i < p.n_mfcc * p.MP; i += kEpiThreads) {
        const int kk = i / p.MP, m = i - kk * p.MP;
        dct[i] = m < p.M ? p.dct[kk * p.M + m] : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kMmaWarp) {
    if (lane == 0) role_mma<PREC>(p, gbase, sbase, B, tmem_base, abort);
    __syncwarp();
  } else if (warp == kBWarp) {
    if (lane == 0) role_basis_producer(p, sbase, B, abort);
    __syncwarp();
  } else if (warp == kProdWarp) {
    if (lane == 0) role_wave_producer(p, sbase, B, abort);
    __syncwarp();
  } else if (warp >= kCvtWarp0) {
    if constexpr (PREC == MELT_FP8E4M3)
      role_convert_fp8(p, gbase, sbase, B, abort);
    else
      role_convert_staged<PREC>(p, gbase, sbase, B, abort);
    __syncwarp();
  } else {
    role_epilogue<PREC, NCH, MFCC>(p, gbase, sbase, B, tmem_base, abort);
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem_base, p.tmem_cols);
  }
}

using KernelFn = void (*)(TcParams);

template <int PREC, bool MFCC>
KernelFn pick_kernel(int nch) {
  if constexpr (!MFCC) {
    (void)nch;
    return melt_tc_kernel<PREC, 1, false>;  // log-Mel: chunk count taken at run time
  } else {
    switch (nch) {
      case 1: return melt_tc_kernel<PREC, 1, true>;
      case 2: return melt_tc_kernel<PREC, 2, true>;
      case 3: return melt_tc_kernel<PREC, 3, true>;
      case 4: return melt_tc_kernel<PREC, 4, true>;
      case 5: return melt_tc_kernel<PREC, 5, true>;
      case 6: return melt_tc_kernel<PREC, 6, true>;
      case 7: return melt_tc_kernel<PREC, 7, true>;
      case 8: return melt_tc_kernel<PREC, 8, true>;
      default: return nullptr;
    }
  }
}

// Defined in melt_tc_plain.cu (log-Mel) and melt_tc_mfcc.cu (MFCC epilogue).
KernelFn kernel_for_plain(int prec, int nch);
KernelFn kernel_for_mfcc(int prec, int nch);

}  // namespace tc
}  // namespace melt
