// Device side of the tensor-core MelT kernels (included by the two
// instantiation units melt_tc_plain.cu and melt_tc_mfcc.cu).
#pragma once
// Tensor-core MelT kernels for sm_103a: BF16 and split-BF16 (three products)
// forms of the projection of Sec. III-A (Eq. 6), with power (Eq. 7), log
// (Eq. 8) and the optional DCT-II (Eq. 9) fused in the epilogue.  (The FP8
// e4m3 form runs in the CTA-pair kernel of melt_tc2_kernel.cuh.)
//
// One persistent CTA per SM walks a static round-robin list of tiles
// (128 consecutive frames of one clip).  Warp roles (18 warps):
//   warps 0-3   epilogue: TMEM -> registers, R^2 + I^2, log, (DCT), store
//   warp  4     TMEM allocator + single-thread tcgen05.mma issuer
//   warp  5     basis producer: bulk async copies (TMA engine) of the basis
//               K-step blocks, once per CTA when the basis fits in shared
//               memory next to two A buffers, else streamed through a ring
//   warps 6-17  converters: waveform samples -> MMA A operand (BF16 Z rows) in shared memory
//
// Waveform path.  The converters read the tile's FP32 samples straight from
// global memory into registers (coalesced 16-byte loads) and write the BF16
// A operand (split-BF16: its hi and lo parts); one converter thread keeps the spans of the CTA's next
// tiles streaming into L2 with bulk prefetches, so those loads are L2 hits.
// No shared memory is spent on staging FP32 samples, which leaves room for a
// resident basis next to two A buffers (conversion of tile k+1 overlaps the
// MMAs of tile k, and the MMAs never wait for basis copies).
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
// accumulate into the same TMEM tile.
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
constexpr int kCvtWarp0 = 6;
constexpr int kCvtWarps = 12;
constexpr int kThreads = 32 * (kCvtWarp0 + kCvtWarps);  // 576
constexpr int kCvtThreads = 32 * kCvtWarps;             // 384
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kF = kTileFrames;  // 128 = UMMA M
constexpr int kSchedRing = 16;   // dynamic pair schedule: published pair indices in flight
constexpr int kSchedWords = 16;  // dynamic pair schedule: counters, one per launch in flight
constexpr int kQuadBatch = 8;    // float4 loads per converter thread per batch (two batches in flight)
constexpr int kEpiGroup = 2;     // 16-column chunks per TMEM wait in the epilogue
constexpr int kMaxMfccTc = 128;  // DCT outputs of the tensor-core epilogue (matrix in shared memory)
constexpr int kMaxPrefetch = 4;  // tiles whose spans may be prefetched into L2 ahead of use

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
  int nq;                // float4 quads of a tile's sample span: zrows * H / 4
  int pf;                // tiles prefetched into L2 ahead of the converters
  int n_out, n_mfcc;
  uint32_t kstep_bytes;  // one B part of one K-step
  uint32_t step_bytes;   // one K-step of the basis (BF16X3: hi + lo parts)
  uint32_t bslot_bytes;  // one basis slot: kps K-steps (resident: one K-step)
  int kps;               // K-steps per streamed basis slot
  uint32_t lbo_a;        // A operand: bytes between K-adjacent core matrices (8 rows x 16 B each)
  uint32_t a_bytes;      // one A part
  uint32_t abuf_bytes;   // one A buffer (BF16X3: hi + lo parts)
  int ZB;                // A buffers
  int NB;                // basis slots (resident: NB == KS)
  int b_resident;        // 1: the whole basis stays in shared memory for the CTA's life
  uint32_t tmem_cols, acc_stride, idesc;
  // More than 128 Mel bins (BF16 forms, streamed basis): the accumulator is
  // cut into nblk blocks of 128 bins (the last of wbl bins), each holding its
  // bins' R then I columns (N = 2 x 128, last 2 wbl); the basis image is
  // block-major, blk_step (blk_step_last) bytes per K-step of a block; a
  // tile's blocks alternate between the two accumulators.  nblk = 1 otherwise.
  int nblk, wbl;
  uint32_t idesc_last, blk_step, blk_step_last;
  // Fused STFT + Mel comparator (stft_bands > 0; the M analysis frequencies
  // are the DFT bins k sr / N): per bin k the filterbank entry {weight of band
  // b0, weight of band b0 + 1, b0 as int bits (-2: no band), 0}, copied to
  // shared memory at off_fb; the epilogue writes stft_bands values per frame.
  const float4* fb;
  int stft_bands;
  uint32_t off_fb;
  uint32_t desc_hi;      // high word of every operand descriptor (SBO = 128 B, version)
  // 1: the caller stated that no kernel still in flight on the stream writes
  // the waveform (MELT_FWD_INPUT_READY), so the roles that read it start
  // without waiting for the preceding kernel; the epilogue still waits
  int early_inputs;
  uint32_t off_a, off_b, off_bar, off_misc, off_tab, off_dct;
  uint32_t smem_total;   // dynamic shared memory bytes (incl. alignment slack)
  // CTA-pair kernel only: FP32 span staging ring and the half-basis layout
  int NS, CH, NCHUNK;    // staging slots, Z rows per chunk, chunks per tile
  uint32_t st_bytes;     // bytes per staging slot
  uint32_t off_st;
  uint32_t b_lbo;        // B operand: bytes between the two K core columns of a K-step block
  int n_pairs;           // tile pairs (tile 2q + rank of pair q goes to CTA `rank`)
  int nacc;              // projection accumulators in TMEM (2: the epilogue of tile k overlaps tile k+1's MMAs)
  // CTA-pair kernel, FP8: per-Z-row scale codes (shared memory, one byte per
  // row and A buffer) and the TMEM scale-factor columns: sfg groups of four
  // columns per A buffer from sf_col, then the basis scale
  uint32_t off_codes, codes_stride;
  uint32_t sf_col;
  int sfg;
  // CTA-pair kernel, dynamic schedule (dyn = 1): after its first pair, each
  // cluster claims the next ones from sched[0] (a launch-wide counter that
  // the last CTA to finish, counted in sched[1], resets to zero)
  int dyn;
  unsigned long long* sched;
  // CTA-pair kernel with the correction MLP fused in its epilogue (Hd > 0)
  const uint8_t* mlp_img;  // two halves of mlp_half bytes (W1 blocks, W2 blocks, vectors)
  uint32_t mlp_half;
  int Hd;                  // hidden units
  uint32_t off_mlp;        // shared-memory offset of this CTA's half
  uint32_t mlp_w2_off, mlp_vec_off;  // W2 blocks and FP32 vectors within a half
  uint32_t w1_step, w2_step;         // bytes per K-step block of this CTA's W1 / W2 rows
  uint32_t idesc1, idesc2;           // the two MLP GEMMs (M = 256, N = Hd / MP)
  uint32_t a1_col, h_col, y_col;     // TMEM columns of x-hat (chunk c at a1_col + 16 c), the hidden layer, the output
  // CTA-pair kernel, MFCC with the DCT-II on the tensor cores (dct_tc = 1):
  // the log-Mel row goes to TMEM as a split-BF16 A operand (hi and lo parts,
  // MP/2 columns each, at dct_ahi / dct_alo), the DCT matrix sits in shared
  // memory at off_dct as this CTA's dct_n / 2 rows (hi part, then lo part,
  // dct_part bytes each, K-major core matrices), and the coefficients
  // accumulate in dct_n TMEM columns at dct_c (M = 256 over the pair)
  int dct_tc, dct_n;
  uint32_t dct_ahi, dct_alo, dct_c, dct_part, idesc_dct;
};

// barrier indices
struct Bars {
  int z_full, z_empty, b_full, b_empty, t_full, t_empty, drain, total;
  __host__ __device__ Bars(int ZB, int NB) {
    z_full = 0;
    z_empty = z_full + ZB;
    b_full = z_empty + ZB;
    b_empty = b_full + NB;
    t_full = b_empty + NB;
    t_empty = t_full + 2;
    drain = t_empty + 2;
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

// Streaming read of 4 samples that were prefetched into L2: read once, keep out of L1.
static __device__ __forceinline__ float4 ldg_stream(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Samples of a tile's span that lie in the clip: the span is zrows * H samples,
// cut at the clip end rounded up to 4 (the caller guarantees that much is readable).
static __device__ __forceinline__ long long tile_avail(const TcParams& p, const TileDesc& td) {
  const long long span = (long long)p.zrows * p.H;
  return min(((long long)td.n_samples + 3) & ~3ll, span);
}

// Bulk prefetch of a tile's sample span into L2 (pieces of <= 32 KB).
static __device__ void prefetch_tile(const TcParams& p, int tile) {
  const TileDesc td = p.tiles[tile];
  const long long avail = tile_avail(p, td);
  const float* src = p.wave + td.in_off;
  for (long long o = 0; o < avail; o += 8192) {
    const long long n = min(8192ll, avail - o);
    prefetch_l2(src + o, (uint32_t)(n * 4));
  }
}

// One converter thread runs the prefetch stream: tiles blockIdx.x + i*gridDim.x,
// `pf` tiles ahead of the tile being converted.  The descriptor of the next
// tile to prefetch is loaded one step early, so a step never waits on it.
struct Prefetcher {
  int next;
  TileDesc pend;
  __device__ void start(const TcParams& p) {
    next = blockIdx.x;
    for (int i = 0; i < p.pf && next < p.n_tiles; ++i, next += gridDim.x) prefetch_tile(p, next);
    if (p.pf > 0 && next < p.n_tiles) pend = p.tiles[next];
  }
  __device__ void step(const TcParams& p) {
    if (p.pf > 0 && next < p.n_tiles) {
      const long long avail = tile_avail(p, pend);
      const float* src = p.wave + pend.in_off;
      for (long long o = 0; o < avail; o += 8192)
        prefetch_l2(src + o, (uint32_t)(min(8192ll, avail - o) * 4));
      next += gridDim.x;
      if (next < p.n_tiles) pend = p.tiles[next];
    }
  }
};

// Zero the samples of a quad that lie past the clip end (s = span index of x.x).
static __device__ __forceinline__ void clip_quad(float4& x, int s, int nsamp) {
  if (s + 4 > nsamp) {
    x.x = s < nsamp ? x.x : 0.f;
    x.y = s + 1 < nsamp ? x.y : 0.f;
    x.z = s + 2 < nsamp ? x.z : 0.f;
    x.w = s + 3 < nsamp ? x.w : 0.f;
  }
}

// ----------------------------------------------------------------- roles
static __device__ void role_basis_producer(const TcParams& p, uint32_t sbase, const Bars& B,
                                    volatile int* abort) {
  const uint64_t pol = policy_evict_last();
  if (p.b_resident) {
    // the whole basis once, in copies of <= 32 KB that all complete on b_full[0];
    // consumers never release it
    const uint32_t full = sbase + p.off_bar + 8 * B.b_full;
    const uint32_t total = p.step_bytes * (uint32_t)p.KS;
    mbar_arrive_expect_tx(full, total);
    for (uint32_t o = 0; o < total; o += 32768u)
      bulk_g2s_hint(sbase + p.off_b + o, p.bimg + o, min(32768u, total - o), full, pol);
    drain_wait(full, 0, p.err);
    return;
  }
  // streamed: slots of kps consecutive K-steps (contiguous in the basis image)
  int slot = 0;
  uint32_t phase = 0;
  int issued = 0;
  bool ok = true;
  for (int tile = blockIdx.x; ok && tile < p.n_tiles; tile += gridDim.x) {
    for (int b = 0; ok && b < p.nblk; ++b) {
      // block b's K-steps are contiguous in the image (one block: the whole image)
      const uint32_t step = b + 1 < p.nblk ? p.blk_step : p.blk_step_last;
      const uint8_t* src = p.bimg + (size_t)b * p.KS * p.blk_step;
      for (int s0 = 0; s0 < p.KS; s0 += p.kps) {
        const uint32_t full = sbase + p.off_bar + 8 * (B.b_full + slot);
        const uint32_t empty = sbase + p.off_bar + 8 * (B.b_empty + slot);
        if (!mbar_wait(empty, phase ^ 1, abort, p.err, kErrTimeout)) {
          ok = false;
          break;
        }
        const uint32_t bytes = (uint32_t)min(p.kps, p.KS - s0) * step;
        mbar_arrive_expect_tx(full, bytes);
        bulk_g2s_hint(sbase + p.off_b + slot * p.bslot_bytes, src + (size_t)s0 * step, bytes, full, pol);
        ++issued;
        if (++slot == p.NB) {
          slot = 0;
          phase ^= 1;
        }
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
  const uint32_t abuf16 = p.abuf_bytes >> 4, apart16 = p.a_bytes >> 4;
  const uint32_t bslot16 = p.bslot_bytes >> 4, bpart16 = p.kstep_bytes >> 4;
  int bslot = 0;
  uint32_t bphase = 0;
  int k = 0, kb = 0;  // tile ordinal; accumulator-block ordinal (kb == k with one block)
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const int zb = p.ZB == 2 ? (k & 1) : 0;
    if (!mbar_wait(sbase + p.off_bar + 8 * (B.z_full + zb), (p.ZB == 2 ? (k >> 1) : k) & 1,
                   abort, p.err, kErrTimeout))
      break;
    bool ok = true;
    const uint32_t alo = a_lo0 + zb * abuf16;
    for (int b = 0; ok && b < p.nblk; ++b, ++kb) {
      const int acc = kb & 1;
      if (!mbar_wait(sbase + p.off_bar + 8 * (B.t_empty + acc), ((kb >> 1) & 1) ^ 1, abort, p.err,
                     kErrTimeout)) {
        ok = false;
        break;
      }
      if (p.b_resident && k == 0) ok = mbar_wait(sbase + p.off_bar + 8 * B.b_full, 0, abort, p.err, kErrTimeout);
      if (!ok) break;
      tc_fence_after();
      const uint32_t d = tmem_base + acc * p.acc_stride;
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
              mma_f16(d, ad, bd, p.idesc, s > 0);
              if constexpr (PREC == MELT_BF16X3) {
                mma_f16(d, ad, hi | (ty[u] + bpart16), p.idesc, 1);
                mma_f16(d, hi | (alo + tx[u] + apart16), bd, p.idesc, 1);
              }
            }
          }
        }
      } else {
        // block b: N = 2 x (its Mel bins) rows, their K-steps streamed through the slot ring
        const bool last = b + 1 == p.nblk;
        const uint32_t step = last ? p.blk_step_last : p.blk_step;
        const uint32_t rows = last ? 2u * (uint32_t)p.wbl : (p.nblk > 1 ? 256u : (uint32_t)p.NC);
        const uint32_t idesc = last ? p.idesc_last : p.idesc;
        const uint32_t step16 = step >> 4;
        const uint32_t part16 = PREC == MELT_BF16X3 ? step16 / 2 : 0u;  // lo part of a K-step block
        const uint32_t blo_b = ((sbase + p.off_b) >> 4) | (((rows * 16u) >> 4) << 16);
        for (int s0 = 0; s0 < p.KS && ok; s0 += p.kps) {
          if (!mbar_wait(sbase + p.off_bar + 8 * (B.b_full + bslot), bphase, abort, p.err,
                         kErrTimeout)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t blo0 = blo_b + bslot * bslot16;
          const int n = min(p.kps, p.KS - s0);
          for (int u = 0; u < n; ++u) {
            const int s = s0 + u;
            const uint2 t = tab[s];
            const uint32_t blo = blo0 + u * step16;
            const uint64_t ad = hi | (alo + t.x);
            const uint64_t bd = hi | blo;
            mma_f16(d, ad, bd, idesc, s > 0);
            if constexpr (PREC == MELT_BF16X3) {
              mma_f16(d, ad, hi | (blo + part16), idesc, 1);
              mma_f16(d, hi | (alo + t.x + apart16), bd, idesc, 1);
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
      mma_commit(sbase + p.off_bar + 8 * (B.t_full + acc));
    }
    if (!ok) break;
    mma_commit(sbase + p.off_bar + 8 * (B.z_empty + zb));
  }
  // no MMA may still be running when TMEM is released
  mma_commit(sbase + p.off_bar + 8 * B.drain);
  drain_wait(sbase + p.off_bar + 8 * B.drain, 0, p.err);
}

// BF16 / BF16X3 converter: waveform quads (global, L2-prefetched) -> Z rows.
//
// Quad q of a tile is the 4 samples at span offset 4q: Z row u = q / (H/4),
// column r = 4 (q % (H/4)).  Thread ct takes quads ct, ct + 256, ...; lanes of
// a warp read 512 contiguous bytes per load instruction.  In shared memory,
// Z element (u, r) sits at (r / 8) * lbo_a + 16 u + 2 (r % 8).
//
// The CTA's tiles are one stream of batches (kQuadBatch quads per thread).
// Two register sets alternate: the loads of batch i+1 are in flight while
// batch i is converted and stored, across tile boundaries too, so the stream
// pays one memory latency at its start rather than one per batch.
struct CvtCursor {
  int tile, k, b;      // tile index, its ordinal for this CTA, batch within the tile
  const float* src;    // sample 0 of the tile's span
  int nsamp;           // samples of the clip from src on
  TileDesc nxt;        // descriptor of the CTA's following tile (loaded early)
};

static __device__ __forceinline__ bool cursor_advance(const TcParams& p, CvtCursor& c, int nb) {
  if (++c.b < nb) return true;
  c.b = 0;
  c.tile += gridDim.x;
  ++c.k;
  if (c.tile >= p.n_tiles) return false;
  c.src = p.wave + c.nxt.in_off;
  c.nsamp = c.nxt.n_samples;
  if (c.tile + (int)gridDim.x < p.n_tiles) c.nxt = p.tiles[c.tile + gridDim.x];
  return true;
}

static __device__ __forceinline__ void cvt_load(const TcParams& p, const CvtCursor& c, int ct,
                                                float4 (&x)[kQuadBatch]) {
  const int q0 = c.b * kQuadBatch * kCvtThreads + ct;
#pragma unroll
  for (int i = 0; i < kQuadBatch; ++i) {
    const int q = q0 + i * kCvtThreads;
    x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < p.nq && 4 * q < c.nsamp) x[i] = ldg_stream(c.src + 4 * q);
  }
}

// Convert and store one batch; waits for the A buffer at a tile's first
// batch and publishes the buffer after its last.  false: a wait gave up.
template <int PREC>
static __device__ __forceinline__ bool cvt_store(const TcParams& p, uint32_t sbase, const Bars& B,
                                                 volatile int* abort, const CvtCursor& c, int ct,
                                                 int nb, float4 (&x)[kQuadBatch]) {
  const int zb = p.ZB == 2 ? (c.k & 1) : 0;
  if (c.b == 0 && !warp_wait(sbase + p.off_bar + 8 * (B.z_empty + zb),
                             ((p.ZB == 2 ? (c.k >> 1) : c.k) & 1) ^ 1, abort, p.err))
    return false;
  const uint32_t zaddr = sbase + p.off_a + zb * p.abuf_bytes;
  const int h4 = p.H >> 2;
  const int du = kCvtThreads / h4, dc = kCvtThreads - du * h4;
  const int q0 = c.b * kQuadBatch * kCvtThreads + ct;
  int u = q0 / h4, cc = q0 - u * h4;
#pragma unroll
  for (int i = 0; i < kQuadBatch; ++i) {
    const int q = q0 + i * kCvtThreads;
    if (q < p.nq) {
      clip_quad(x[i], 4 * q, c.nsamp);
      const uint32_t h0 = pack_bf16(x[i].x, x[i].y), h1 = pack_bf16(x[i].z, x[i].w);
      const uint32_t a = zaddr + (uint32_t)(cc >> 1) * p.lbo_a + (uint32_t)u * 16u + (cc & 1) * 8u;
      asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(h0), "r"(h1));
      if constexpr (PREC == MELT_BF16X3) {
        const uint32_t l0 = pack_bf16(x[i].x - __uint_as_float(h0 << 16),
                                      x[i].y - __uint_as_float(h0 & 0xffff0000u));
        const uint32_t l1 = pack_bf16(x[i].z - __uint_as_float(h1 << 16),
                                      x[i].w - __uint_as_float(h1 & 0xffff0000u));
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + p.a_bytes), "r"(l0), "r"(l1));
      }
    }
    cc += dc;
    u += du;
    if (cc >= h4) {
      cc -= h4;
      ++u;
    }
  }
  if (c.b == nb - 1) {
    fence_proxy_async();
    warp_arrive(sbase + p.off_bar + 8 * (B.z_full + zb));
  }
  return true;
}

template <int PREC>
static __device__ void role_convert_bf16(const TcParams& p, uint32_t sbase, const Bars& B,
                                         volatile int* abort) {
  const int ct = threadIdx.x - 32 * kCvtWarp0;
  const int nb = (p.nq + kQuadBatch * kCvtThreads - 1) / (kQuadBatch * kCvtThreads);
  if ((int)blockIdx.x >= p.n_tiles) return;
  Prefetcher pf;
  if (ct == 0) pf.start(p);
  CvtCursor cur;
  cur.tile = blockIdx.x;
  cur.k = 0;
  cur.b = 0;
  {
    const TileDesc td = p.tiles[cur.tile];
    cur.src = p.wave + td.in_off;
    cur.nsamp = td.n_samples;
  }
  if (cur.tile + (int)gridDim.x < p.n_tiles) cur.nxt = p.tiles[cur.tile + gridDim.x];
  float4 xa[kQuadBatch], xb[kQuadBatch];
  cvt_load(p, cur, ct, xa);
  CvtCursor nxt = cur;
  bool more = cursor_advance(p, nxt, nb);
  for (;;) {
    if (more) cvt_load(p, nxt, ct, xb);
    if (ct == 0 && cur.b == 0) pf.step(p);
    if (!cvt_store<PREC>(p, sbase, B, abort, cur, ct, nb, xa) || !more) break;
    cur = nxt;
    more = cursor_advance(p, nxt, nb);
    if (more) cvt_load(p, nxt, ct, xa);
    if (ct == 0 && cur.b == 0) pf.step(p);
    if (!cvt_store<PREC>(p, sbase, B, abort, cur, ct, nb, xb) || !more) break;
    cur = nxt;
    more = cursor_advance(p, nxt, nb);
  }
}

// MFCC (Eq. 9): coefficients kk0 .. kk0+3 of one frame, C[kk] = sum_m lm[m]
// D[kk][m], from its log-Mel row in registers and the DCT-II matrix in shared
// memory (rows of 16 NCH floats, zero past M; the matrix is padded with zero
// rows to a multiple of four).  Four independent sums, each in order m = 0,
// 1, ..., so that one FMA issues per cycle.
template <int NCH>
static __device__ __forceinline__ float4 dct_quad(const float (&lm)[16 * NCH], const float* dct, int kk0) {
  float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int qq = 0; qq < 4 * NCH; ++qq) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 d = reinterpret_cast<const float4*>(dct + (kk0 + r) * 16 * NCH)[qq];
      a[r] = fmaf(lm[4 * qq], d.x, a[r]);
      a[r] = fmaf(lm[4 * qq + 1], d.y, a[r]);
      a[r] = fmaf(lm[4 * qq + 2], d.z, a[r]);
      a[r] = fmaf(lm[4 * qq + 3], d.w, a[r]);
    }
  }
  return make_float4(a[0], a[1], a[2], a[3]);
}

// Stores coefficients kk0 .. kk0+3 (those below n_mfcc) of a frame's row:
// one 16-byte store when the row is 16-byte aligned and all four exist.
static __device__ __forceinline__ void store_quad(float* orow, int kk0, int n_mfcc, float4 v, bool vec4) {
  if (vec4 && kk0 + 4 <= n_mfcc) {
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(orow + kk0), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
  } else {
    const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (kk0 + r < n_mfcc) orow[kk0 + r] = a[r];
  }
}

// Fills the shared-memory DCT-II matrix: n_mfcc rows of MP floats (zero past
// M), then zero rows up to a multiple of four.
static __device__ __forceinline__ void fill_dct(const TcParams& p, float* dct, int t0, int nt) {
  const int rows = (p.n_mfcc + 3) & ~3;
  for (int i = t0; i < rows * p.MP; i += nt) {
    const int kk = i / p.MP, m = i - kk * p.MP;
    dct[i] = (kk < p.n_mfcc && m < p.M) ? p.dct[kk * p.M + m] : 0.f;
  }
}

// Fused STFT + Mel comparator, epilogue state of one frame: the bands run in
// order; acc0 holds band c, acc1 band c + 1.  A bin k adds w0 |X_k|^2 to band
// b0(k) and w1 |X_k|^2 to band b0(k) + 1 (b0 is the same for every frame, so
// the control flow is uniform); bands below b0(k) are complete and are
// written (log(E + eps)) as c moves up to b0(k).  The host table gives, per
// bin, how many bands complete before it (nf = b0(k) minus the previous
// in-range bin's b0; 0 or 1 almost everywhere), so the walk takes no
// comparison per bin: one flush on a uniform branch, a loop only for the
// rare larger steps of narrow low-frequency bands.
struct StftBands {
  float acc0, acc1;
  int c;
};

static __device__ __forceinline__ void stft_flush(StftBands& st, float* orow, int nb, float eps, bool valid) {
  if (valid && st.c >= 0 && st.c < nb) orow[st.c] = fast_ln(st.acc0 + eps);
  st.acc0 = st.acc1;
  st.acc1 = 0.f;
  ++st.c;
}

static __device__ __forceinline__ void stft_bin(StftBands& st, const float4* fbs, int k, float s2, float* orow,
                                                int nb, float eps, bool valid) {
  const float4 f = fbs[k];
  const int nf = __float_as_int(f.w);
  if (nf > 0) {
    stft_flush(st, orow, nb, eps, valid);
    for (int i = 1; i < nf; ++i) stft_flush(st, orow, nb, eps, valid);
  }
  // bins outside every triangle carry zero weights
  st.acc0 = fmaf(f.x, s2, st.acc0);
  st.acc1 = fmaf(f.y, s2, st.acc1);
}

template <int PREC, int NCH, bool MFCC, bool STFT = false>
__device__ void role_epilogue(const TcParams& p, uint8_t* gbase, uint32_t sbase, const Bars& B,
                              uint32_t tmem_base, volatile int* abort) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * warp + lane;
  const float* dct = reinterpret_cast<const float*>(gbase + p.off_dct);  // [n_mfcc][dct_ld]
  const bool vec8 = ((p.n_out & 7) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 31) == 0);
  const bool vec4 = ((p.n_out & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 15) == 0);
  int k = 0, kb = 0;  // tile ordinal; accumulator-block ordinal (kb == k with one block)
  TileDesc td_next;
  if ((int)blockIdx.x < p.n_tiles) td_next = p.tiles[blockIdx.x];
  for (int tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x, ++k) {
    const TileDesc td = td_next;  // loaded one tile early
    if (tile + (int)gridDim.x < p.n_tiles) td_next = p.tiles[tile + gridDim.x];
    const bool valid = row < td.n_frames;
    float* orow = p.out + (size_t)(td.out_row + row) * p.n_out;
    if constexpr (!MFCC) {
      bool ok = true;
      [[maybe_unused]] StftBands stb{0.f, 0.f, -1};  // fused STFT + Mel comparator: no band started yet
      for (int b = 0; b < p.nblk; ++b, ++kb) {
        const int acc = kb & 1;
        if (!warp_wait(sbase + p.off_bar + 8 * (B.t_full + acc), (kb >> 1) & 1, abort, p.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // block b: Mel bins m0 .. m0 + wb - 1, R in columns [0, wb), I in [wb, 2 wb)
        const int wb = b + 1 == p.nblk ? (p.nblk > 1 ? p.wbl : p.MP) : 128;
        const int m0 = 128 * b;
        const int nch = wb >> 4;
        const uint32_t t0 = tmem_base + ((uint32_t)(32 * warp) << 16) + acc * p.acc_stride;
        // groups of up to kEpiGroup 16-column chunks: all of a group's TMEM loads
        // are issued before one wait; TMEM is released after the last group's wait
#pragma unroll 1
        for (int c0 = 0; c0 < nch; c0 += kEpiGroup) {
          float re[kEpiGroup][16], im[kEpiGroup][16];
#pragma unroll
          for (int g = 0; g < kEpiGroup; ++g) {
            if (c0 + g < nch) {
              tmem_ld16(t0 + 16 * (c0 + g), re[g]);
              tmem_ld16(t0 + wb + 16 * (c0 + g), im[g]);
            }
          }
          tmem_ld_wait();
#pragma unroll
          for (int g = 0; g < kEpiGroup; ++g) {
            reg_fence16(re[g]);
            reg_fence16(im[g]);
          }
          if (c0 + kEpiGroup >= nch) {
            tc_fence_before();
            warp_arrive(sbase + p.off_bar + 8 * (B.t_empty + acc));
          }
          if constexpr (STFT) {
            // the comparator: |X_k|^2 of DFT bin k into the triangular bands, in
            // bin order.  Every loop over the chunk's registers is fully
            // unrolled: a runtime index would move re/im to local memory.
            const float4* fbs = reinterpret_cast<const float4*>(gbase + p.off_fb);
#pragma unroll
            for (int g = 0; g < kEpiGroup; ++g) {
#pragma unroll
              for (int e = 0; e < 16; ++e) re[g][e] = fmaf(re[g][e], re[g][e], im[g][e] * im[g][e]);
            }
#pragma unroll
            for (int g = 0; g < kEpiGroup; ++g) {
              const int cc = c0 + g;
              if (cc < nch) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                  const int kbin = m0 + 16 * cc + e;
                  if (kbin < p.M) stft_bin(stb, fbs, kbin, re[g][e], orow, p.stft_bands, p.eps, valid);
                }
              }
            }
            continue;
          }
#pragma unroll
          for (int g = 0; g < kEpiGroup; ++g) {
            const int cc = c0 + g;
            if (cc < nch) {
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float r = re[g][e], i = im[g][e];
                re[g][e] = fast_ln(fmaf(r, r, fmaf(i, i, p.eps)));
              }
              const int m = m0 + 16 * cc;
              if (valid) {
                if (vec8 && m + 16 <= p.M) {
                  stg256(orow + m, re[g]);
                  stg256(orow + m + 8, re[g] + 8);
                } else {
#pragma unroll
                  for (int e = 0; e < 16; ++e)
                    if (m + e < p.M) orow[m + e] = re[g][e];
                }
              }
            }
          }
        }
      }
      if (!ok) break;
      if constexpr (STFT)
        while (stb.c < p.stft_bands) stft_flush(stb, orow, p.stft_bands, p.eps, valid);
      continue;
    } else {
      // MFCC (one accumulator block): the frame's log-Mel row stays in
      // registers; C[k] = sum_m lm[m] D[k][m]
      const int acc = k & 1;
      if (!warp_wait(sbase + p.off_bar + 8 * (B.t_full + acc), (k >> 1) & 1, abort, p.err)) break;
      tc_fence_after();
      const uint32_t t0 = tmem_base + ((uint32_t)(32 * warp) << 16) + acc * p.acc_stride;
      float lm[16 * NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        float re[16], im[16];
        tmem_ld16(t0 + 16 * c, re);
        tmem_ld16(t0 + 16 * NCH + 16 * c, im);
        tmem_ld_wait(re, im);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float r = re[e], i = im[e];
          lm[16 * c + e] = (16 * c + e < p.M) ? fast_ln(fmaf(r, r, i * i) + p.eps) : 0.f;
        }
      }
      tc_fence_before();
      warp_arrive(sbase + p.off_bar + 8 * (B.t_empty + acc));
#pragma unroll 1
      for (int kk0 = 0; kk0 < p.n_mfcc; kk0 += 4) {
        const float4 v = dct_quad<NCH>(lm, dct, kk0);
        if (valid) store_quad(orow, kk0, p.n_mfcc, v, vec4);
      }
    }
  }
}

// STFT: the fused STFT + Mel comparator's epilogue (its own instantiation, so
// that the log-Mel kernel does not carry its registers)
template <int PREC, int NCH, bool MFCC, bool STFT = false>
__global__ void __launch_bounds__(kThreads, 1) melt_tc_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 127u) & ~127u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Bars B(p.ZB, p.NB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + p.off_misc);
  volatile int* abort = reinterpret_cast<volatile int*>(gbase + p.off_misc + 4);

  if (threadIdx.x == 0) {
    auto bar = [&](int i) { return sbase + p.off_bar + 8 * i; };
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
    mbar_init(bar(B.drain), 1);
    *abort = 0;
    fence_mbar_init();
  }
  // K-step descriptor table: A start offset (16-byte units) and resident B low word
  if (warp == kBWarp) {
    uint2* tab = reinterpret_cast<uint2*>(gbase + p.off_tab);
    const uint32_t b_lo0 = ((sbase + p.off_b) >> 4) | (((uint32_t)p.NC * 16 >> 4) << 16);
    const uint32_t bslot16 = p.step_bytes >> 4;
    // steps in (slice j, 16-column group kk) order, the order of the basis image
    for (int j = 0, s0 = 0; j < p.J; ++j) {
      const int steps = (min(p.H, p.N - j * p.H) + 15) / 16;
      for (int kk = lane; kk < steps; kk += 32)
        tab[s0 + kk] = make_uint2((2u * kk * p.lbo_a + 16u * j) >> 4, b_lo0 + (s0 + kk) * bslot16);
      s0 += steps;
    }
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(tmem_slot), p.tmem_cols);
    tmem_relinquish();
  }
  if (STFT && warp < kEpiWarps) {  // the comparator's filterbank table
    float4* fbs = reinterpret_cast<float4*>(gbase + p.off_fb);
    for (int i = threadIdx.x; i < p.M; i += kEpiThreads) fbs[i] = p.fb[i];
  }
  if constexpr (MFCC) {
    // DCT-II rows padded with zeros to MP columns (16-byte aligned rows)
    if (warp < kEpiWarps) {
      fill_dct(p, reinterpret_cast<float*>(gbase + p.off_dct), threadIdx.x, kEpiThreads);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  if (threadIdx.x == 0) pdl_launch_dependents();

  // The MMA issuer and the basis producer touch only this launch's own
  // basis and shared memory, so they start at once; every role that reads
  // the tile list, the waveform or writes features first waits for the
  // previous kernel of the stream (programmatic dependent launch), except
  // that the converters skip that wait when the caller stated that the
  // waveform is not written by a kernel still in flight (early_inputs).
  if (warp == kMmaWarp) {
    if (lane == 0) role_mma<PREC>(p, gbase, sbase, B, tmem_base, abort);
    __syncwarp();
  } else if (warp == kBWarp) {
    if (lane == 0) role_basis_producer(p, sbase, B, abort);
    __syncwarp();
  } else if (warp >= kCvtWarp0) {
    if (!p.early_inputs) pdl_wait();
    role_convert_bf16<PREC>(p, sbase, B, abort);
    __syncwarp();
  } else {
    pdl_wait();
    role_epilogue<PREC, NCH, MFCC, STFT>(p, gbase, sbase, B, tmem_base, abort);
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
KernelFn kernel_for_plain(int prec, int nch, bool stft = false);
KernelFn kernel_for_mfcc(int prec, int nch);
// Defined in melt_tc2.cu: the CTA-pair kernel (BF16).
KernelFn kernel_for_pair(bool mfcc, int nch, bool dtc);
// Defined in melt_tc2_mlp.cu: the CTA-pair kernel with the fused correction MLP.
KernelFn kernel_for_pair_mlp(int nch);
// Defined in melt_tc2_fp8.cu: the CTA-pair kernel with FP8 e4m3 operands.
KernelFn kernel_for_pair_fp8(bool mfcc, int nch, bool dtc);
// Defined in melt_tc2_x3.cu: the CTA-pair kernel with split-BF16 operands.
KernelFn kernel_for_pair_x3();

}  // namespace tc
}  // namespace melt
