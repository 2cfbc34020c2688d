// Device side of the CTA-pair tensor-core MelT kernel (BF16), included by
// melt_tc2.cu.
#pragma once
// The pair kernel (BF16 and FP8 e4m3) runs as clusters of two CTAs on
// neighbouring SMs.  The even
// CTA issues 2-SM MMAs (tcgen05 cta_group::2, M = 256): each CTA supplies the
// A operand of its own 128-frame tile, and the basis B is split by its rows
// between the two, so each CTA keeps only half of it (W_r rows in the even
// CTA, W_i rows in the odd one) resident in shared memory.  The half that is
// saved holds a TMA staging ring for the waveform, so the FP32 samples arrive
// by bulk copies (deep in flight, no registers) while the basis never moves.
// Each CTA's TMEM receives R and I of its own frames, so the epilogue is the
// single-CTA one.
//
// FP8 e4m3 (template PREC): the converters quantise each polyphase Z row
// (H samples) with its own power-of-two scale 2^e_u, e_u the least integer
// with max|row| 2^-e_u <= 448, and write the rows' UE8M0 scale codes into
// TMEM; the MMAs are block-scaled (kind::mxf8f6f4), so the tensor cores apply
// 2^e_u to every product of row u (the scale of A row t in slice j is that of
// Z row t + j, selected by the scale-factor byte j) and 2^-8 to the basis,
// which is stored as e4m3(W 2^8).  The accumulator holds R and I directly.
//
// Warp roles per CTA (11 warps; 16 with the fused MLP):
//   warps 0-3   epilogue: TMEM -> registers, R^2 + I^2, log, (DCT), store (with
//               the fused MLP, warps 0-11: warps e, e+4 and e+8 read the same
//               32 TMEM lanes (frames) and split the bands and hidden units)
//   next warp   TMEM allocation for the pair; in the even CTA, the MMA issuer
//   next warp   basis producer: this CTA's half of the basis, once (with the
//               fused MLP, lane 1 of the MMA warp instead)
//   next warp   waveform producer: bulk copies of the tile's FP32 span into a ring
//   last four   converters: staged FP32 samples -> polyphase Z rows (BF16, or
//               e4m3 with per-row scales written to TMEM; two warps with the
//               fused MLP)
//
// Fused correction MLP (template flag MLP).  After the log-Mel of a tile the
// epilogue writes x-hat = (x - mu)/sd as BF16 into TMEM and the even CTA
// issues two more 2-SM MMAs with the A operand in TMEM: H = x-hat W1^T (W1
// rows split between the CTAs like the basis) and, after the epilogue has
// written GELU(H + b1) in BF16 over H and x + b2 into the output columns,
// Y = x + b2 + GELU(H) W2^T, which the epilogue stores.  TMEM per CTA: the
// projection accumulator (one, columns [0, NC)), the output at y_col with
// x-hat's band chunk c in the first half of the output's chunk c (consumed
// by GEMM1 before anything is written there; each epilogue warp writes only
// chunks it has read back itself), H and GELU(H) at h_col.  The next tile's
// projection MMAs run while the epilogue works through the MLP of this one.
//
// Synchronisation.  Barriers that gate the pair's MMAs live in the even CTA
// and count arrivals from both CTAs (the odd CTA arrives through its
// shared::cluster address): Z buffers full (converters of both), accumulators
// drained (epilogues of both), odd half of the basis loaded.  MMA completion
// is multicast to both CTAs' barriers (Z buffer free, accumulator full).
// Every wait is bounded; both CTAs meet in a cluster barrier before either
// releases TMEM or exits, so no CTA touches a peer that has left.
#include "melt_tc_kernel.cuh"

namespace melt {
namespace tc {

// Warp layout of a pair kernel with `epw` epilogue warps: epilogue
// 0..epw-1, MMA epw, basis epw+1, waveform epw+2, then the converters.  With
// the fused MLP the basis producer runs on lane 1 of the MMA warp instead
// (its work is a few copies at the start), so the block is 16 warps: 12
// epilogue, MMA + basis, waveform, 2 converters, and keeps 128 registers a
// thread.
constexpr int kPCvtWarps = 4;
constexpr int kPCvtThreads = 32 * kPCvtWarps;  // 128
constexpr int kMlpCvtWarps = 2;                // converter warps with the fused MLP
// Epilogue warps: 12 (three per TMEM lane quarter) with the fused MLP,
// whose GELU of every hidden unit is the longest step of a tile; 8 (two per
// quarter) for the MFCC epilogue with the DCT on the tensor cores and for the
// MFCC epilogue with the DCT on the CUDA cores where M <= 80 (the two split
// the coefficients); 4 otherwise.
constexpr int kMlpParts = 3;  // fused MLP: epilogue warps per lane quarter
__host__ __device__ constexpr int pair_epi_warps(bool mlp, bool mfcc = false, int nch = 1, bool dtc = false) {
  return mlp ? 4 * kMlpParts : (mfcc && (dtc || nch <= 5)) ? 8 : 4;
}

// Part j of `parts` near-equal runs of n chunks: chunks [lo_j, lo_{j+1}),
// the larger runs first (part_lo) or last (part_lo_tail).  The fused MLP's
// epilogue splits the bands with the first and the hidden units with the
// second, so that its warps' shares of the two even out.
__host__ __device__ constexpr int part_lo(int n, int parts, int j) {
  return j * (n / parts) + (j < n % parts ? j : n % parts);
}
__host__ __device__ constexpr int part_lo_tail(int n, int parts, int j) {
  return j * (n / parts) + (j > parts - n % parts ? j - (parts - n % parts) : 0);
}
// Converter warps: 4 (BF16: each sample converted once, short chains), 8 for
// FP8's log-Mel kernel and its MFCC kernel with the DCT on the tensor cores,
// whose per-row max makes each chunk one dependent chain per row set (twice
// the warps, half the chain).  The MFCC kernels with the DCT on the CUDA
// cores keep 4 (their epilogue warps and registers fill the block).  With
// the fused MLP, 2: a tile takes several microseconds there, and the warps
// go to the epilogue.
__host__ __device__ constexpr int pair_cvt_warps(int prec, bool mfcc, int nch, bool dtc = false, bool mlp = false) {
  return mlp ? kMlpCvtWarps : prec == MELT_FP8E4M3 && (!mfcc || dtc) ? 8 : 4;
}
__host__ __device__ constexpr int pair_threads(bool mlp, int prec = MELT_BF16, bool mfcc = false, int nch = 1,
                                               bool dtc = false) {
  return 32 * (pair_epi_warps(mlp, mfcc, nch, dtc) + (mlp ? 2 : 3) + pair_cvt_warps(prec, mfcc, nch, dtc, mlp));
}
constexpr int kPQuads = 8;  // float4s per converter thread per staged chunk (<= 16 KB)
constexpr uint32_t kSfOne = 0x7F7F7F7Fu;    // four UE8M0 codes of 2^0
constexpr uint32_t kSfBasis = 0x77777777u;  // four UE8M0 codes of 2^-8 (the e4m3 basis holds W 2^8)
constexpr int kSfBCols = 16;                // TMEM columns holding the basis scale (any layout reads 2^-8)

struct PairBars {
  int s_full, s_empty, z_full, z_empty, b_full, peer_b, t_full, t_empty, h_full, a2_full, y_full,
      drain, sched_full, sched_empty, bs_full, bs_peer, bs_empty, total;
  // NB: basis slots of a streamed half basis (0 when it is resident)
  __host__ __device__ PairBars(int NS, int ZB, int KS, int NB = 0) {
    s_full = 0;
    s_empty = s_full + NS;
    z_full = s_empty + NS;
    z_empty = z_full + ZB;
    b_full = z_empty + ZB;
    peer_b = b_full + 1;  // the resident half basis completes on one barrier
    t_full = peer_b + 1;
    t_empty = t_full + 2;
    h_full = t_empty + 2;  // fused MLP: hidden layer in TMEM
    a2_full = h_full + 1;  //            GELU(H) written back (both CTAs' epilogues)
    y_full = a2_full + 1;  //            MLP output in TMEM
    drain = y_full + 1;
    sched_full = drain + 1;              // dynamic schedule: ring entry published (per CTA)
    sched_empty = sched_full + kSchedRing;  //               ring entry read by both epilogues
    bs_full = sched_empty + kSchedRing;  // streamed basis: this CTA's slot filled (transaction bytes)
    bs_peer = bs_full + NB;              //                 the odd CTA's slot filled (even CTA only)
    bs_empty = bs_peer + NB;             //                 the slot's MMAs completed (both CTAs)
    total = bs_empty + NB;
  }
};

struct PairCtx {
  uint32_t sbase;      // this CTA's shared base (shared::cta address)
  uint32_t rank;       // 0 = even CTA (MMA issuer), 1 = odd
  int cluster, n_clusters;
  volatile int* abort;
};

static __device__ __forceinline__ uint32_t pbar(const TcParams& p, const PairCtx& c, int i) {
  return c.sbase + p.off_bar + 8 * i;
}

// Arrival of one warp on a barrier of the even CTA.
static __device__ __forceinline__ void warp_arrive_leader(uint32_t local_bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive_cluster(mapa_shared(local_bar, 0));
}

// ---- pair schedule
// Every role walks the same pair sequence: the cluster's own pair first, then
// either (static) every n_clusters-th pair, or (dynamic) the pairs the even
// CTA's waveform producer claims, one pair ahead of itself, from the
// launch's counter and publishes to both CTAs through a ring of kSchedRing
// entries in shared memory (a pair index >= n_pairs ends the sequence).
static __device__ __forceinline__ uint32_t sched_slot(const TcParams& p, const PairCtx& c, int r) {
  return c.sbase + p.off_misc + 64 + 4 * (r % kSchedRing);
}

// Pair of ordinal k >= 1, read by one thread (dynamic: ring entry k - 1).
// ok turns false if the wait for the entry timed out.
static __device__ int pair_next_thread(const TcParams& p, const PairCtx& c, const PairBars& B, int k,
                                       bool& ok) {
  if (!p.dyn) return c.cluster + k * c.n_clusters;
  const int r = k - 1;
  ok = mbar_wait(pbar(p, c, B.sched_full + r % kSchedRing), (r / kSchedRing) & 1, c.abort, p.err,
                 kErrTimeout);
  if (!ok) return p.n_pairs;
  int q;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(q) : "r"(sched_slot(p, c, r)) : "memory");
  return q;
}

// The same for a whole warp (lane 0 waits and reads).
static __device__ int pair_next_warp(const TcParams& p, const PairCtx& c, const PairBars& B, int k,
                                     bool& ok) {
  int q = 0, good = 1;
  if ((threadIdx.x & 31) == 0) {
    bool o = true;
    q = pair_next_thread(p, c, B, k, o);
    good = o ? 1 : 0;
  }
  q = __shfl_sync(0xffffffffu, q, 0);
  good = __shfl_sync(0xffffffffu, good, 0);
  ok = good != 0;
  return q;
}

// An epilogue warp counts itself out of the ring entry of its pair ordinal
// k >= 1 on the even CTA's barrier.  It does so once the pair's accumulator
// is full: by then both producers, both CTAs' converters and the MMA thread
// have read the entry, so once both epilogues have, the slot may be reused.
static __device__ __forceinline__ void sched_release(const TcParams& p, const PairCtx& c,
                                                     const PairBars& B, int k) {
  if (p.dyn && k > 0) warp_arrive_leader(pbar(p, c, B.sched_empty + (k - 1) % kSchedRing));
}

// Even CTA's producer: publish pair q as ring entry r to both CTAs, a plain
// store and arrival here, an asynchronous store completing on the barrier
// there.  Entry r reuses the slot of entry r - kSchedRing once both CTAs'
// epilogues have read that one.
static __device__ bool sched_publish(const TcParams& p, const PairCtx& c, const PairBars& B, int r,
                                     int q) {
  const int s = r % kSchedRing;
  if (r >= kSchedRing &&
      !mbar_wait(pbar(p, c, B.sched_empty + s), ((r / kSchedRing) - 1) & 1, c.abort, p.err, kErrTimeout))
    return false;
  const uint32_t slot = sched_slot(p, c, r);
  const uint32_t full = pbar(p, c, B.sched_full + s);
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(slot), "r"(q) : "memory");
  mbar_arrive(full);
  const uint32_t peer_full = mapa_shared(full, 1);
  mbar_arrive_expect_tx_cluster(peer_full, 4);
  st_async_u32(mapa_shared(slot, 1), (uint32_t)q, peer_full);
  return true;
}

static __device__ __forceinline__ bool warp_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort,
                                                    int* err) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_cluster(bar, parity, abort, err, kErrTimeout);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// Tile of pair q for this CTA; an odd tile past the end is an empty tile.
static __device__ __forceinline__ TileDesc pair_tile(const TcParams& p, const PairCtx& c, int q) {
  const int t = 2 * q + (int)c.rank;
  TileDesc td;
  if (t < p.n_tiles) return p.tiles[t];
  td.in_off = 0;
  td.out_row = 0;
  td.n_frames = 0;
  td.n_samples = 0;
  td.group = 0;
  td.clip = -1;
  return td;
}

// Bulk prefetch of a tile's sample span into L2 (pieces of <= 32 KB).
static __device__ __forceinline__ void pair_prefetch_span(const TcParams& p, const TileDesc& td) {
  if (td.n_frames == 0) return;
  const long long avail = tile_avail(p, td);
  const float* src = p.wave + td.in_off;
  for (long long o = 0; o < avail; o += 8192)
    prefetch_l2(src + o, (uint32_t)(min(8192ll, avail - o) * 4));
}

// Waveform producer.  Besides the staging copies it keeps (static schedule)
// an L2 prefetch stream `pf` tiles ahead: when it starts tile k it
// prefetches the span of tile k + pf, so the DRAM reads in flight per SM are
// not limited to the staging ring.  The next descriptor to prefetch is read
// one tile early.  In the dynamic schedule the even CTA's producer is the
// one that claims and publishes the pairs.
static __device__ void pair_wave_producer(const TcParams& p, const PairCtx& c, const PairBars& B) {
  const uint64_t pol = policy_evict_first();
  int g = 0;
  bool ok = true;
  int qn = c.cluster + p.pf * c.n_clusters;  // pair whose span is prefetched next
  TileDesc pend = pair_tile(p, c, p.pf > 0 && qn < p.n_pairs ? qn : p.n_pairs);
  for (int i = 1; i < p.pf; ++i) {
    const int qi = c.cluster + i * c.n_clusters;
    if (qi < p.n_pairs) pair_prefetch_span(p, pair_tile(p, c, qi));
  }
  int q = c.cluster;
  for (int k = 0; q < p.n_pairs; ++k) {
    // dynamic schedule, even CTA: claim the pair after this one now; the
    // counter's answer is used after this pair's copies are issued
    unsigned long long claim = 0;
    if (p.dyn && c.rank == 0) claim = atomicAdd(p.sched, 1ull);
    if (p.pf > 0 && qn < p.n_pairs) {
      pair_prefetch_span(p, pend);
      qn += c.n_clusters;
      if (qn < p.n_pairs) pend = pair_tile(p, c, qn);
    }
    const TileDesc td = pair_tile(p, c, q);
    const long long avail = tile_avail(p, td);
    // (an empty tile issues nothing: the converters skip it too)
    for (int ch = 0; td.n_frames > 0 && ch < p.NCHUNK; ++ch, ++g) {
      const int slot = g % p.NS;
      const uint32_t full = pbar(p, c, B.s_full + slot);
      if (!mbar_wait(pbar(p, c, B.s_empty + slot), ((g / p.NS) & 1) ^ 1, c.abort, p.err,
                     kErrTimeout)) {
        ok = false;
        break;
      }
      const long long f0 = (long long)ch * p.CH * p.H;
      const long long nf = max(0ll, min((long long)p.CH * p.H, avail - f0));
      if (nf > 0) {
        mbar_arrive_expect_tx(full, (uint32_t)(nf * 4));
        bulk_g2s_hint(c.sbase + p.off_st + slot * p.st_bytes, p.wave + td.in_off + f0,
                      (uint32_t)(nf * 4), full, pol);
      } else {
        mbar_arrive(full);
      }
    }
    if (!ok) break;
    if (!p.dyn) {
      q += c.n_clusters;
    } else if (c.rank == 0) {
      // claims count from zero in every launch; the first n_clusters pairs are the clusters' own
      const long long ord = (long long)claim;
      const int nq = ord >= (long long)(p.n_pairs - c.n_clusters) ? p.n_pairs : c.n_clusters + (int)ord;
      if (!sched_publish(p, c, B, k, nq)) break;
      q = nq;
    } else {
      q = pair_next_thread(p, c, B, k + 1, ok);
      if (!ok) break;
    }
  }
  // every issued copy has landed before the CTA can exit
  for (int k = max(0, g - p.NS); k < g; ++k)
    drain_wait(pbar(p, c, B.s_full + k % p.NS), (k / p.NS) & 1, p.err);
}

// Streamed half basis (b_resident == 0; static schedule, log-Mel only): for
// every pair of the cluster, this CTA's half of the basis flows through NB
// slots of kps K-steps.  Fill g uses slot g % NB; the even CTA's MMAs of a
// slot release it in both CTAs (multicast commit on bs_empty).
static __device__ void pair_basis_stream(const TcParams& p, const PairCtx& c, const PairBars& B) {
  const uint64_t pol = policy_evict_last();
  const uint32_t total = p.step_bytes * (uint32_t)p.KS;
  const uint8_t* src = p.bimg + (size_t)c.rank * total;  // this CTA's half
  int g = 0;
  bool ok = true;
  for (int q = c.cluster; ok && q < p.n_pairs; q += c.n_clusters) {
    for (int s0 = 0; s0 < p.KS; s0 += p.kps, ++g) {
      const int slot = g % p.NB;
      if (!mbar_wait(pbar(p, c, B.bs_empty + slot), ((g / p.NB) & 1) ^ 1, c.abort, p.err, kErrTimeout)) {
        ok = false;
        break;
      }
      const uint32_t bytes = p.step_bytes * (uint32_t)min(p.kps, p.KS - s0);
      const uint32_t full = pbar(p, c, B.bs_full + slot);
      mbar_arrive_expect_tx(full, bytes);
      bulk_g2s_hint(c.sbase + p.off_b + slot * p.bslot_bytes, src + (size_t)s0 * p.step_bytes, bytes, full, pol);
    }
  }
  // every issued copy has landed before the CTA can exit
  for (int k = max(0, g - p.NB); k < g; ++k) drain_wait(pbar(p, c, B.bs_full + k % p.NB), (k / p.NB) & 1, p.err);
}

// Streamed half basis, odd CTA (its idle MMA warp): as each of its slots
// fills, one arrival on the even CTA's bs_peer barrier of that slot, which
// the even CTA's MMA thread waits on beside its own bs_full.
static __device__ void pair_basis_signal(const TcParams& p, const PairCtx& c, const PairBars& B) {
  int g = 0;
  for (int q = c.cluster; q < p.n_pairs; q += c.n_clusters)
    for (int s0 = 0; s0 < p.KS; s0 += p.kps, ++g) {
      const int slot = g % p.NB;
      if (!mbar_wait(pbar(p, c, B.bs_full + slot), (g / p.NB) & 1, c.abort, p.err, kErrTimeout)) return;
      mbar_arrive_cluster(mapa_shared(pbar(p, c, B.bs_peer + slot), 0));
    }
}

static __device__ void pair_basis_producer(const TcParams& p, const PairCtx& c, const PairBars& B) {
  if (!p.b_resident) {
    pair_basis_stream(p, c, B);
    return;
  }
  const uint64_t pol = policy_evict_last();
  const uint32_t total = p.step_bytes * (uint32_t)p.KS;
  const uint8_t* src = p.bimg + (size_t)c.rank * total;  // this CTA's half
  const uint32_t full = pbar(p, c, B.b_full);
  const uint32_t mlp = p.Hd > 0 ? p.mlp_half : 0u;       // fused MLP: this CTA's weight half
  mbar_arrive_expect_tx(full, total + mlp);
  for (uint32_t o = 0; o < total; o += 32768u)
    bulk_g2s_hint(c.sbase + p.off_b + o, src + o, min(32768u, total - o), full, pol);
  // the weight image is repacked by the kernel just before this one on the
  // stream: read it only once that kernel's writes are visible
  if (mlp > 0) pdl_wait();
  const uint8_t* msrc = p.mlp_img + (size_t)c.rank * mlp;
  for (uint32_t o = 0; o < mlp; o += 32768u)
    bulk_g2s_hint(c.sbase + p.off_mlp + o, msrc + o, min(32768u, mlp - o), full, pol);
  drain_wait(full, 0, p.err);
  if (c.rank == 1) mbar_arrive_cluster(mapa_shared(pbar(p, c, B.peer_b), 0));
}

// Column of the packed GELU(H) of hidden chunk cc (16 units) in the fused
// MLP, relative to H's first column (nh = Hd/16 chunks).  GELU(H) is written
// over H itself: the kMlpParts epilogue warps of a lane quarter take runs
// [lo_j, lo_{j+1}) of the hidden chunks (part_lo_tail), in order, and each
// stores chunk cc only into H columns it has already read: 8 cc + 8 lo_j,
// inside its own run's columns [16 lo_j, 16 cc + 16).
__host__ __device__ constexpr uint32_t mlp_gelu_off(int nh, int cc) {
  int lo = 0;
  for (int j = 1; j < kMlpParts; ++j)
    if (cc >= part_lo_tail(nh, kMlpParts, j)) lo = part_lo_tail(nh, kMlpParts, j);
  return 8u * (uint32_t)(cc + lo);
}
static __device__ __forceinline__ uint32_t gelu_col(const TcParams& p, int cc) {
  return p.h_col + mlp_gelu_off(p.Hd / 16, cc);
}

// Fused MLP (even CTA's MMA thread), hidden layer: H = x-hat W1^T, K-step s
// reading x-hat's band chunk s at a1_col + 16 s.  The caller has seen the
// epilogues' release of the tile's accumulator, which follows the x-hat
// stores.
static __device__ void pair_mlp_gemm1(const TcParams& p, const PairCtx& c, const PairBars& B,
                                      uint32_t tmem_base) {
  const uint64_t hi = (uint64_t)p.desc_hi << 32;
  const uint32_t w1 = ((c.sbase + p.off_mlp) >> 4) | ((((uint32_t)p.Hd / 2 * 16) >> 4) << 16);
  tc_fence_after();
  for (int s = 0; s < p.MP / 16; ++s)
    mma_f16_pair_ts(tmem_base + p.h_col, tmem_base + p.a1_col + 16 * s, hi | (w1 + s * (p.w1_step >> 4)),
                    p.idesc1, s > 0);
  mma_commit_pair_mc(pbar(p, c, B.h_full), 3);
}

// Fused MLP, output layer of the tile with ordinal j: once both CTAs'
// epilogues have written GELU(H + b1) back and x + b2 into the output
// columns, Y = x + b2 + GELU(H) W2^T (every K-step accumulates).
static __device__ bool pair_mlp_gemm2(const TcParams& p, const PairCtx& c, const PairBars& B,
                                      uint32_t tmem_base, int j) {
  const uint64_t hi = (uint64_t)p.desc_hi << 32;
  const uint32_t w2 = ((c.sbase + p.off_mlp + p.mlp_w2_off) >> 4) | ((((uint32_t)p.MP / 2 * 16) >> 4) << 16);
  // the K-steps' A columns before the wait, so that the MMAs issue back to back
  const int nh = p.Hd / 16;  // <= 16
  uint32_t ta[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) ta[s] = tmem_base + gelu_col(p, s < nh ? s : 0);
  if (!mbar_wait_cluster(pbar(p, c, B.a2_full), j & 1, c.abort, p.err, kErrTimeout)) return false;
  tc_fence_after();
#pragma unroll
  for (int s = 0; s < 16; ++s)
    if (s < nh) mma_f16_pair_ts(tmem_base + p.y_col, ta[s], hi | (w2 + s * (p.w2_step >> 4)), p.idesc2, true);
  mma_commit_pair_mc(pbar(p, c, B.y_full), 3);
  return true;
}

// This CTA's rows of the DCT-II matrix as the B operand of the tensor-core
// DCT: rows n = rank dct_n / 2 + i (zero for n >= n_mfcc) over the MP Mel
// bins (zero past M), each value split into BF16 hi = rn(D) and lo =
// rn(D - hi); K-major core matrices of 8 rows x 8 bins, the two parts
// dct_part bytes apart.
static __device__ __forceinline__ void fill_dct_split(const TcParams& p, uint8_t* img, uint32_t rank, int t0,
                                                      int nt) {
  const int nh = p.dct_n / 2;
  __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(img);
  __nv_bfloat16* lo = reinterpret_cast<__nv_bfloat16*>(img + p.dct_part);
  for (int i = t0; i < nh * p.MP; i += nt) {
    const int r = i / p.MP, m = i - r * p.MP;
    const int n = (int)rank * nh + r;
    const float v = (n < p.n_mfcc && m < p.M) ? p.dct[n * p.M + m] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const size_t at = (size_t)(m >> 3) * nh * 8 + (size_t)r * 8 + (m & 7);  // in 2-byte units
    hi[at] = h;
    lo[at] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// MFCC with the DCT on the tensor cores: once both CTAs' epilogues have
// written a tile's log-Mel rows (split into BF16 hi + lo) to TMEM, the
// coefficients C = L D^T accumulate as hi*hi + hi*lo + lo*hi over the K-steps
// of 16 Mel bins (the lo*lo term, below 2^-16 of each product, is dropped).
static __device__ void pair_dct_gemm(const TcParams& p, const PairCtx& c, const PairBars& B, uint32_t tmem_base) {
  const uint64_t hi = (uint64_t)p.desc_hi << 32;
  const uint32_t nh16 = (uint32_t)p.dct_n / 2 * 16;  // bytes between the two K core columns of a K-step
  const uint32_t dhi = ((c.sbase + p.off_dct) >> 4) | ((nh16 >> 4) << 16);
  const uint32_t dlo = dhi + (p.dct_part >> 4);
  const uint32_t step16 = (2 * nh16) >> 4;
  const uint32_t d = tmem_base + p.dct_c;
  tc_fence_after();
  for (int s = 0; s < p.MP / 16; ++s) {
    mma_f16_pair_ts(d, tmem_base + p.dct_ahi + 8 * s, hi | (dhi + s * step16), p.idesc_dct, s > 0);
    mma_f16_pair_ts(d, tmem_base + p.dct_ahi + 8 * s, hi | (dlo + s * step16), p.idesc_dct, true);
    mma_f16_pair_ts(d, tmem_base + p.dct_alo + 8 * s, hi | (dhi + s * step16), p.idesc_dct, true);
  }
  mma_commit_pair_mc(pbar(p, c, B.h_full), 3);
}

// Even CTA only: one thread issues every pair MMA.
template <bool MLP, int PREC, bool DTC = false>
static __device__ void pair_mma(const TcParams& p, uint8_t* gbase, const PairCtx& c,
                                const PairBars& B, uint32_t tmem_base) {
  const uint2* tab = reinterpret_cast<const uint2*>(gbase + p.off_tab);
  const uint64_t hi = (uint64_t)p.desc_hi << 32;
  const uint32_t a_lo0 = ((c.sbase + p.off_a) >> 4) | ((p.lbo_a >> 4) << 16);
  const uint32_t abuf16 = p.abuf_bytes >> 4;
  const int nacc = MLP ? 1 : p.nacc;  // the fused MLP's TMEM leaves room for one accumulator
  const uint32_t sfb = tmem_base + p.sf_col + (uint32_t)(4 * p.sfg * p.ZB);  // FP8: basis scale 2^-8
  // split BF16: the lo part of an A buffer follows its hi part; the lo part
  // of a K-step block of this CTA's basis half follows its hi part
  const uint32_t apart16 = p.a_bytes >> 4, bpart16 = (p.step_bytes / 2) >> 4;
  // streamed half basis: slot descriptors (low word) and the fill count
  const uint32_t bslot0 = ((c.sbase + p.off_b) >> 4) | ((p.b_lbo >> 4) << 16);
  const uint32_t bslot16 = p.bslot_bytes >> 4, step16 = p.step_bytes >> 4;
  int g = 0;
  int k = 0;
  bool ok = true;
  for (;; ++k) {
    const int q = k == 0 ? c.cluster : pair_next_thread(p, c, B, k, ok);
    if (!ok || q >= p.n_pairs) break;
    const int zb = p.ZB == 2 ? (k & 1) : 0;
    const int acc = k % nacc;
    ok = mbar_wait_cluster(pbar(p, c, B.t_empty + acc), ((k / nacc) & 1) ^ 1, c.abort, p.err,
                           kErrTimeout);
    if constexpr (MLP) {
      // the previous tile's x-hat is in TMEM (its accumulator was just
      // released): its hidden layer goes to the tensor cores first, so the
      // epilogue can start on GELU while this tile's projection runs
      if (ok && k > 0) pair_mlp_gemm1(p, c, B, tmem_base);
    }
    ok = ok && mbar_wait_cluster(pbar(p, c, B.z_full + zb), (p.ZB == 2 ? (k >> 1) : k) & 1, c.abort,
                                 p.err, kErrTimeout);
    if (ok && k == 0 && p.b_resident)
      ok = mbar_wait(pbar(p, c, B.b_full), 0, c.abort, p.err, kErrTimeout) &&
           mbar_wait_cluster(pbar(p, c, B.peer_b), 0, c.abort, p.err, kErrTimeout);
    if (!ok) break;
    tc_fence_after();
    const uint32_t d = tmem_base + acc * p.acc_stride;
    const uint32_t alo = a_lo0 + zb * abuf16;
    const uint32_t tab_s = smem_u32(tab);
    if constexpr (PREC != MELT_FP8E4M3 && !MLP && !DTC) {  // (the host plans a streamed basis for these only)
      if (!p.b_resident) {
        // streamed half basis: slot by slot, each once both CTAs' halves are in
        for (int s0 = 0; s0 < p.KS; s0 += p.kps, ++g) {
          const int slot = g % p.NB;
          const uint32_t ph = (g / p.NB) & 1;
          if (!mbar_wait(pbar(p, c, B.bs_full + slot), ph, c.abort, p.err, kErrTimeout) ||
              !mbar_wait(pbar(p, c, B.bs_peer + slot), ph, c.abort, p.err, kErrTimeout)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int n = min(p.kps, p.KS - s0);
          for (int u = 0; u < n; ++u) {
            uint32_t tx, ty;
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(tx), "=r"(ty) : "r"(tab_s + 8u * (s0 + u)));
            const uint32_t bl = bslot0 + slot * bslot16 + u * step16;
            mma_f16_pair(d, hi | (alo + tx), hi | bl, p.idesc, s0 + u > 0);
            if constexpr (PREC == MELT_BF16X3) {
              mma_f16_pair(d, hi | (alo + tx), hi | (bl + bpart16), p.idesc, true);
              mma_f16_pair(d, hi | (alo + tx + apart16), hi | bl, p.idesc, true);
            }
          }
          mma_commit_pair_mc(pbar(p, c, B.bs_empty + slot), 3);
        }
        if (!ok) break;
        mma_commit_pair_mc(pbar(p, c, B.z_empty + zb), 3);
        mma_commit_pair_mc(pbar(p, c, B.t_full + acc), 3);
        continue;
      }
    }
#pragma unroll 1
    for (int s0 = 0; s0 < p.KS; s0 += 8) {
      uint32_t tx[8], ty[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                     : "=r"(tx[u]), "=r"(ty[u])
                     : "r"(tab_s + 8u * min(s0 + u, p.KS - 1)));
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < p.KS) {
          if constexpr (PREC == MELT_FP8E4M3) {
            // K-step of slice j = tx >> 24: A row t is Z row t + j, whose scale is
            // byte j % 4 of scale group j / 4 of this A buffer
            const uint32_t j = tx[u] >> 24;
            const uint32_t sfa = tmem_base + p.sf_col + (uint32_t)(4 * (p.sfg * zb)) + 4u * (j >> 2);
            mma_f8_pair_bs(d, hi | (alo + (tx[u] & 0xFFFFFFu)), hi | ty[u], p.idesc | ((j & 3u) << 29), sfa, sfb,
                           s0 + u > 0);
          } else {
            mma_f16_pair(d, hi | (alo + tx[u]), hi | ty[u], p.idesc, s0 + u > 0);
            if constexpr (PREC == MELT_BF16X3) {
              // hi*lo and lo*hi, in the order of the single-CTA kernel (bit-identical sums)
              mma_f16_pair(d, hi | (alo + tx[u]), hi | (ty[u] + bpart16), p.idesc, true);
              mma_f16_pair(d, hi | (alo + tx[u] + apart16), hi | ty[u], p.idesc, true);
            }
          }
        }
    }
    mma_commit_pair_mc(pbar(p, c, B.z_empty + zb), 3);
    mma_commit_pair_mc(pbar(p, c, B.t_full + acc), 3);
    if constexpr (DTC) {
      // the previous tile's DCT once its epilogues released its accumulator
      // (their log-Mel rows are in TMEM by then); this tile's projection is
      // already queued ahead of it
      if (k > 0) {
        const int pa = (k - 1) % nacc;
        if (!mbar_wait_cluster(pbar(p, c, B.t_empty + pa), ((k - 1) / nacc) & 1, c.abort, p.err, kErrTimeout)) {
          ok = false;
          break;
        }
        pair_dct_gemm(p, c, B, tmem_base);
      }
    }
    if constexpr (MLP) {
      // the previous tile's output layer, once its GELU(H) is written
      if (k > 0 && !pair_mlp_gemm2(p, c, B, tmem_base, k - 1)) {
        ok = false;
        break;
      }
    }
  }
  if constexpr (MLP) {
    // the last tile's MLP: wait for its x-hat (the release of its accumulator)
    if (ok && k > 0 &&
        mbar_wait_cluster(pbar(p, c, B.t_empty), (k - 1) & 1, c.abort, p.err, kErrTimeout)) {
      pair_mlp_gemm1(p, c, B, tmem_base);
      pair_mlp_gemm2(p, c, B, tmem_base, k - 1);
    }
  }
  if constexpr (DTC) {
    // the last tile's DCT
    if (ok && k > 0 &&
        mbar_wait_cluster(pbar(p, c, B.t_empty + (k - 1) % nacc), ((k - 1) / nacc) & 1, c.abort, p.err,
                          kErrTimeout))
      pair_dct_gemm(p, c, B, tmem_base);
  }
  // no pair MMA may still be running when either CTA releases TMEM
  mma_commit_pair_mc(pbar(p, c, B.drain), 3);
}

// Staged FP32 span chunks -> Z rows (bf16).  Chunk ch of a tile holds Z rows
// [ch*CH, ch*CH + rows) as contiguous FP32 samples, read as float4 "quads"
// (lanes read consecutive quads: conflict-free); quad hq is the low or high
// half (hq & 1) of the Z row segment (row ul, 8-sample group kc) with
// 8 * (hq >> 1) = (ul - ch*CH) H + 8 kc.
template <bool SPLIT, int CT = kPCvtThreads>
static __device__ void pair_convert(const TcParams& p, const PairCtx& c, const PairBars& B, int cvt0) {
  const int ct = threadIdx.x - 32 * cvt0;
  const int H8 = p.H >> 3;
  const int nq_full = p.CH * (p.H >> 2);
  uint32_t qoff[kPQuads];
  int qrow[kPQuads];
#pragma unroll
  for (int q = 0; q < kPQuads; ++q) {
    const int hq = ct + q * CT;
    const int il = hq >> 1;
    const int ull = il / H8;
    const int kc = il - ull * H8;
    qrow[q] = hq < nq_full ? ull : 1 << 30;
    qoff[q] = kc * p.lbo_a + ull * 16 + (hq & 1) * 8;
  }
  const uint32_t st0 = c.sbase + p.off_st;
  int slot = 0;
  uint32_t sphase = 0;
  for (int k = 0;; ++k) {
    bool okq = true;
    const int qp = k == 0 ? c.cluster : pair_next_warp(p, c, B, k, okq);
    if (!okq || qp >= p.n_pairs) break;
    const int zb = p.ZB == 2 ? (k & 1) : 0;
    if (!warp_wait_cl(pbar(p, c, B.z_empty + zb), ((p.ZB == 2 ? (k >> 1) : k) & 1) ^ 1, c.abort,
                      p.err))
      break;
    const TileDesc td = pair_tile(p, c, qp);
    const int nsamp = td.n_samples;
    const uint32_t zaddr = c.sbase + p.off_a + zb * p.abuf_bytes;
    bool ok = true;
    for (int ch = 0; td.n_frames > 0 && ch < p.NCHUNK; ++ch) {
      if (!warp_wait(pbar(p, c, B.s_full + slot), sphase, c.abort, p.err)) {
        ok = false;
        break;
      }
      const int rows = min(p.CH, p.zrows - ch * p.CH);
      const uint32_t st = st0 + slot * p.st_bytes;
      const int s_base = ch * p.CH * p.H;
      const uint32_t zrow0 = zaddr + ch * p.CH * 16;
      const bool tail = s_base + rows * p.H > nsamp;
      float4 x[kPQuads];
#pragma unroll
      for (int q = 0; q < kPQuads; ++q)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(x[q].x), "=f"(x[q].y), "=f"(x[q].z), "=f"(x[q].w)
                     : "r"(st + 16u * min(ct + q * CT, nq_full - 1)));
      if (tail) {
#pragma unroll
        for (int q = 0; q < kPQuads; ++q) clip_quad(x[q], s_base + 4 * (ct + q * CT), nsamp);
      }
#pragma unroll
      for (int q = 0; q < kPQuads; ++q) {
        if (qrow[q] < rows) {
          const uint32_t h0 = pack_bf16(x[q].x, x[q].y), h1 = pack_bf16(x[q].z, x[q].w);
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(zrow0 + qoff[q]), "r"(h0), "r"(h1));
          if constexpr (SPLIT) {
            // split BF16: lo = rn(x - hi), the second part p.a_bytes further
            const uint32_t l0 = pack_bf16(x[q].x - __uint_as_float(h0 << 16), x[q].y - __uint_as_float(h0 & 0xffff0000u));
            const uint32_t l1 = pack_bf16(x[q].z - __uint_as_float(h1 << 16), x[q].w - __uint_as_float(h1 & 0xffff0000u));
            asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(zrow0 + qoff[q] + p.a_bytes), "r"(l0), "r"(l1));
          }
        }
      }
      warp_arrive(pbar(p, c, B.s_empty + slot));
      if (++slot == p.NS) {
        slot = 0;
        sphase ^= 1;
      }
    }
    if (!ok) break;
    fence_proxy_async();
    warp_arrive_leader(pbar(p, c, B.z_full + zb));
  }
}

// UE8M0 exponent of the scale of a Z row whose max |x| has float bits `bits`:
// the least e with amax 2^-e <= 448 (amax = m 2^E, m in [1, 2): e = E - 8,
// one more when m > 1.75), at least -127; -127 for an all-zero or subnormal
// row.  Returns the code e + 127 (0..247).
static __device__ __forceinline__ uint32_t fp8_row_code(uint32_t bits) {
  const int ef = (int)(bits >> 23);
  const int e = max(-127, ef - 127 - 8 + ((bits & 0x7FFFFFu) > 0x600000u ? 1 : 0));
  return ef == 0 ? 0u : (uint32_t)(e + 127);
}

// Shared-memory stores under a predicate, without a branch.
static __device__ __forceinline__ void sts32_if(uint32_t addr, uint32_t v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %2, 0;\n\t"
      "@p st.shared.b32 [%0], %1;\n\t}" ::"r"(addr),
      "r"(v), "r"((uint32_t)pred)
      : "memory");
}

static __device__ __forceinline__ void sts8_if(uint32_t addr, uint32_t v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %2, 0;\n\t"
      "@p st.shared.u8 [%0], %1;\n\t}" ::"r"(addr),
      "r"(v), "r"((uint32_t)pred)
      : "memory");
}

// The samples of a quad at or past the clip end set to zero, by selects (s =
// clip sample index of x.x).
static __device__ __forceinline__ float4 clip_quad_sel(float4 x, int s, int nsamp) {
  x.x = s < nsamp ? x.x : 0.f;
  x.y = s + 1 < nsamp ? x.y : 0.f;
  x.z = s + 2 < nsamp ? x.z : 0.f;
  x.w = s + 3 < nsamp ? x.w : 0.f;
  return x;
}

// FP8 e4m3 converter: staged FP32 chunks -> polyphase Z rows of e4m3 with a
// power-of-two scale per row, and the rows' scale codes in TMEM.
//
// Eight lanes share a Z row: lane l8 of a group holds quads l8, l8 + 8, ...
// of the row (H <= 256: at most 8 each), so the row's max |x| is a local max
// and three butterfly shuffles inside the group.  A warp takes four rows at a
// time and both of its row sets of a chunk (rows 4 w + g and 4 w + g + 16,
// chunks of at most 32 rows) at once: all of a chunk's loads are in flight
// together and the two reductions overlap.  The row's exponent is the least
// e with amax 2^-e <= 448; its samples are multiplied by 2^-e (exact) and
// converted with saturating round-to-nearest-even.  Z element (u, r) sits at
// (r / 16) lbo_a + 16 u + r % 16, so quad q of row u is 4 bytes at core
// column q / 4, byte 4 (q % 4).  The row's scale code goes to shared memory;
// after the tile's last chunk each warp writes, for the 32 TMEM lanes of its
// quarter (frame t), one 32-bit word per group of four slices: byte j is the
// code of Z row t + 4g + j, the scale of A row t in slice 4g + j, repeated
// over the group's four columns (the MMA reads row t's scale in lane t,
// column t / 32 of the group).
constexpr int kF8LanesPerRow = 8;
constexpr int kF8MaxQuads = 8;   // quads per lane per row: H <= 4 * 8 * 8 = 256
constexpr int kF8MaxRows = 32;   // rows per staged chunk: two sets of 4 rows per warp

// One staged chunk of the FP8 converter (rows [r0, r0 + rows) of the tile's
// Z rows): NQ = quads per lane per row (ceil(H / 32)), a compile-time count
// so that every load is issued unconditionally and all are in flight at once.
template <int NQ, int CW>
static __device__ __forceinline__ void fp8_convert_chunk(const TcParams& p, uint32_t st, uint32_t zaddr,
                                                         uint32_t codes_s, int r0, int rows, int nsamp, int cw,
                                                         int g, int l8) {
  constexpr int NS = kF8MaxRows / (4 * CW);  // row sets per warp: rows 4 cw + g + 4 CW h
  const int h4 = p.H >> 2;
  const int s_base = r0 * p.H;
  const bool tail = s_base + rows * p.H > nsamp;
  // loads at clamped (always valid) addresses; quads outside the chunk's rows
  // or past H are zeroed by selects after
  float4 x[NS][NQ];
#pragma unroll
  for (int h = 0; h < NS; ++h) {
    const int u = min(4 * cw + g + 4 * CW * h, rows - 1);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(x[h][q].x), "=f"(x[h][q].y), "=f"(x[h][q].z), "=f"(x[h][q].w)
                   : "r"(st + 16u * (uint32_t)(u * h4 + min(kF8LanesPerRow * q + l8, h4 - 1))));
  }
  float m[NS];
#pragma unroll
  for (int h = 0; h < NS; ++h) {
    const int u = 4 * cw + g + 4 * CW * h;
    m[h] = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int j = kF8LanesPerRow * q + l8;
      const bool live = u < rows && j < h4;
      float4 v = x[h][q];
      if (tail) v = clip_quad_sel(v, s_base + u * p.H + 4 * j, nsamp);
      v.x = live ? v.x : 0.f;
      v.y = live ? v.y : 0.f;
      v.z = live ? v.z : 0.f;
      v.w = live ? v.w : 0.f;
      x[h][q] = v;
      m[h] = fmaxf(m[h], fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
  }
#pragma unroll
  for (int o = 1; o < kF8LanesPerRow; o <<= 1)
#pragma unroll
    for (int h = 0; h < NS; ++h) m[h] = fmaxf(m[h], __shfl_xor_sync(0xffffffffu, m[h], o));
#pragma unroll
  for (int h = 0; h < NS; ++h) {
    const int u = 4 * cw + g + 4 * CW * h;
    const bool row_live = u < rows;
    const uint32_t code = fp8_row_code(__float_as_uint(m[h]));
    const float inv = __uint_as_float((254u - code) << 23);  // 2^-e, e = code - 127
    sts8_if(codes_s + (uint32_t)(r0 + u), code, row_live && l8 == 0);
    const uint32_t zrow = zaddr + 16u * (uint32_t)(r0 + u);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int j = kF8LanesPerRow * q + l8;
      const uint32_t w = pack_e4m3x4(x[h][q].x * inv, x[h][q].y * inv, x[h][q].z * inv, x[h][q].w * inv);
      sts32_if(zrow + (uint32_t)(j >> 2) * p.lbo_a + 4u * (uint32_t)(j & 3), w, row_live && j < h4);
    }
  }
}

template <int CW>
static __device__ __forceinline__ void fp8_convert_chunk_any(const TcParams& p, int nqr, uint32_t st, uint32_t zaddr,
                                                             uint32_t codes_s, int r0, int rows, int nsamp, int cw,
                                                             int g, int l8) {
  switch (nqr) {
    case 1: fp8_convert_chunk<1, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
    case 2: fp8_convert_chunk<2, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
    case 3: fp8_convert_chunk<3, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
    case 4: fp8_convert_chunk<4, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
    case 5: fp8_convert_chunk<5, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
    case 6: fp8_convert_chunk<6, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
    case 7: fp8_convert_chunk<7, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
    default: fp8_convert_chunk<8, CW>(p, st, zaddr, codes_s, r0, rows, nsamp, cw, g, l8); break;
  }
}

template <int CW>
static __device__ void pair_convert_fp8(const TcParams& p, uint8_t* gbase, const PairCtx& c,
                                        const PairBars& B, int cvt0, uint32_t tmem_base) {
  constexpr int kThr = 32 * CW;
  const int cw = (int)(threadIdx.x >> 5) - cvt0, lane = threadIdx.x & 31;
  const int quarter = (threadIdx.x >> 5) & 3;  // the TMEM lanes this warp may access
  const int g = lane >> 3, l8 = lane & 7;
  const int h4 = p.H >> 2;                     // quads per Z row
  const int nqr = (h4 + kF8LanesPerRow - 1) / kF8LanesPerRow;  // quads per lane per row
  const uint32_t st0 = c.sbase + p.off_st;
  uint8_t* codes_all = gbase + p.off_codes;
  // zero both A buffers once: bytes past H in a row's last core columns stay zero
  for (uint32_t o = 16u * (uint32_t)(threadIdx.x - 32 * cvt0); o < p.abuf_bytes * p.ZB; o += 16u * kThr)
    sts128(c.sbase + p.off_a + o, make_uint4(0u, 0u, 0u, 0u));
  fence_proxy_async();
  int slot = 0;
  uint32_t sphase = 0;
  for (int k = 0;; ++k) {
    bool okq = true;
    const int qp = k == 0 ? c.cluster : pair_next_warp(p, c, B, k, okq);
    // every converter warp reads the same entry and takes every named barrier
    // below, or none: a timeout in any of them stops all of them here
    if (!named_barrier_and(1, kThr, okq) || qp >= p.n_pairs) break;
    const int zb = p.ZB == 2 ? (k & 1) : 0;
    bool ok = warp_wait_cl(pbar(p, c, B.z_empty + zb), ((p.ZB == 2 ? (k >> 1) : k) & 1) ^ 1, c.abort, p.err);
    const TileDesc td = pair_tile(p, c, qp);
    const int nsamp = td.n_samples;
    const uint32_t zaddr = c.sbase + p.off_a + zb * p.abuf_bytes;
    uint8_t* codes = codes_all + zb * p.codes_stride;
    const uint32_t codes_s = smem_u32(codes);
    for (int ch = 0; ok && td.n_frames > 0 && ch < p.NCHUNK; ++ch) {
      if (!warp_wait(pbar(p, c, B.s_full + slot), sphase, c.abort, p.err)) {
        ok = false;
        break;
      }
      const int r0 = ch * p.CH;
      fp8_convert_chunk_any<CW>(p, nqr, st0 + slot * p.st_bytes, zaddr, codes_s, r0, min(p.CH, p.zrows - r0),
                                nsamp, cw, g, l8);
      warp_arrive(pbar(p, c, B.s_empty + slot));
      if (++slot == p.NS) {
        slot = 0;
        sphase ^= 1;
      }
    }
    // all leave together when a wait gave up; otherwise every row's code is in
    // shared memory: the scale words of this warp's TMEM lanes
    if (!named_barrier_and(1, kThr, ok)) break;
    if (td.n_frames > 0 && cw < 4) {  // one warp per TMEM lane quarter
      const int t = 32 * quarter + lane;
      for (int gg = 0; gg < p.sfg; ++gg) {
        uint32_t w = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int jj = 4 * gg + j;
          w |= (jj < p.J ? (uint32_t)codes[t + jj] : 0x7Fu) << (8 * j);
        }
        tmem_st4(tmem_base + ((uint32_t)(32 * quarter) << 16) + p.sf_col + (uint32_t)(4 * (p.sfg * zb + gg)), w);
      }
      tmem_st_wait();
    }
    tc_fence_before();
    fence_proxy_async();
    warp_arrive_leader(pbar(p, c, B.z_full + zb));
  }
}

// Columns of a row split between the warps that share a lane quarter: with
// two, 16-column chunks [lo, hi) of n for half h (the first half takes the
// odd one); with one, all of them.
static __device__ __forceinline__ void half_chunks(int n, int halves, int h, int& lo, int& hi) {
  const int first = halves == 2 ? (n + 1) / 2 : n;
  lo = h ? first : 0;
  hi = h ? n : first;
}

// MFCC epilogue with the DCT on the tensor cores: per tile, the log-Mel row
// (Eq. 8) of this warp's chunks goes to TMEM as BF16 hi and lo parts (the A
// operand of the DCT MMAs), the accumulator is released, and once the DCT's
// commit arrives the coefficients (Eq. 9) are read back and stored.  Empty
// tiles take every step but the loads and stores, so that both CTAs keep the
// barrier phases in step.
template <int EPW>
__device__ void pair_epilogue_dct(const TcParams& p, const PairCtx& c, const PairBars& B, uint32_t tmem_base) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = 32 * quarter + lane;
  const bool vec8 = ((p.n_mfcc & 7) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 31) == 0);
  const uint32_t tl = tmem_base + ((uint32_t)(32 * quarter) << 16);
  int c_lo, c_hi, k_lo, k_hi;
  half_chunks(p.MP >> 4, EPW / 4, half, c_lo, c_hi);
  half_chunks(p.dct_n >> 4, EPW / 4, half, k_lo, k_hi);
  for (int k = 0;; ++k) {
    bool okq = true;
    const int q = k == 0 ? c.cluster : pair_next_warp(p, c, B, k, okq);
    if (!okq || q >= p.n_pairs) break;
    const int acc = p.nacc == 2 ? (k & 1) : 0;
    const uint32_t tphase = p.nacc == 2 ? ((k >> 1) & 1) : (k & 1);
    const TileDesc td = pair_tile(p, c, q);
    if (!warp_wait_cl(pbar(p, c, B.t_full + acc), tphase, c.abort, p.err)) break;
    sched_release(p, c, B, k);
    tc_fence_after();
    const bool live = td.n_frames > 0;
    const uint32_t t0 = tl + acc * p.acc_stride;
    if (live) {
#pragma unroll 1
      for (int c0 = c_lo; c0 < c_hi; c0 += kEpiGroup) {
        float re[kEpiGroup][16], im[kEpiGroup][16];
#pragma unroll
        for (int g = 0; g < kEpiGroup; ++g) {
          if (c0 + g < c_hi) {
            tmem_ld16(t0 + 16 * (c0 + g), re[g]);
            tmem_ld16(t0 + p.MP + 16 * (c0 + g), im[g]);
          }
        }
        tmem_ld_wait();
#pragma unroll
        for (int g = 0; g < kEpiGroup; ++g) {
          reg_fence16(re[g]);
          reg_fence16(im[g]);
          const int cc = c0 + g;
          if (cc < c_hi) {
            uint32_t wh[8], wl[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              // bins past M hold zero basis rows: their log is replaced by 0
              const int m = 16 * cc + 2 * e;
              const float a = m < p.M ? fast_ln(fmaf(re[g][2 * e], re[g][2 * e], fmaf(im[g][2 * e], im[g][2 * e], p.eps))) : 0.f;
              const float b = m + 1 < p.M
                                  ? fast_ln(fmaf(re[g][2 * e + 1], re[g][2 * e + 1],
                                                fmaf(im[g][2 * e + 1], im[g][2 * e + 1], p.eps)))
                                  : 0.f;
              wh[e] = pack_bf16(a, b);
              wl[e] = pack_bf16(a - __uint_as_float(wh[e] << 16), b - __uint_as_float(wh[e] & 0xFFFF0000u));
            }
            tmem_st8(tl + p.dct_ahi + 8 * cc, wh);
            tmem_st8(tl + p.dct_alo + 8 * cc, wl);
          }
        }
      }
      tmem_st_wait();
    }
    tc_fence_before();
    warp_arrive_leader(pbar(p, c, B.t_empty + acc));
    if (!warp_wait_cl(pbar(p, c, B.h_full), k & 1, c.abort, p.err)) break;
    tc_fence_after();
    if (live) {
      float* orow = p.out + (size_t)(td.out_row + row) * p.n_mfcc;
      const bool valid = row < td.n_frames;
#pragma unroll 1
      for (int kc = k_lo; kc < k_hi; ++kc) {
        float v[16];
        tmem_ld16(tl + p.dct_c + 16 * kc, v);
        tmem_ld_wait();
        reg_fence16(v);
        if (valid) {
          if (vec8 && 16 * kc + 16 <= p.n_mfcc) {
            stg256(orow + 16 * kc, v);
            stg256(orow + 16 * kc + 8, v + 8);
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (16 * kc + e < p.n_mfcc) orow[16 * kc + e] = v[e];
          }
        }
      }
    }
  }
}

template <int NCH, bool MFCC, int EPW, int PREC>
__device__ void pair_epilogue(const TcParams& p, uint8_t* gbase, const PairCtx& c, const PairBars& B,
                              uint32_t tmem_base) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = 32 * quarter + lane;
  const float* dct = reinterpret_cast<const float*>(gbase + p.off_dct);
  const bool vec8 = ((p.n_out & 7) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 31) == 0);
  const bool vec4 = ((p.n_out & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 15) == 0);
  const int nch = p.MP >> 4;
  int c_lo, c_hi;
  half_chunks(nch, EPW / 4, half, c_lo, c_hi);
  constexpr float sc = 1.f;  // every form's accumulator holds R and I (FP8: scaled by the MMA)
  for (int k = 0;; ++k) {
    bool okq = true;
    const int q = k == 0 ? c.cluster : pair_next_warp(p, c, B, k, okq);
    if (!okq || q >= p.n_pairs) break;
    const int acc = p.nacc == 2 ? (k & 1) : 0;
    const uint32_t tphase = p.nacc == 2 ? ((k >> 1) & 1) : (k & 1);
    const TileDesc td = pair_tile(p, c, q);
    if (!warp_wait_cl(pbar(p, c, B.t_full + acc), tphase, c.abort, p.err)) break;
    sched_release(p, c, B, k);
    tc_fence_after();
    const bool valid = row < td.n_frames;
    const uint32_t t0 = tmem_base + ((uint32_t)(32 * quarter) << 16) + acc * p.acc_stride;
    float* orow = p.out + (size_t)(td.out_row + row) * p.n_out;
    // an empty tile: no reads
    if (td.n_frames == 0) {
      tc_fence_before();
      warp_arrive_leader(pbar(p, c, B.t_empty + acc));
      continue;
    }
    if constexpr (!MFCC) {
#pragma unroll 1
      for (int c0 = c_lo; c0 < c_hi; c0 += kEpiGroup) {
        float re[kEpiGroup][16], im[kEpiGroup][16];
#pragma unroll
        for (int g = 0; g < kEpiGroup; ++g) {
          if (c0 + g < c_hi) {
            tmem_ld16(t0 + 16 * (c0 + g), re[g]);
            tmem_ld16(t0 + p.MP + 16 * (c0 + g), im[g]);
          }
        }
        tmem_ld_wait();
#pragma unroll
        for (int g = 0; g < kEpiGroup; ++g) {
          reg_fence16(re[g]);
          reg_fence16(im[g]);
        }
        if (c0 + kEpiGroup >= c_hi) {
          tc_fence_before();
          warp_arrive_leader(pbar(p, c, B.t_empty + acc));
        }
#pragma unroll
        for (int g = 0; g < kEpiGroup; ++g) {
          const int cc = c0 + g;
          if (cc < c_hi) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float r = re[g][e] * sc, i = im[g][e] * sc;
              re[g][e] = fast_ln(fmaf(r, r, fmaf(i, i, p.eps)));
            }
            if (valid) {
              if (vec8 && 16 * cc + 16 <= p.M) {
                stg256(orow + 16 * cc, re[g]);
                stg256(orow + 16 * cc + 8, re[g] + 8);
              } else {
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (16 * cc + e < p.M) orow[16 * cc + e] = re[g][e];
              }
            }
          }
        }
      }
      if (c_lo >= c_hi) {  // nothing to read (a single-chunk row goes to the first half)
        tc_fence_before();
        warp_arrive_leader(pbar(p, c, B.t_empty + acc));
      }
    } else {
      float lm[16 * NCH];
#pragma unroll
      for (int cc = 0; cc < NCH; ++cc) {
        float re[16], im[16];
        tmem_ld16(t0 + 16 * cc, re);
        tmem_ld16(t0 + 16 * NCH + 16 * cc, im);
        tmem_ld_wait(re, im);
#pragma unroll
        for (int e = 0; e < 16; ++e)
          lm[16 * cc + e] =
              (16 * cc + e < p.M) ? fast_ln(fmaf(re[e] * sc, re[e] * sc, (im[e] * sc) * (im[e] * sc)) + p.eps) : 0.f;
      }
      tc_fence_before();
      warp_arrive_leader(pbar(p, c, B.t_empty + acc));
      // the two warps of a lane quarter (EPW = 8) each read the whole row and
      // take alternate groups of four coefficients
#pragma unroll 1
      for (int kk0 = 4 * half; kk0 < p.n_mfcc; kk0 += 4 * (EPW / 4)) {
        const float4 v = dct_quad<NCH>(lm, dct, kk0);
        if (valid) store_quad(orow, kk0, p.n_mfcc, v, vec4);
      }
    }
  }
}

// GELU(h) = h Phi(h), the exact-erf form the model is trained with, for the
// fused epilogue, whose result is rounded to BF16 (8 significant bits).
// With t = |h| and Q(t) = 1 - Phi(t) the upper normal tail,
//     GELU(h) = max(h, 0) - t Q(t),   log2 Q(t) = -t^2 log2(e) / 2 + S(t),
// where S (log2 of the Mills ratio over sqrt(2 pi)) is smooth on [0, 5],
// from -1 at t = 0 to about -3.7 at t = 5.  S is a degree-6 polynomial in
// u = 0.4 t - 1: the Chebyshev fit on [0, 5] refined towards minimax by
// Lawson reweighting (30 passes on a 4e5-point grid), in the power basis
// rounded to float32; Q = 2^(S - t^2 log2(e) / 2) from the hardware base-2
// exponential.  Against the exact function (float64) the float32 evaluation
// has a relative error <= 2e-5 for |h| <= 5 (about 2^-16, far below half a
// BF16 ulp) and an absolute error <= 3e-6 everywhere (S is taken at
// min(t, 5): beyond, the tail is below 1.5e-6 in magnitude).  About a dozen
// FP32 operations and one multi-function-unit operation (the degree-9 fit of
// the Mills ratio it replaces took 17).
static __device__ __forceinline__ float gelu_poly(float h) {
  const float t = fabsf(h);
  const float u = fmaf(0.4f, fminf(t, 5.f), -1.f);
  float r = 7.192788180e-03f;
  r = fmaf(r, u, -2.606392093e-02f);
  r = fmaf(r, u, 6.437100470e-02f);
  r = fmaf(r, u, -1.599922627e-01f);
  r = fmaf(r, u, 4.010236561e-01f);
  r = fmaf(r, u, -1.164181113e+00f);
  r = fmaf(r, u, -2.822842598e+00f);
  float q;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(fmaf(t * -0.72134752044448170f, t, r)));  // Q(t)
  return fmaf(-t, q, fmaxf(h, 0.f));
}

// GELU(H + b1) of hidden chunk cc (16 units, in h) to BF16 over H at TMEM
// address `to` (gelu_col: the chunk's warp starts its run at lo, to = lanes +
// h_col + 8 (cc + lo)).
static __device__ __forceinline__ void gelu_chunk(uint32_t to, const float* b1, int cc, const float (&h)[16]) {
  const float4* b4 = reinterpret_cast<const float4*>(b1 + 16 * cc);  // 16-byte aligned
  float bb[16];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float4 q = b4[v];
    bb[4 * v] = q.x;
    bb[4 * v + 1] = q.y;
    bb[4 * v + 2] = q.z;
    bb[4 * v + 3] = q.w;
  }
  uint32_t w[8];
#pragma unroll
  for (int e = 0; e < 8; ++e)
    w[e] = pack_bf16(gelu_poly(h[2 * e] + bb[2 * e]), gelu_poly(h[2 * e + 1] + bb[2 * e + 1]));
  tmem_st8(to, w);
}

// The fused-MLP epilogue's log-Mel (Eq. 8) of this warp's band chunks of
// the row, from the projection accumulator into v (one chunk per wait).
template <int NV>
static __device__ __forceinline__ void mlp_logmel(const TcParams& p, uint32_t tl, int c_lo, int c_hi,
                                                  float (&v)[16 * NV]) {
#pragma unroll
  for (int g = 0; g < NV; ++g) {
    if (c_lo + g < c_hi) {
      const int cc = c_lo + g;
      float re[16], im[16];
      tmem_ld16(tl + 16 * cc, re);
      tmem_ld16(tl + p.MP + 16 * cc, im);
      tmem_ld_wait(re, im);
#pragma unroll
      for (int e = 0; e < 16; ++e) v[16 * g + e] = fast_ln(fmaf(re[e], re[e], fmaf(im[e], im[e], p.eps)));
    }
  }
}

// Epilogue with the fused correction MLP.  Per pair step k: x-hat of the
// row (BF16) into TMEM and the accumulator released; once the hidden layer
// is in, x + b2 into the output columns (over x-hat) and GELU(H + b1) over
// H; while the output layer runs, the log-Mel of step k + 1 from its
// accumulator into registers; then the output layer's sum
// x + b2 + GELU(H) W2^T stored.  The kMlpParts warps of a lane quarter
// split the bands (part_lo) and the hidden units (part_lo_tail).  Every step is taken for an empty tile too
// (without loads or stores) so that both CTAs keep the barrier phases in
// step.
template <int NCH>
__device__ void pair_epilogue_mlp(const TcParams& p, uint8_t* gbase, const PairCtx& c, const PairBars& B,
                                  uint32_t tmem_base) {
  constexpr int NV = (NCH + kMlpParts - 1) / kMlpParts;  // band chunks of the largest part
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, part = warp >> 2;
  const int row = 32 * quarter + lane;
  const float* vec = reinterpret_cast<const float*>(gbase + p.off_mlp + p.mlp_vec_off);
  const float* b1 = vec;                 // [Hd]
  const float* b2 = vec + p.Hd;          // [MP]
  const float* mu = b2 + p.MP;           // [MP]
  const float* isd = mu + p.MP;          // [MP]
  const bool vec8 = ((p.n_out & 7) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 31) == 0);
  const uint32_t tl = tmem_base + ((uint32_t)(32 * quarter) << 16);  // this warp's lanes
  const int c_lo = part_lo(NCH, kMlpParts, part), c_hi = part_lo(NCH, kMlpParts, part + 1);
  const int h_lo = part_lo_tail(p.Hd / 16, kMlpParts, part), h_hi = part_lo_tail(p.Hd / 16, kMlpParts, part + 1);
  if (c.cluster >= p.n_pairs) return;
  TileDesc td = pair_tile(p, c, c.cluster);
  if (!warp_wait_cl(pbar(p, c, B.t_full), 0, c.abort, p.err)) return;
  tc_fence_after();
  bool live = td.n_frames > 0;
  float v[16 * NV];
  if (live) mlp_logmel<NV>(p, tl, c_lo, c_hi, v);
  for (int k = 0;; ++k) {
    const bool valid = row < td.n_frames;
    float* orow = p.out + (size_t)(td.out_row + row) * p.n_out;
    // 1. x-hat in BF16 into TMEM (chunk cc over the first half of the
    // output's chunk cc, which this warp has read back) and x + b2 of the
    // chunk's upper 8 bands into its second half (GEMM1 reads only the
    // first); the accumulator released
    if (live) {
#pragma unroll
      for (int g = 0; g < NV; ++g) {
        const int cc = c_lo + g;
        if (cc < c_hi) {
          uint32_t w[8], r1[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int m = 16 * cc + 2 * e;
            w[e] = pack_bf16((v[16 * g + 2 * e] - mu[m]) * isd[m], (v[16 * g + 2 * e + 1] - mu[m + 1]) * isd[m + 1]);
            r1[e] = __float_as_uint(v[16 * g + 8 + e] + b2[16 * cc + 8 + e]);
          }
          tmem_st8(tl + p.a1_col + 16 * cc, w);
          tmem_st8(tl + p.y_col + 16 * cc + 8, r1);
        }
      }
      tmem_st_wait();
    }
    tc_fence_before();
    warp_arrive_leader(pbar(p, c, B.t_empty));
    // 2. once H is in (x-hat consumed): x + b2 of the lower 8 bands into the
    // output columns (over x-hat), then GELU(H + b1) in BF16 over H (see
    // gelu_col), the next chunk's load in flight while one chunk is evaluated
    if (!warp_wait_cl(pbar(p, c, B.h_full), k & 1, c.abort, p.err)) break;
    tc_fence_after();
    if (live) {
      float ha[16], hb[16];
      tmem_ld16(tl + p.h_col + 16 * h_lo, ha);  // (every part has hidden chunks)
#pragma unroll
      for (int g = 0; g < NV; ++g) {
        const int cc = c_lo + g;
        if (cc < c_hi) {
          uint32_t r0[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) r0[e] = __float_as_uint(v[16 * g + e] + b2[16 * cc + e]);
          tmem_st8(tl + p.y_col + 16 * cc, r0);
        }
      }
      tmem_ld_wait();
      reg_fence16(ha);
#pragma unroll 1
      for (int cc = h_lo; cc < h_hi; cc += 2) {
        // chunk cc in ha; chunk cc + 1 loads into hb meanwhile
        if (cc + 1 < h_hi) tmem_ld16(tl + p.h_col + 16 * (cc + 1), hb);
        gelu_chunk(tl + p.h_col + 8u * (uint32_t)(cc + h_lo), b1, cc, ha);
        if (cc + 1 >= h_hi) break;
        tmem_ld_wait();
        reg_fence16(hb);
        // chunk cc + 1 in hb; chunk cc + 2 loads into ha meanwhile
        if (cc + 2 < h_hi) tmem_ld16(tl + p.h_col + 16 * (cc + 2), ha);
        gelu_chunk(tl + p.h_col + 8u * (uint32_t)(cc + 1 + h_lo), b1, cc + 1, hb);
        tmem_ld_wait();
        reg_fence16(ha);
      }
      tmem_st_wait();
    }
    tc_fence_before();
    warp_arrive_leader(pbar(p, c, B.a2_full));
    // 3. while the output layer runs: the next step's pair, and its log-Mel
    // (its projection was queued right after this step's hidden layer)
    bool okq = true;
    const int qn = pair_next_warp(p, c, B, k + 1, okq);
    const bool more = okq && qn < p.n_pairs;
    TileDesc tn = td;
    bool live_n = false;
    if (more) {
      tn = pair_tile(p, c, qn);
      if (!warp_wait_cl(pbar(p, c, B.t_full), (k + 1) & 1, c.abort, p.err)) break;
      sched_release(p, c, B, k + 1);
      tc_fence_after();
      live_n = tn.n_frames > 0;
      if (live_n) mlp_logmel<NV>(p, tl, c_lo, c_hi, v);  // (this step's v is in TMEM as x + b2)
    }
    // 4. the output layer's sum for this warp's bands
    if (!warp_wait_cl(pbar(p, c, B.y_full), k & 1, c.abort, p.err)) break;
    tc_fence_after();
    if (live) {
#pragma unroll
      for (int g = 0; g < NV; ++g) {
        const int cc = c_lo + g;
        if (cc < c_hi) {
          float y[16];
          tmem_ld16(tl + p.y_col + 16 * cc, y);
          tmem_ld_wait();
          reg_fence16(y);
          if (valid) {
            if (vec8 && 16 * cc + 16 <= p.M) {
              stg256(orow + 16 * cc, y);
              stg256(orow + 16 * cc + 8, y + 8);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (16 * cc + e < p.M) orow[16 * cc + e] = y[e];
            }
          }
        }
      }
    }
    if (!more) break;
    td = tn;
    live = live_n;
  }
}

// The work of one CTA of a pair kernel: cluster `cluster` of `n_clusters`
// clusters that share the tile list of `p`.
template <int NCH, bool MFCC, bool MLP, int PREC, bool DTC>
__device__ __forceinline__ void pair_cta(const TcParams& p, int cluster, int n_clusters) {
  constexpr int EPW = pair_epi_warps(MLP, MFCC, NCH, DTC);
  // (fused MLP: the basis producer on lane 1 of the MMA warp)
  constexpr int kPMmaWarp = EPW, kPBWarp = MLP ? EPW : EPW + 1, kPProdWarp = kPBWarp + 1, kPCvtWarp0 = kPProdWarp + 1;
  constexpr int CW = pair_cvt_warps(PREC, MFCC, NCH, DTC, MLP);
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 127u) & ~127u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PairBars B(p.NS, p.ZB, p.KS, p.b_resident ? 0 : p.NB);
  PairCtx c;
  c.sbase = sbase;
  c.rank = cluster_ctarank();
  c.cluster = cluster;
  c.n_clusters = n_clusters;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + p.off_misc);
  c.abort = reinterpret_cast<volatile int*>(gbase + p.off_misc + 4);

  if (threadIdx.x == 0) {
    auto bar = [&](int i) { return sbase + p.off_bar + 8 * i; };
    for (int i = 0; i < p.NS; ++i) {
      mbar_init(bar(B.s_full + i), 1);
      mbar_init(bar(B.s_empty + i), CW);
    }
    for (int i = 0; i < p.ZB; ++i) {
      mbar_init(bar(B.z_full + i), 2 * CW);  // converters of both CTAs (even CTA's copy is used)
      mbar_init(bar(B.z_empty + i), 1);
    }
    mbar_init(bar(B.b_full), 1);
    mbar_init(bar(B.peer_b), 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(B.t_full + i), 1);
      mbar_init(bar(B.t_empty + i), 2 * EPW);  // epilogues of both CTAs
    }
    mbar_init(bar(B.h_full), 1);
    mbar_init(bar(B.a2_full), 2 * EPW);
    mbar_init(bar(B.y_full), 1);
    mbar_init(bar(B.drain), 1);
    for (int i = 0; i < kSchedRing; ++i) {
      mbar_init(bar(B.sched_full + i), 1);           // the even CTA's producer (here or remote)
      mbar_init(bar(B.sched_empty + i), 2 * EPW);    // epilogues of both CTAs (even CTA's copy is used)
    }
    for (int i = 0; i < (p.b_resident ? 0 : p.NB); ++i) {
      mbar_init(bar(B.bs_full + i), 1);   // this CTA's producer (expect_tx)
      mbar_init(bar(B.bs_peer + i), 1);   // the odd CTA's signal (even CTA's copy is used)
      mbar_init(bar(B.bs_empty + i), 1);  // the even CTA's multicast commit
    }
    *c.abort = 0;
    fence_mbar_init();
  }
  if (warp == kPBWarp) {
    // K-step table: A start offset (16-byte units, polyphase j-shift) and B low word
    uint2* tab = reinterpret_cast<uint2*>(gbase + p.off_tab);
    const uint32_t b_lo0 = ((sbase + p.off_b) >> 4) | ((p.b_lbo >> 4) << 16);
    const uint32_t step16 = p.step_bytes >> 4;
    // steps in (slice j, K-group kk) order, the order of the basis image; a
    // K-step is 16 samples (BF16) or 32 (FP8, which also keeps j in bits 24..31
    // of the A entry for the scale-factor selection)
    constexpr int kstep = PREC == MELT_FP8E4M3 ? 32 : 16;
    for (int j = 0, s0 = 0; j < p.J; ++j) {
      const int steps = (min(p.H, p.N - j * p.H) + kstep - 1) / kstep;
      const uint32_t jtag = PREC == MELT_FP8E4M3 ? (uint32_t)j << 24 : 0u;
      for (int kk = lane; kk < steps; kk += 32)
        tab[s0 + kk] = make_uint2(((2u * kk * p.lbo_a + 16u * j) >> 4) | jtag, b_lo0 + (s0 + kk) * step16);
      s0 += steps;
    }
  }
  if (warp == kPMmaWarp) {
    tmem_alloc_pair(smem_u32(tmem_slot), p.tmem_cols);
    tmem_relinquish_pair();
  }
  if constexpr (MFCC) {
    if (warp < EPW) {
      if constexpr (DTC)
        fill_dct_split(p, gbase + p.off_dct, c.rank, threadIdx.x, 32 * EPW);
      else
        fill_dct(p, reinterpret_cast<float*>(gbase + p.off_dct), threadIdx.x, 32 * EPW);
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers exist before either arrives on the other's
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  if constexpr (PREC == MELT_FP8E4M3) {
    // scale-factor columns: every row scale 2^0 until the converters write a
    // tile's codes; the basis scale 2^-8 for good (the epilogue warps cover
    // the four lane quarters); both CTAs' columns are set before any MMA
    if (warp < 4) {
      const uint32_t tl = tmem_base + ((uint32_t)(32 * warp) << 16) + p.sf_col;
      const int na = 4 * p.sfg * p.ZB;
      for (int col = 0; col < na; col += 4) tmem_st4(tl + col, kSfOne);
      for (int col = 0; col < kSfBCols; col += 4) tmem_st4(tl + na + col, kSfBasis);
      tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
  }
  if (threadIdx.x == 0) pdl_launch_dependents();

  // MMA issuer and basis producer start at once (own data only; the basis
  // producer waits before it reads the fused MLP's weight image); the roles
  // that read tiles or the waveform, or write features, wait for the
  // previous kernel of the stream first (programmatic dependent launch).
  // With early_inputs (the caller stated that no kernel still in flight
  // writes the waveform) the waveform producer and the converters skip that
  // wait, so a launch fills and converts its first tiles while the previous
  // one drains; the epilogue, which stores features, always waits.
  if (warp == kPMmaWarp) {
    if (lane == 0) {
      if (c.rank == 0) pair_mma<MLP, PREC, DTC>(p, gbase, c, B, tmem_base);
      else if (!p.b_resident) pair_basis_signal(p, c, B);  // the odd CTA's slots, to the even CTA
      drain_wait(pbar(p, c, B.drain), 0, p.err);
    } else if (MLP && lane == 1) {
      pair_basis_producer(p, c, B);
    }
    __syncwarp();
  } else if (warp == kPBWarp) {
    if (lane == 0) pair_basis_producer(p, c, B);
    __syncwarp();
  } else if (warp == kPProdWarp) {
    if (!p.early_inputs) pdl_wait();
    if (lane == 0) pair_wave_producer(p, c, B);
    __syncwarp();
  } else if (warp >= kPCvtWarp0) {
    if (!p.early_inputs) pdl_wait();
    if constexpr (PREC == MELT_FP8E4M3)
      pair_convert_fp8<CW>(p, gbase, c, B, kPCvtWarp0, tmem_base);
    else
      pair_convert<PREC == MELT_BF16X3, 32 * CW>(p, c, B, kPCvtWarp0);
    __syncwarp();
  } else {
    pdl_wait();
    if constexpr (MLP)
      pair_epilogue_mlp<NCH>(p, gbase, c, B, tmem_base);
    else if constexpr (DTC)
      pair_epilogue_dct<EPW>(p, c, B, tmem_base);
    else
      pair_epilogue<NCH, MFCC, EPW, PREC>(p, gbase, c, B, tmem_base);
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (p.dyn && threadIdx.x == 0) {
    // every claim of this CTA is settled: the last CTA of the launch to get
    // here leaves the launch's counter at zero for the next launch that uses it
    __threadfence();
    if (atomicAdd(p.sched + 1, 1ull) == (unsigned long long)(2 * n_clusters) - 1) {
      atomicExch(p.sched, 0ull);
      atomicExch(p.sched + 1, 0ull);
    }
  }
  cluster_sync_all();  // neither CTA leaves (or frees TMEM) while its peer may still use it
  if (warp == kPMmaWarp) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, p.tmem_cols);
  }
}

template <int NCH, bool MFCC, bool MLP, int PREC = MELT_BF16, bool DTC = false>
__global__ void __launch_bounds__(pair_threads(MLP, PREC, MFCC, NCH, DTC), 1)
    melt_tc_pair_kernel(const __grid_constant__ TcParams p) {
  pair_cta<NCH, MFCC, MLP, PREC, DTC>(p, (int)(blockIdx.x >> 1), (int)(gridDim.x >> 1));
}

// Two bases in one persistent launch (the grouped call): clusters
// [0, split) work through the tiles of g[0], the others through those of
// g[1], each with its own geometry, shared-memory layout and TMEM size (the
// launch provides the larger shared-memory size).  Every tile is computed
// exactly as in its basis's own launch.
struct TcGroupParams {
  TcParams g[2];
  int split;
};

template <int NCH, bool MFCC, bool MLP, int PREC = MELT_BF16, bool DTC = false>
__global__ void __launch_bounds__(pair_threads(MLP, PREC, MFCC, NCH, DTC), 1)
    melt_tc_pair_group_kernel(const __grid_constant__ TcGroupParams q) {
  const int cl = (int)(blockIdx.x >> 1), nc = (int)(gridDim.x >> 1);
  const bool second = cl >= q.split;
  pair_cta<NCH, MFCC, MLP, PREC, DTC>(second ? q.g[1] : q.g[0], second ? cl - q.split : cl,
                                      second ? nc - q.split : q.split);
}

using GroupKernelFn = void (*)(TcGroupParams);
// Defined in melt_tc2.cu: the two-basis launch of the BF16 log-Mel pair kernel.
GroupKernelFn kernel_for_pair_group();

template <bool MFCC>
KernelFn pick_pair_kernel(int nch, bool dtc = false) {
  if constexpr (!MFCC) {
    (void)nch;
    (void)dtc;
    return melt_tc_pair_kernel<1, false, false>;
  } else {
    if (dtc) return melt_tc_pair_kernel<1, true, false, MELT_BF16, true>;
    switch (nch) {
      case 1: return melt_tc_pair_kernel<1, true, false>;
      case 2: return melt_tc_pair_kernel<2, true, false>;
      case 3: return melt_tc_pair_kernel<3, true, false>;
      case 4: return melt_tc_pair_kernel<4, true, false>;
      case 5: return melt_tc_pair_kernel<5, true, false>;
      case 6: return melt_tc_pair_kernel<6, true, false>;
      case 7: return melt_tc_pair_kernel<7, true, false>;
      case 8: return melt_tc_pair_kernel<8, true, false>;
      default: return nullptr;
    }
  }
}

// FP8 e4m3 instantiations (log-Mel, and MFCC by chunk count).  The pickers are
// templates so that only the translation unit that calls one instantiates
// its kernels.
template <int = 0>
KernelFn pick_pair_fp8_kernel(bool mfcc, int nch, bool dtc = false) {
  if (!mfcc) return melt_tc_pair_kernel<1, false, false, MELT_FP8E4M3>;
  if (dtc) return melt_tc_pair_kernel<1, true, false, MELT_FP8E4M3, true>;
  switch (nch) {
    case 1: return melt_tc_pair_kernel<1, true, false, MELT_FP8E4M3>;
    case 2: return melt_tc_pair_kernel<2, true, false, MELT_FP8E4M3>;
    case 3: return melt_tc_pair_kernel<3, true, false, MELT_FP8E4M3>;
    case 4: return melt_tc_pair_kernel<4, true, false, MELT_FP8E4M3>;
    case 5: return melt_tc_pair_kernel<5, true, false, MELT_FP8E4M3>;
    case 6: return melt_tc_pair_kernel<6, true, false, MELT_FP8E4M3>;
    case 7: return melt_tc_pair_kernel<7, true, false, MELT_FP8E4M3>;
    case 8: return melt_tc_pair_kernel<8, true, false, MELT_FP8E4M3>;
    default: return nullptr;
  }
}

// Split-BF16 (BF16x3) instantiation: log-Mel only.
template <int = 0>
KernelFn pick_pair_x3_kernel() {
  return melt_tc_pair_kernel<1, false, false, MELT_BF16X3>;
}

// Fused-MLP instantiations: log-Mel rows of 16 * nch bands (the fused TMEM
// layout holds M <= 80, so nch <= 5).
template <int = 0>
KernelFn pick_pair_mlp_kernel(int nch) {
  switch (nch) {
    case 1: return melt_tc_pair_kernel<1, false, true>;
    case 2: return melt_tc_pair_kernel<2, false, true>;
    case 3: return melt_tc_pair_kernel<3, false, true>;
    case 4: return melt_tc_pair_kernel<4, false, true>;
    case 5: return melt_tc_pair_kernel<5, false, true>;
    default: return nullptr;
  }
}

}  // namespace tc
}  // namespace melt
