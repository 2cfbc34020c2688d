// Host side of the tensor-core MelT kernels: basis operand images, the
// shared-memory plan and the launch.  The device code is in melt_tc_kernel.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "melt_tc2_kernel.cuh"

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
constexpr int kMaxCands = 512;

bool try_layout(const TcBasis* tb, TcParams& p, const melt_plan& c, int n_mfcc);
bool try_layout_pair(const TcBasis* tb, TcParams& p, const melt_plan& c, int n_mfcc);
int candidate_list(const TcBasis* tb, const TcParams& p, melt_plan* out, int cap);

uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// Shared-memory plan for one basis; false if it cannot fit.
bool plan_smem(const TcBasis* tb, TcParams& p, int n_mfcc) {
  const int P = tb->precision;
  p.N = tb->n_fft;
  p.H = tb->hop;
  p.M = tb->n_mels;
  p.MP = (p.M + 15) / 16 * 16;
  p.NC = 2 * p.MP;
  p.nblk = (p.MP + 127) / 128;  // accumulator blocks of 128 Mel bins (one when M <= 128)
  p.wbl = p.MP - 128 * (p.nblk - 1);
  p.J = tb->J;
  p.KS = tb->ksteps;
  p.zrows = kF + p.J - 1;
  p.nq = p.zrows * (p.H / 4);
  p.kstep_bytes = (uint32_t)tb->kstep_bytes;
  const int parts = P == MELT_BF16X3 ? 2 : 1;
  // A operand: the tile's Z rows in the K-major core-matrix layout, one core
  // column per 16 bytes of a row (8 BF16 or 16 e4m3 samples; FP8 rows are
  // padded to whole 32-sample K-steps)
  int zr = p.zrows;
  while ((zr & 7) != 1) ++zr;                  // rows % 8 == 1: converter stores spread banks
  p.lbo_a = (uint32_t)zr * 16;
  p.a_bytes = p.lbo_a * (uint32_t)(P == MELT_FP8E4M3 ? 2 * ((p.H + 31) / 32) : p.H / 8);
  p.abuf_bytes = p.a_bytes * parts;
  p.step_bytes = p.kstep_bytes * parts;
  melt_plan cands[kMaxCands];
  int nc = 0;
  if (tb->forced) {
    cands[nc++] = tb->plan;
  } else {
    nc = candidate_list(tb, p, cands, kMaxCands);
  }
  for (int i = 0; i < nc; ++i) {
    if (cands[i].cta_pair ? try_layout_pair(tb, p, cands[i], n_mfcc) : try_layout(tb, p, cands[i], n_mfcc))
      return true;
  }
  return false;
}

}  // namespace

// ---- layouts
namespace {

bool try_layout(const TcBasis* tb, TcParams& p, const melt_plan& c, int n_mfcc) {
  const int P = tb->precision;
  if (c.cta_pair != 0 || c.schedule != 0 || P == MELT_FP8E4M3) return false;  // FP8 runs in CTA pairs
  p.nacc = 2;
  p.Hd = 0;
  p.NS = p.CH = p.NCHUNK = 0;
  p.st_bytes = p.off_st = 0;
  p.b_lbo = (uint32_t)p.NC * 16;
  p.step_bytes = p.kstep_bytes * (P == MELT_BF16X3 ? 2 : 1);
  if (c.a_buffers < 1 || c.a_buffers > 2 || c.prefetch_tiles < 0 || c.prefetch_tiles > kMaxPrefetch)
    return false;
  if (!c.basis_resident && (c.basis_slots < 2 || c.basis_slots > 32 || c.ksteps_per_slot < 1))
    return false;
  const bool wide = p.nblk > 1;  // more than 128 Mel bins: streamed basis, no MFCC
  if (wide && (c.basis_resident || n_mfcc != 0)) return false;
  p.b_resident = c.basis_resident ? 1 : 0;
  p.ZB = c.a_buffers;
  p.pf = c.prefetch_tiles;
  p.kps = p.b_resident ? 1 : std::min(c.ksteps_per_slot, p.KS);
  p.NB = p.b_resident ? p.KS : c.basis_slots;
  const uint32_t parts = P == MELT_BF16X3 ? 2u : 1u;
  p.blk_step = wide ? 256u * 32u * parts : p.step_bytes;
  p.blk_step_last = wide ? 2u * (uint32_t)p.wbl * 32u * parts : p.step_bytes;
  p.bslot_bytes = p.b_resident ? p.step_bytes : p.blk_step * p.kps;
  const Bars B(p.ZB, p.NB);
  uint32_t off = 0;
  p.off_a = off;
  off += align_up(p.abuf_bytes * p.ZB, 128);
  p.off_b = off;
  off += align_up(p.bslot_bytes * p.NB, 128);
  p.off_bar = off;
  off += align_up(8 * B.total, 128);
  p.off_tab = off;
  off += align_up(8 * p.KS, 128);
  p.off_misc = off;
  off += 128;
  p.off_dct = off;
  off += align_up(4 * ((n_mfcc + 3) & ~3) * p.MP, 128);
  p.off_fb = off;  // fused STFT + Mel comparator: one 16-byte filterbank entry per DFT bin
  off += tb->stft_bands > 0 ? align_up(16u * (uint32_t)p.MP, 128) : 0u;
  if (off + 128 > kSmemLimit) return false;
  p.smem_total = off + 128;
  p.tmem_cols = p.NC <= 32 ? 64 : p.NC <= 64 ? 128 : p.NC <= 128 ? 256 : 512;
  p.acc_stride = p.tmem_cols / 2;
  p.idesc = idesc_f32acc(1u, kF, wide ? 256u : (uint32_t)p.NC);
  p.idesc_last = idesc_f32acc(1u, kF, wide ? 2u * (uint32_t)p.wbl : (uint32_t)p.NC);
  p.desc_hi = (128u >> 4) | (1u << 14);  // SBO = 128 B; version bit (descriptor bit 46)
  return true;
}

// CTA-pair layout (BF16, FP8): A buffers, the waveform staging ring and this
// CTA's half of the basis (resident, or streamed through NB slots of kps
// K-steps), then barriers and tables.  The ring takes every slot that still
// fits (2..8).  A streamed half basis serves the BF16 and split-BF16 log-Mel
// kernels with the static schedule (no fused MLP, no MFCC); split BF16 runs
// in pairs only that way (hi + lo halves do not fit resident beside two
// split A buffers).
bool try_layout_pair(const TcBasis* tb, TcParams& p, const melt_plan& c, int n_mfcc) {
  const bool fp8 = tb->precision == MELT_FP8E4M3;
  const bool x3 = tb->precision == MELT_BF16X3;
  if (c.cta_pair != 1 || (tb->precision != MELT_BF16 && !fp8 && !x3) || !tb->d_b2 || p.nblk > 1 ||
      tb->stft_bands > 0)
    return false;
  // FP8: a converter lane holds at most two quads of a Z row
  if (fp8 && p.H > 256) return false;
  if (c.basis_resident < 0 || c.basis_resident > 1 || c.a_buffers < 1 || c.a_buffers > 2) return false;
  if (c.prefetch_tiles < 0 || c.prefetch_tiles > kMaxPrefetch) return false;
  if (c.schedule != 0 && c.schedule != 1) return false;
  const bool streamed = c.basis_resident == 0;
  if (streamed && (fp8 || c.schedule != 0 || n_mfcc != 0 || tb->mlp_hd > 0 || c.basis_slots < 2 ||
                   c.basis_slots > 8 || c.ksteps_per_slot < 1 || c.ksteps_per_slot > 16))
    return false;
  if (x3 && (!streamed || n_mfcc != 0)) return false;
  p.dyn = c.schedule;
  p.b_resident = streamed ? 0 : 1;
  p.blk_step = p.blk_step_last = 0;
  p.ZB = c.a_buffers;
  p.pf = c.schedule ? 0 : c.prefetch_tiles;  // L2 prefetch stream of the waveform producer (static schedule)
  // one K-step block of this CTA's N/2 basis rows (split BF16: hi, then lo)
  p.step_bytes = p.kstep_bytes / 2 * (x3 ? 2 : 1);
  p.kps = streamed ? std::min(c.ksteps_per_slot, p.KS) : 1;
  p.NB = streamed ? c.basis_slots : p.KS;
  p.bslot_bytes = p.step_bytes * (uint32_t)p.kps;
  p.b_lbo = (uint32_t)(p.NC / 2) * 16;
  // fused correction MLP: its weight half in shared memory, one projection
  // accumulator in TMEM and the MLP's operands beside it
  p.Hd = fp8 || x3 || streamed ? 0 : tb->mlp_hd;
  // TMEM: two projection accumulators 256 columns apart when room is left
  // beside the first for FP8's scale-factor columns (sfg groups of four per A
  // buffer, then kSfBCols for the basis scale), else one
  p.sfg = fp8 ? (p.J + 3) / 4 : 0;
  const int sf_cols = fp8 ? 4 * p.sfg * p.ZB + kSfBCols : 0;
  p.nacc = (p.Hd > 0 || p.NC + sf_cols > 256) ? 1 : 2;
  // MFCC: the DCT on the tensor cores where its TMEM columns fit beside the
  // projection accumulators (two 256 columns apart, else one) and FP8's scale
  // factors: the coefficient accumulator (dct_n columns) and the split-BF16
  // log-Mel operand (MP / 2 columns per part), first fit into what is free
  p.dct_tc = 0;
  if (n_mfcc > 0 && p.Hd == 0) {
    const int nd = (n_mfcc + 15) & ~15;
    for (int na = 2; na >= 1 && !p.dct_tc; --na) {
      if (na == 2 && p.NC + sf_cols > 256) continue;
      int iv[2][2] = {{p.NC + (na == 2 ? sf_cols : 0), 256}, {256 + (na == 2 ? p.NC : sf_cols), 512}};
      auto place = [&](int w, int align, uint32_t& col) {
        for (auto& v : iv) {
          const int s0 = (v[0] + align - 1) / align * align;
          if (s0 + w <= v[1]) {
            col = (uint32_t)s0;
            v[0] = s0 + w;
            return true;
          }
        }
        return false;
      };
      if (place(nd, 16, p.dct_c) && place(p.MP / 2, 8, p.dct_ahi) && place(p.MP / 2, 8, p.dct_alo)) {
        p.dct_tc = 1;
        p.nacc = na;
        p.dct_n = nd;
        p.dct_part = (uint32_t)(p.MP / 8) * (uint32_t)(nd / 2) * 16u;
        p.idesc_dct = idesc_f32acc(1u, 2 * kF, (uint32_t)nd);
      }
    }
  }
  p.sf_col = (uint32_t)(p.nacc == 2 ? p.NC : 256);
  if (fp8 && (p.nacc == 2 ? p.NC + sf_cols > 256 : p.NC > 256 || 256 + sf_cols > 512)) return false;
  if (p.Hd > 0) {
    if (n_mfcc != 0 || p.NC > 160 || 160 + p.MP > 256 || 256 + p.Hd > 512) return false;
    p.mlp_half = (uint32_t)tb->mlp_half;
    p.w1_step = (uint32_t)(p.Hd / 2) * 32;
    p.w2_step = (uint32_t)(p.MP / 2) * 32;
    p.mlp_w2_off = (uint32_t)(p.MP / 16) * p.w1_step;
    p.mlp_vec_off = p.mlp_w2_off + (uint32_t)(p.Hd / 16) * p.w2_step;
    // TMEM: accumulator [0, NC), Y [160, 160 + MP) with x-hat's band chunk c
    // at 160 + 16 c (GEMM1 consumes it before Y is written), H and, in place,
    // GELU(H) [256, 256 + Hd)
    p.a1_col = 160;
    p.h_col = 256;
    p.y_col = 160;
    p.idesc1 = idesc_f32acc(1u, 2 * kF, (uint32_t)p.Hd);
    p.idesc2 = idesc_f32acc(1u, 2 * kF, (uint32_t)p.MP);
  }
  // staging chunks: whole Z rows.  BF16: <= 16 KB and <= what one converter
  // pass covers (kPQuads quads per thread); FP8: up to kF8MaxRows rows (all
  // row slots of the converter warps) and 20 KB, fewer where that does not fit
  const uint32_t row_bytes = (uint32_t)p.H * 4;
  const uint32_t span_bytes = row_bytes * p.zrows;
  int chs[3] = {0, 0, 0}, nch_c = 0;
  if (fp8) {
    for (int c8 = std::max(1, std::min(kF8MaxRows, (int)(20480u / row_bytes))); c8 >= 1 && nch_c < 3; c8 /= 2)
      chs[nch_c++] = c8;
  } else {
    const int nchunk = (int)((span_bytes + 16383) / 16384);
    int ch = (p.zrows + nchunk - 1) / nchunk;
    const int max_rows = kPQuads * (p.Hd > 0 ? 32 * kMlpCvtWarps : kPCvtThreads) * 4 / p.H;
    if (ch > max_rows) ch = std::max(1, max_rows);
    chs[nch_c++] = ch;
    // smaller chunks where the 16 KB ones leave no room for a ring of two
    // (split BF16's two A parts, long frames)
    for (int c2 = ch / 2; c2 >= 4 && nch_c < 3; c2 /= 2) chs[nch_c++] = c2;
  }
  p.codes_stride = fp8 ? align_up((uint32_t)p.zrows + 3, 16) : 0u;
  for (int ci = 0; ci < nch_c; ++ci) {
    const int ch = chs[ci];
    p.CH = ch;
    p.NCHUNK = (p.zrows + ch - 1) / ch;
    p.st_bytes = row_bytes * ch;
    for (int ns = 8; ns >= 2; --ns) {
      const PairBars B(ns, p.ZB, p.KS, streamed ? p.NB : 0);
      uint32_t off = 0;
      p.off_a = off;
      off += align_up(p.abuf_bytes * p.ZB, 128);
      p.off_st = off;
      off += align_up(p.st_bytes * ns, 128);
      p.off_b = off;
      off += align_up(streamed ? p.bslot_bytes * p.NB : p.step_bytes * p.KS, 128);
      p.off_mlp = off;
      off += p.Hd > 0 ? align_up(p.mlp_half, 128) : 0u;
      p.off_bar = off;
      off += align_up(8 * B.total, 128);
      p.off_tab = off;
      off += align_up(8 * p.KS, 128);
      p.off_misc = off;
      off += 128;
      p.off_codes = off;  // FP8: the scale code of every Z row of the tile, per A buffer
      off += fp8 ? align_up(p.codes_stride * (uint32_t)p.ZB, 128) : 0u;
      p.off_dct = off;
      off += align_up(p.dct_tc ? 2 * p.dct_part : 4 * ((n_mfcc + 3) & ~3) * p.MP, 128);
      if (off + 128 > kSmemLimit) continue;
      p.NS = ns;
      p.smem_total = off + 128;
      p.tmem_cols = fp8 || p.dct_tc ? 512 : p.NC <= 32 ? 64 : p.NC <= 64 ? 128 : p.NC <= 128 ? 256 : 512;
      p.acc_stride = p.tmem_cols / 2;
      p.idesc = fp8 ? idesc_mxf8(2 * kF, p.NC) : idesc_f32acc(1u, 2 * kF, p.NC);  // M = 256 over the pair
      p.desc_hi = (128u >> 4) | (1u << 14);
      return true;
    }
  }
  return false;
}

// Layouts in preference order (whether each fits is checked by try_layout).
// The waveform needs no shared memory (converters load it from L2, where it
// was prefetched), so shared memory holds the A buffers and the basis.  A
// resident basis with two A buffers comes first: the MMAs never wait for a
// basis copy and the conversion of tile k+1 overlaps the MMAs of tile k.
// When the basis does not fit beside two A buffers (M > 80 at N = 400, or
// BF16x3), the basis is streamed from L2 through a ring of the largest slots
// that fit; the single-buffer layouts come last.
constexpr int kDefaultSchedule = 0;  // pair schedule of the default plans (0 static, 1 dynamic)

int candidate_list(const TcBasis* tb, const TcParams& p, melt_plan* out, int cap) {
  (void)tb;
  int n = 0;
  auto add = [&](int res, int zb, int pf, int nb, int kps) {
    if (n < cap) out[n++] = melt_plan{res, zb, pf, nb, kps, 0, 0};
  };
  const uint32_t parts = tb->precision == MELT_BF16X3 ? 2u : 1u;
  // bytes of one streamed K-step: all basis rows, or one block of 128 Mel bins when M > 128
  const int sb = (int)std::max(1u, p.nblk > 1 ? 256u * 32u * parts : p.kstep_bytes * parts);
  melt_plan alts[2];
  int n_alt = 0;
  if ((tb->precision == MELT_BF16 || tb->precision == MELT_FP8E4M3) && tb->d_b2) {
    // CTA pairs first (measured on the 64 x 30 s batch at M = 80: 41 us
    // against 50 us single-CTA).  A staging ring of fewer than 4 slots keeps
    // too few bytes in flight; an L2 prefetch stream one tile ahead makes up
    // for it (M = 128, two A buffers, 2 slots: 58 us against 66 us without,
    // and 63 us with one A buffer and more slots), but costs time where the
    // ring is deep enough (M = 80, 5 slots: 42.5 against 42.1 us) and with
    // the correction fused (167 against 164 us).  When launches overlap
    // (MELT_FWD_INPUT_READY) the stream pays at M = 80 too (BF16 log-Mel:
    // 37.4 against 38.1 us; FP8: 52.1 against 51.3 us, so not for FP8).
    // FP8 runs in CTA pairs only
    // (its converter is the polyphase one with a per-row scale).  The static
    // schedule is the default: the dynamic one measured no gain (42.6 against
    // 42.4 us).
    for (int zb = 2; zb >= 1; --zb) {
      melt_plan pc{1, zb, 0, p.KS, 1, 1, kDefaultSchedule};
      TcParams q = p;
      if (n < cap && try_layout_pair(tb, q, pc, tb->n_mfcc) && q.NS >= 2) {
        const bool bf16_logmel = tb->precision == MELT_BF16 && tb->n_mfcc == 0;
        if ((q.NS < 4 || bf16_logmel) && !tb->mlp_hd) pc.prefetch_tiles = kDefaultSchedule ? 0 : 1;
        out[n++] = pc;
        // the other pair schedule, for melt_autotune (after every default layout)
        melt_plan alt = pc;
        alt.schedule = 1 - kDefaultSchedule;
        alt.prefetch_tiles = alt.schedule ? 0 : (q.NS < 4 && !tb->mlp_hd ? 1 : 0);
        if (n_alt < 2) alts[n_alt++] = alt;
      }
    }
  }
  if (tb->precision == MELT_FP8E4M3) {  // no single-CTA FP8 layouts
    for (int i = 0; i < n_alt && n < cap; ++i) out[n++] = alts[i];
    return n;
  }
  add(1, 2, 2, p.KS, 1);
  const int kps_hi = std::max(1, std::min(p.KS, 65536 / sb));   // <= 64 KB per slot
  for (int kps = kps_hi; kps >= 1; --kps)
    for (int nb = 2; nb <= 3; ++nb) add(0, 2, 2, nb, kps);
  add(1, 1, 2, p.KS, 1);
  for (int kps = kps_hi; kps >= 1; --kps) add(0, 1, 2, 2, kps);
  for (int nb = 24; nb >= 2; nb -= 2) add(0, 1, 2, nb, 1);
  if ((tb->precision == MELT_BF16 || tb->precision == MELT_BF16X3) && tb->d_b2 && tb->n_mfcc == 0 &&
      !tb->mlp_hd) {
    // CTA pairs with each CTA's half basis streamed through slots (split
    // BF16, long frames): a 2-SM MMA shares every basis block between two
    // tiles, so each tile reads half the basis a single-CTA layout streams.
    // Measured no faster than the single-CTA streamed layouts (64 x 30 s
    // split BF16: 86.6 against 83.4 us; 64 x 20 s at 22.05 kHz, N = 1024:
    // 51.2 against 51.1 us): each slot's turnaround (copy from L2, the odd
    // CTA's signal, the MMAs' release) is the limit, not L2 traffic.  So
    // they come after the single-CTA layouts, for melt_autotune.
    const int shapes[][2] = {{4, 4}, {4, 2}, {3, 4}, {2, 8}, {3, 2}, {2, 4}, {2, 2}, {2, 1}};
    for (int zb = 2; zb >= 1; --zb)
      for (const auto& sh : shapes) {
        melt_plan pc{0, zb, 0, sh[0], sh[1], 1, 0};
        TcParams q = p;
        if (n < cap && try_layout_pair(tb, q, pc, 0) && q.NS >= 2) {
          if (q.NS < 4) pc.prefetch_tiles = 1;
          out[n++] = pc;
        }
      }
  }
  for (int i = 0; i < n_alt && n < cap; ++i) out[n++] = alts[i];
  return n;
}

}  // namespace

melt_status tc_build(TcBasis* tb, const TcConfig& c, const double* w64) {
  const int N = c.n_fft, H = c.hop, M = c.n_mels, P = c.precision;
  if (P != MELT_BF16 && P != MELT_BF16X3 && P != MELT_FP8E4M3) return MELT_ERR_ARG;
  if (P != MELT_FP8E4M3 && (H % 16) != 0) return MELT_ERR_UNSUPPORTED;
  // M > 128 (up to 1024): BF16 forms only, as blocks of 128 Mel bins (FP8 runs in CTA pairs, M <= 128)
  if (M > 1024 || (M > 128 && P == MELT_FP8E4M3)) return MELT_ERR_UNSUPPORTED;
  if (M > 128 && c.n_mfcc > 0) return MELT_ERR_UNSUPPORTED;
  const int MP = (M + 15) / 16 * 16, NC = 2 * MP;
  const int nblk = (MP + 127) / 128;
  const int J = (N + H - 1) / H;
  // K-steps in (slice j, first sample r0 of the step) order; a step covers
  // 16 samples of slice j (BF16 forms) or 32 (FP8)
  const int kstep = P == MELT_FP8E4M3 ? 32 : 16;
  std::vector<std::pair<int, int>> steps;
  for (int j = 0; j < J; ++j) {
    const int kj = std::min(H, N - j * H);
    for (int kk = 0; kk < (kj + kstep - 1) / kstep; ++kk) steps.push_back({j, kstep * kk});
  }
  const int KS = (int)steps.size();
  const size_t kstep_bytes = (size_t)NC * 32;  // 2 core columns x NC rows x 16 B
  const int parts = (P == MELT_BF16X3) ? 2 : 1;
  std::vector<uint8_t> img((size_t)KS * parts * kstep_bytes, 0);
  auto wval = [&](int row, int n) -> double {  // row of the stacked, padded basis
    if (n < 0 || n >= N) return 0.0;
    if (row < MP) return row < M ? w64[(size_t)row * N + n] : 0.0;
    const int m = row - MP;
    return m < M ? w64[(size_t)(M + m) * N + n] : 0.0;
  };
  // Image layout: one block per K-step of all NC rows, [part][core column
  // cc][row][16 B] (parts: hi, then lo for BF16x3).  With more than 128 Mel
  // bins the image is block-major instead: block b (Mel bins [128 b, 128 b +
  // wb), R rows then I rows, 2 wb rows) holds all its K-steps contiguously.
  auto blk_rows = [&](int b) { return nblk == 1 ? NC : 2 * std::min(128, MP - 128 * b); };
  auto stacked_row = [&](int b, int r) {  // row of the stacked [W_r (MP rows); W_i (MP rows)] basis
    if (nblk == 1) return r;
    const int wb = blk_rows(b) / 2;
    return r < wb ? 128 * b + r : MP + 128 * b + (r - wb);
  };
  for (int b = 0; b < nblk; ++b)
  for (int s = 0; s < KS; ++s) {
    const int rows_b = blk_rows(b);
    const size_t part_b = (size_t)rows_b * 32;  // one part of one K-step of block b
    uint8_t* blk = img.data() + (size_t)b * KS * parts * 256 * 32 + (size_t)s * parts * part_b;
    const int j = steps[s].first, r0 = steps[s].second;
    const int kj = std::min(H, N - j * H);  // samples of slice j; zero past them
    for (int cc = 0; cc < 2; ++cc)
      for (int brow = 0; brow < rows_b; ++brow) {
        const int row = stacked_row(b, brow);
        if (P == MELT_FP8E4M3) {
          // 16 e4m3 values per core-column row: W 2^8 (the MMA scales by 2^-8)
          for (int e = 0; e < 16; ++e) {
            const int r = r0 + 16 * cc + e;
            const double w = r < kj ? std::ldexp(wval(row, j * H + r), 8) : 0.0;
            blk[(size_t)cc * rows_b * 16 + brow * 16 + e] = e4m3_bits(w);
          }
        } else {
          for (int e = 0; e < 8; ++e) {
            const int r = r0 + 8 * cc + e;
            const double w = (r < H) ? wval(row, j * H + r) : 0.0;
            const uint16_t hi = bf16_bits(w);
            std::memcpy(blk + (size_t)cc * rows_b * 16 + brow * 16 + e * 2, &hi, 2);
            if (P == MELT_BF16X3) {
              const uint16_t lo = bf16_bits(w - bf16_value(hi));
              std::memcpy(blk + part_b + (size_t)cc * rows_b * 16 + brow * 16 + e * 2, &lo, 2);
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
  tb->kstep_k = kstep;
  tb->n_cols = NC;
  tb->kstep_bytes = kstep_bytes;
  tb->n_mfcc = c.n_mfcc;
  tb->stft_bands = c.stft_bands;
  if (P != MELT_FP8E4M3) {  // the single-CTA image (FP8 runs in CTA pairs only)
    if (melt::dev_alloc(&tb->d_b, img.size()) != cudaSuccess) return MELT_ERR_OOM;
    if (cudaMemcpy(tb->d_b, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return MELT_ERR_CUDA;
  }
  if ((P == MELT_BF16 || P == MELT_FP8E4M3 || P == MELT_BF16X3) && nblk == 1) {
    // CTA-pair image: the K-step blocks of basis rows [0, MP) (W_r), then those
    // of rows [MP, 2 MP) (W_i); each block is 2 core columns x MP rows x 16 B
    // per part (split BF16: the hi part, then the lo part)
    const size_t half_step = (size_t)MP * 32;
    std::vector<uint8_t> img2((size_t)2 * KS * parts * half_step, 0);
    for (int h = 0; h < 2; ++h)
      for (int s = 0; s < KS; ++s)
        for (int pt = 0; pt < parts; ++pt)
          for (int cc = 0; cc < 2; ++cc)
            for (int r = 0; r < MP; ++r)
              std::memcpy(img2.data() + (((size_t)h * KS + s) * parts + pt) * half_step + (size_t)cc * MP * 16 +
                              (size_t)r * 16,
                          img.data() + ((size_t)s * parts + pt) * kstep_bytes + (size_t)cc * NC * 16 +
                              (size_t)(h * MP + r) * 16,
                          16);
    if (melt::dev_alloc(&tb->d_b2, img2.size()) != cudaSuccess) return MELT_ERR_OOM;
    if (cudaMemcpy(tb->d_b2, img2.data(), img2.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return MELT_ERR_CUDA;
    // counters of the dynamic pair schedule (each launch leaves its pair at zero)
    const size_t sb = sizeof(unsigned long long) * 2 * kSchedWords;
    if (melt::dev_alloc(&tb->d_sched, sb) != cudaSuccess) return MELT_ERR_OOM;
    if (cudaMemset(tb->d_sched, 0, sb) != cudaSuccess) return MELT_ERR_CUDA;
  }
  {
    TcParams probe;
    std::memset(&probe, 0, sizeof(probe));
    if (!plan_smem(tb, probe, c.n_mfcc)) return MELT_ERR_UNSUPPORTED;  // operands do not fit shared memory
  }
  return MELT_OK;
}

void tc_free(TcBasis* tb) {
  cudaFree(tb->d_b);
  cudaFree(tb->d_b2);
  cudaFree(tb->d_mlp_img);
  cudaFree(tb->d_sched);
  tb->d_b = tb->d_b2 = nullptr;
  tb->d_mlp_img = nullptr;
  tb->d_sched = nullptr;
}

int tc_max_mfcc() { return kMaxMfccTc; }

int tc_candidates(const TcBasis* tb, melt_plan* out, int cap) {
  TcBasis probe = *tb;
  probe.forced = false;
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  if (!plan_smem(&probe, p, tb->n_mfcc)) return 0;  // fills the geometry
  melt_plan all[kMaxCands];
  const int n = candidate_list(tb, p, all, kMaxCands);
  int m = 0;
  for (int i = 0; i < n && m < cap; ++i) {
    TcParams q = p;
    if (all[i].cta_pair ? try_layout_pair(tb, q, all[i], tb->n_mfcc) : try_layout(tb, q, all[i], tb->n_mfcc)) {
      bool dup = false;  // several candidates collapse to one layout (e.g. kps clipped)
      for (int j = 0; j < m; ++j)
        dup |= std::memcmp(&out[j], &all[i], sizeof(melt_plan)) == 0;
      if (!dup) out[m++] = all[i];
    }
  }
  return m;
}

bool tc_plan_fits(const TcBasis* tb, const melt_plan& plan) {
  TcBasis probe = *tb;
  probe.forced = true;
  probe.plan = plan;
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  return plan_smem(&probe, p, tb->n_mfcc);
}

bool tc_current_plan(const TcBasis* tb, melt_plan* out) {
  if (tb->forced) {
    *out = tb->plan;
    return true;
  }
  melt_plan c[1];
  if (tc_candidates(tb, c, 1) < 1) return false;
  *out = c[0];
  return true;
}

cudaError_t tc_launch(const TcBasis* tb, const TcLaunch& L, cudaStream_t stream) {
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  if (!plan_smem(tb, p, L.n_mfcc)) return cudaErrorInvalidConfiguration;
  if (L.n_mfcc > kMaxMfccTc) return cudaErrorInvalidValue;
  const bool pair = p.NS > 0;  // only the CTA-pair layout stages the waveform
  p.wave = L.wave;
  p.tiles = L.tiles;
  p.n_tiles = L.n_tiles;
  p.bimg = static_cast<const uint8_t*>(pair ? tb->d_b2 : tb->d_b);
  p.dct = L.dct;
  p.out = L.out;
  p.err = L.err;
  p.eps = L.eps;
  p.n_mfcc = L.n_mfcc;
  p.n_out = L.stft_bands ? L.stft_bands : L.n_mfcc ? L.n_mfcc : tb->n_mels;
  p.fb = L.fb;
  p.stft_bands = L.stft_bands;
  // the dynamic pair schedule claims pairs from a counter an earlier launch
  // resets when it ends, so its waveform producer keeps the wait
  p.early_inputs = L.early_inputs && L.pdl && !p.dyn ? 1 : 0;
  const bool fused = pair && p.Hd > 0 && L.mlp != nullptr;
  if (pair && p.Hd > 0 && !L.mlp) p.Hd = 0;  // plan made for a correction that is not passed
  KernelFn fn = fused ? kernel_for_pair_mlp(p.MP / 16)
                : pair ? (tb->precision == MELT_FP8E4M3   ? kernel_for_pair_fp8(L.n_mfcc > 0, p.MP / 16, p.dct_tc)
                          : tb->precision == MELT_BF16X3 ? kernel_for_pair_x3()
                                                         : kernel_for_pair(L.n_mfcc > 0, p.MP / 16, p.dct_tc))
                       : (L.n_mfcc ? kernel_for_mfcc(tb->precision, p.MP / 16)
                                   : kernel_for_plain(tb->precision, p.MP / 16, L.stft_bands > 0));
  if (!fn) return cudaErrorInvalidValue;
  if (fused) {
    // the MLP's current parameters (training may have changed them) as BF16
    p.mlp_img = static_cast<const uint8_t*>(tb->d_mlp_img);
    if (mlp_fused_image(L.mlp, tb->d_mlp_img, stream) != MELT_OK) return cudaErrorLaunchFailure;
  }
  if (L.fused) *L.fused = fused;
  const int smem = (int)p.smem_total;
  static thread_local KernelFn last_fn[4] = {nullptr, nullptr, nullptr, nullptr};
  static thread_local int last_smem[4] = {0, 0, 0, 0};
  static thread_local int last_i = 0;
  int hit = -1;
  for (int i = 0; i < 4; ++i)
    if (last_fn[i] == fn && last_smem[i] >= smem) hit = i;
  if (hit < 0) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    last_fn[last_i] = fn;
    last_smem[last_i] = smem;
    last_i = (last_i + 1) & 3;
  }
  // Programmatic dependent launch: this grid may be scheduled while the
  // previous kernel of the stream drains; the kernel orders its own global
  // memory accesses after that kernel with griddepcontrol.wait.
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = L.pdl ? 1 : 0;
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!pair) {
    cfg.gridDim = dim3(std::min(L.n_tiles, L.sm_count), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    return cudaLaunchKernelEx(&cfg, fn, p);
  }
  // CTA pairs: clusters of two, as many as can be resident at once (persistent)
  p.n_pairs = (L.n_tiles + 1) / 2;
  if (p.dyn) {
    if (!tb->d_sched) return cudaErrorInvalidValue;
    TcBasis* sb = const_cast<TcBasis*>(tb);
    p.sched = tb->d_sched + 2 * (sb->sched_next++ % kSchedWords);
  }
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = 2;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.blockDim = dim3(pair_threads(fused, tb->precision, L.n_mfcc > 0, p.MP / 16, p.dct_tc), 1, 1);
  cfg.numAttrs = 2;
  TcBasis* mtb = const_cast<TcBasis*>(tb);
  if (mtb->pair_clusters < 0 || mtb->pair_smem != smem) {
    cfg.gridDim = dim3(2 * (L.sm_count / 2), 1, 1);
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
    if (e != cudaSuccess) return e;
    mtb->pair_clusters = n;
    mtb->pair_smem = smem;
  }
  if (mtb->pair_clusters < 1) return cudaErrorInvalidConfiguration;
  const int clusters = std::min(p.n_pairs, mtb->pair_clusters);
  cfg.gridDim = dim3(2 * clusters, 1, 1);
  return cudaLaunchKernelEx(&cfg, fn, p);
}

}  // namespace melt

namespace melt {

namespace {

// Parameters of one basis's half of a two-basis pair launch; false if the
// basis cannot run as a BF16 log-Mel CTA pair there.
bool group_pair_params(const TcBasis* tb, const TcLaunch& L, TcParams& p) {
  if (tb->precision != MELT_BF16 || tb->n_mfcc != 0 || tb->stft_bands > 0 || L.n_mfcc != 0 || L.mlp || !tb->d_b2)
    return false;
  TcBasis probe = *tb;
  melt_plan cands[kMaxCands];
  const int n = tc_candidates(tb, cands, kMaxCands);
  if (n < 1) return false;
  if (!tb->forced && cands[0].cta_pair != 1) {
    // default plan single-CTA: the first CTA-pair layout among the candidates
    int i = 0;
    while (i < n && cands[i].cta_pair != 1) ++i;
    if (i == n) return false;
    probe.forced = true;
    probe.plan = cands[i];
  }
  std::memset(&p, 0, sizeof(p));
  if (!plan_smem(&probe, p, 0) || p.NS == 0 || p.dyn || p.Hd > 0) return false;
  p.wave = L.wave;
  p.tiles = L.tiles;
  p.n_tiles = L.n_tiles;
  p.n_pairs = (L.n_tiles + 1) / 2;
  p.bimg = static_cast<const uint8_t*>(tb->d_b2);
  p.dct = L.dct;
  p.out = L.out;
  p.err = L.err;
  p.eps = L.eps;
  p.n_mfcc = 0;
  p.n_out = tb->n_mels;
  p.early_inputs = L.early_inputs && L.pdl ? 1 : 0;
  return true;
}

}  // namespace

cudaError_t tc_launch_pair_group(const TcBasis* tb0, const TcLaunch& L0, const TcBasis* tb1, const TcLaunch& L1,
                                 double frac0, cudaStream_t stream, bool* launched) {
  *launched = false;
  if (L0.n_tiles < 1 || L1.n_tiles < 1) return cudaSuccess;
  TcGroupParams q;
  std::memset(&q, 0, sizeof(q));
  if (!group_pair_params(tb0, L0, q.g[0]) || !group_pair_params(tb1, L1, q.g[1])) return cudaSuccess;
  GroupKernelFn fn = kernel_for_pair_group();
  const int smem = (int)std::max(q.g[0].smem_total, q.g[1].smem_total);
  int dev = 0;
  {
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
  }
  // per thread: the device, the shared-memory size the attribute was set
  // for, and the co-resident cluster count at that size
  static thread_local int last_dev = -1, set_smem = 0, occ_smem = -1, occ_clusters = 0;
  if (last_dev != dev) {
    last_dev = dev;
    set_smem = 0;
    occ_smem = -1;
  }
  if (set_smem < smem) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    set_smem = smem;
  }
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = L0.pdl ? 1 : 0;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = 2;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cfg.blockDim = dim3(pair_threads(false, MELT_BF16, false, 1, false), 1, 1);
  if (occ_smem != smem) {
    cfg.gridDim = dim3(2 * (L0.sm_count / 2), 1, 1);
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
    if (e != cudaSuccess) return e;
    occ_smem = smem;
    occ_clusters = n;
  }
  const int C = std::min(occ_clusters, q.g[0].n_pairs + q.g[1].n_pairs);
  if (C < 2) return cudaSuccess;
  // clusters for the first basis: its share of the work, at least one each,
  // none beyond a basis's own pair count
  int s = (int)std::lround(frac0 * C);
  s = std::max(s, C - q.g[1].n_pairs);
  s = std::min(s, q.g[0].n_pairs);
  s = std::max(1, std::min(C - 1, s));
  q.split = s;
  cfg.gridDim = dim3(2 * C, 1, 1);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, q);
  if (e == cudaSuccess) *launched = true;
  return e;
}

}  // namespace melt
