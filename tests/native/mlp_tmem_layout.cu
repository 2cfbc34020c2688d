// Host check of the fused correction MLP's TMEM layout rules, from the
// kernel's own index functions (no GPU): for every hidden-chunk count nh and
// band-chunk count, the epilogue warps' runs partition the chunks; each
// chunk's packed GELU(H) block (8 columns) lies inside H, inside the columns
// its own warp has already read (so it overwrites nothing another warp, or
// the chunk loaded next, still needs), and no two blocks overlap; the column
// the epilogue stores a chunk at equals the one the output layer's MMA reads.
#include <cstdio>
#include <vector>

#include "melt_tc2_kernel.cuh"

using melt::tc::kMlpParts;
using melt::tc::mlp_gelu_off;
using melt::tc::part_lo;
using melt::tc::part_lo_tail;

int main() {
  int bad = 0, cases = 0;
  for (int nh = kMlpParts; nh <= 16; ++nh) {
    ++cases;
    std::vector<int> owner(16 * nh, -1);  // FP32 H columns written with packed GELU
    int prev = 0;
    for (int j = 0; j < kMlpParts; ++j) {
      const int lo = part_lo_tail(nh, kMlpParts, j), hi = part_lo_tail(nh, kMlpParts, j + 1);
      if (lo != prev || hi < lo) {
        std::printf("nh %d: run %d is [%d, %d) after %d\n", nh, j, lo, hi, prev);
        ++bad;
      }
      prev = hi;
      for (int cc = lo; cc < hi; ++cc) {
        const int off = (int)mlp_gelu_off(nh, cc);
        if (off != 8 * (cc + lo)) {  // the epilogue's store column (gelu_run: h_col + 8 (cc + lo))
          std::printf("nh %d: chunk %d stored at %d, read by the MMA at %d\n", nh, cc, 8 * (cc + lo), off);
          ++bad;
        }
        if (off < 16 * lo || off + 8 > 16 * (cc + 1)) {  // own run, already read (and not the next chunk)
          std::printf("nh %d: chunk %d block [%d, %d) outside [%d, %d)\n", nh, cc, off, off + 8, 16 * lo, 16 * (cc + 1));
          ++bad;
        }
        for (int c = off; c < off + 8 && c < 16 * nh; ++c) {
          if (owner[c] != -1) {
            std::printf("nh %d: column %d holds chunks %d and %d\n", nh, c, owner[c], cc);
            ++bad;
          }
          owner[c] = cc;
        }
      }
    }
    if (prev != nh) {
      std::printf("nh %d: runs end at %d\n", nh, prev);
      ++bad;
    }
  }
  for (int nch = 1; nch <= 8; ++nch) {  // band chunks (part_lo): a partition too
    ++cases;
    int prev = 0;
    for (int j = 0; j < kMlpParts; ++j) {
      const int lo = part_lo(nch, kMlpParts, j), hi = part_lo(nch, kMlpParts, j + 1);
      if (lo != prev || hi < lo) ++bad;
      prev = hi;
    }
    if (prev != nch) ++bad;
  }
  std::printf("cases %d bad %d\n", cases, bad);
  return bad == 0 ? 0 : 1;
}
