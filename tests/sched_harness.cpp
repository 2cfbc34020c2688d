// Runs melt::balance_tiles on tile lists read from stdin and prints each
// resulting order as the original tile indices.
//
// Input, repeated until end of file: "n unit W" and then n frame counts.
// Output per case: one line of n indices.
#include <cstdio>
#include <vector>

#include "../paper_2606_01009_gb300/csrc/melt_internal.h"

int main() {
  long long n = 0;
  int unit = 0, W = 0;
  while (std::scanf("%lld %d %d", &n, &unit, &W) == 3) {
    std::vector<melt::TileDesc> t((size_t)n), tmp((size_t)n);
    std::vector<int32_t> order((size_t)n);
    for (long long i = 0; i < n; ++i) {
      int f = 0;
      if (std::scanf("%d", &f) != 1) return 2;
      t[i] = melt::TileDesc{};
      t[i].n_frames = f;
      t[i].clip = (int32_t)i;
    }
    melt::balance_tiles(t.data(), n, unit, W, tmp.data(), order.data());
    for (long long i = 0; i < n; ++i) std::printf(i ? " %d" : "%d", t[i].clip);
    std::printf("\n");
  }
  return 0;
}
