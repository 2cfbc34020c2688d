// Work order of the persistent kernels' static schedule (host only).
//
// The balancing is host code with no CUDA calls, so it also builds with a
// plain C++ compiler (`-x c++`), which lets its tests run without a GPU.
#include <algorithm>
#include <cstring>

#include "melt_internal.h"

namespace melt {

void balance_tiles(TileDesc* t, long long n, int unit, int W, TileDesc* tmp, int32_t* order) {
  if (n < 2 || W < 1 || W > kMaxBalanceWorkers || (unit != 1 && unit != 2) || n > INT32_MAX) return;
  const long long N = (n + unit - 1) / unit;  // work units; the last one may be a lone tile
  // 1. tiles longest first (a stable counting sort on the frame count), so
  //    consecutive tiles, the members of one pair, have about the same length
  auto frames = [&](long long i) {
    return (int)std::min<int64_t>(std::max<int64_t>(t[i].n_frames, 0), kTileFrames);
  };
  long long start[kTileFrames + 2] = {};
  for (long long i = 0; i < n; ++i) ++start[kTileFrames - frames(i) + 1];
  for (int k = 1; k <= kTileFrames + 1; ++k) start[k] += start[k - 1];
  for (long long i = 0; i < n; ++i) order[start[kTileFrames - frames(i)]++] = (int32_t)i;
  // a unit costs what its longest tile costs: the pair's MMAs wait for both CTAs
  auto cost = [&](long long u) { return (long long)frames(order[u * unit]) + kTileFixedFrames; };
  // 2. worker w runs the units at list positions w, w + W, ...: cap[w] of them
  long long load[kMaxBalanceWorkers], rem[kMaxBalanceWorkers], taken[kMaxBalanceWorkers];
  for (int w = 0; w < W; ++w) {
    rem[w] = w < N ? (N - 1 - w) / W + 1 : 0;
    load[w] = 0;
    taken[w] = 0;
  }
  auto place = [&](long long u, int w) {
    const long long pos = taken[w]++ * W + w;
    for (int j = 0; j < unit; ++j) {
      const long long src = u * unit + j;
      if (src < n) tmp[pos * unit + j] = t[order[src]];
    }
  };
  // an odd tile count leaves the last pair with one tile: it must sit at the
  // last list position, i.e. the last unit of worker (N - 1) mod W
  const bool lone = (n % unit) != 0;
  const long long ng = lone ? N - 1 : N;
  const int wl = (int)((N - 1) % W);
  if (lone) {
    rem[wl] -= 1;
    load[wl] += cost(N - 1);
  }
  // 3. units longest first, each to the worker with the lowest projected load
  //    (its load plus its remaining slots at the cheapest unit's cost); a
  //    binary min-heap on (projection, worker)
  const long long cmin = ng > 0 ? cost(ng - 1) : 0;
  long long hk[kMaxBalanceWorkers];
  int hw[kMaxBalanceWorkers];
  int hs = 0;
  auto less = [&](int i, int j) { return hk[i] < hk[j] || (hk[i] == hk[j] && hw[i] < hw[j]); };
  auto swap_at = [&](int i, int j) {
    std::swap(hk[i], hk[j]);
    std::swap(hw[i], hw[j]);
  };
  auto push = [&](int w) {
    int i = hs++;
    hk[i] = load[w] + (rem[w] - 1) * cmin;
    hw[i] = w;
    while (i > 0 && less(i, (i - 1) / 2)) {
      swap_at(i, (i - 1) / 2);
      i = (i - 1) / 2;
    }
  };
  auto pop = [&]() {
    const int w = hw[0];
    swap_at(0, --hs);
    for (int i = 0;;) {
      int m = i;
      const int l = 2 * i + 1, r = l + 1;
      if (l < hs && less(l, m)) m = l;
      if (r < hs && less(r, m)) m = r;
      if (m == i) break;
      swap_at(i, m);
      i = m;
    }
    return w;
  };
  for (int w = 0; w < W; ++w)
    if (rem[w] > 0) push(w);
  for (long long u = 0; u < ng; ++u) {
    const int w = pop();
    place(u, w);
    load[w] += cost(u);
    if (--rem[w] > 0) push(w);
  }
  if (lone) place(N - 1, wl);
  std::memcpy(t, tmp, (size_t)n * sizeof(TileDesc));
}

}  // namespace melt
