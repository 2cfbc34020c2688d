// Grouped launch: one batch whose clips use different bases (Sec. V batches
// many clips per call; here the batch may also mix frame geometries).
//
// A call plans one work list of tiles (basis, clip, 128-frame run), grouped
// by basis so that each basis's tiles are contiguous, and runs one persistent
// kernel per basis over its range.  Output rows follow the batch order of the
// clips, whatever basis each clip uses, so the result equals melt_forward on
// each clip with its own basis.  The work list of a batch layout is copied to
// the device once and kept; with graphs enabled the per-basis launches are
// captured once into a CUDA graph and later calls with the same layout replay
// it with a single cudaGraphLaunch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "melt_internal.h"

using namespace melt;

namespace {

constexpr int kCacheEntries = 8;

struct GroupEntry {
  // batch layout (cache key)
  const float* wave = nullptr;
  float* out = nullptr;
  int batch = 0;
  bool has_offsets = false;
  std::vector<int64_t> offsets, lengths;
  std::vector<int32_t> ids;
  // device work list and launches
  TileDesc* d_tiles = nullptr;
  std::vector<long long> first, count;  // per basis: range in d_tiles
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;           // recorded after the last launch that read d_tiles
  unsigned long long last_use = 0;
};

void free_entry(GroupEntry* e) {
  if (!e) return;
  if (e->done) cudaEventSynchronize(e->done);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->d_tiles) cudaFree(e->d_tiles);
  if (e->done) cudaEventDestroy(e->done);
  delete e;
}

}  // namespace

struct melt_group {
  int device = 0;
  int flags = 0;
  std::vector<melt_basis*> bases;
  std::vector<GroupEntry*> cache;
  unsigned long long tick = 0;
  cudaStream_t capture = nullptr;  // private stream the graphs are captured on
  std::vector<TileDesc> host;      // planning scratch
  std::vector<int64_t> rows;       // planning scratch: first output row of each clip
  double split = 0.0;              // shared launch: the first basis's share of the clusters (0: by work)
};

namespace {

bool same_layout(const GroupEntry* e, const float* wave, const int64_t* offsets,
                 const int64_t* lengths, const int32_t* ids, int batch, const float* out) {
  if (e->wave != wave || e->out != out || e->batch != batch) return false;
  if (e->has_offsets != (offsets != nullptr)) return false;
  if (std::memcmp(e->lengths.data(), lengths, sizeof(int64_t) * batch) != 0) return false;
  if (std::memcmp(e->ids.data(), ids, sizeof(int32_t) * batch) != 0) return false;
  return !offsets || std::memcmp(e->offsets.data(), offsets, sizeof(int64_t) * batch) == 0;
}

melt_status launch_all(melt_group* g, const GroupEntry* e, cudaStream_t stream) {
  if ((g->flags & MELT_GROUP_SHARED) && g->bases.size() == 2 && e->count[0] > 0 && e->count[1] > 0 &&
      e->count[0] <= 0x7fffffffLL && e->count[1] <= 0x7fffffffLL) {
    // both bases in one persistent launch where their kernels allow it
    bool launched = false;
    const melt_status st = launch_forward_tiles_pair2(g->bases[0], e->d_tiles + e->first[0], (int)e->count[0],
                                                      g->bases[1], e->d_tiles + e->first[1], (int)e->count[1],
                                                      e->wave, e->out, g->split, stream, &launched);
    if (st != MELT_OK || launched) return st;
  }
  for (size_t k = 0; k < g->bases.size(); ++k) {
    if (e->count[k] == 0) continue;
    const melt_status st = launch_forward_tiles(g->bases[k], e->wave, e->d_tiles + e->first[k],
                                                (int)e->count[k], e->out, 0 /* grouped bases carry no correction */, stream);
    if (st != MELT_OK) return st;
  }
  return MELT_OK;
}

// Plan, upload and (optionally) capture a new batch layout.
melt_status make_entry(melt_group* g, const float* wave, const int64_t* offsets,
                       const int64_t* lengths, const int32_t* ids, int batch, float* out,
                       cudaStream_t stream, GroupEntry** out_entry) {
  const int nb = (int)g->bases.size();
  // output rows in batch order; validate every clip first
  g->rows.resize(batch);
  int64_t row = 0, off = 0;
  std::vector<int64_t> offs(batch);
  for (int c = 0; c < batch; ++c) {
    const int64_t L = lengths[c];
    const int32_t k = ids[c];
    if (L < 0 || k < 0 || k >= nb) return MELT_ERR_ARG;
    const int64_t o = offsets ? offsets[c] : off;
    if (o < 0 || (o & 3)) return MELT_ERR_ARG;
    off += (L + 3) & ~int64_t(3);
    offs[c] = o;
    g->rows[c] = row;
    row += basis_frames(g->bases[k], L);
  }
  GroupEntry* e = new (std::nothrow) GroupEntry;
  if (!e) return MELT_ERR_OOM;
  e->first.assign(nb, 0);
  e->count.assign(nb, 0);
  g->host.clear();
  for (int k = 0; k < nb; ++k) {
    e->first[k] = (long long)g->host.size();
    for (int c = 0; c < batch; ++c) {
      if (ids[c] != k) continue;
      const int64_t T = basis_frames(g->bases[k], lengths[c]);
      const size_t at = g->host.size();
      g->host.resize(at + (size_t)((T + kTileFrames - 1) / kTileFrames));
      const long long n = plan_clip_tiles(g->bases[k], offs[c], lengths[c], g->rows[c], c, k,
                                          g->host.data() + at, (long long)(g->host.size() - at));
      if (n < 0) {
        delete e;
        return MELT_ERR_ARG;
      }
    }
    e->count[k] = (long long)g->host.size() - e->first[k];
    if (e->count[k] > 0x7fffffffLL) {
      delete e;
      return MELT_ERR_ARG;
    }
  }
  e->wave = wave;
  e->out = out;
  e->batch = batch;
  e->has_offsets = offsets != nullptr;
  if (offsets) e->offsets.assign(offsets, offsets + batch);
  e->lengths.assign(lengths, lengths + batch);
  e->ids.assign(ids, ids + batch);
  melt_status st = MELT_OK;
  if (cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming) != cudaSuccess) st = MELT_ERR_CUDA;
  const size_t bytes = std::max<size_t>(g->host.size(), 1) * sizeof(TileDesc);
  if (st == MELT_OK && melt::dev_alloc(&e->d_tiles, bytes) != cudaSuccess) st = MELT_ERR_OOM;
  // pageable source: the call returns once the bytes are staged, so g->host may be reused
  if (st == MELT_OK && !g->host.empty() &&
      cudaMemcpyAsync(e->d_tiles, g->host.data(), g->host.size() * sizeof(TileDesc),
                      cudaMemcpyHostToDevice, stream) != cudaSuccess)
    st = MELT_ERR_CUDA;
  if (st == MELT_OK && !(g->flags & MELT_GROUP_NO_GRAPH) && !g->host.empty()) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      st = MELT_ERR_CUDA;
    } else {
      const melt_status ls = launch_all(g, e, g->capture);
      const cudaError_t ce = cudaStreamEndCapture(g->capture, &graph);
      if (ls != MELT_OK) st = ls;
      else if (ce != cudaSuccess || !graph) st = MELT_ERR_CUDA;
      if (st == MELT_OK && cudaGraphInstantiate(&e->exec, graph, 0) != cudaSuccess) {
        e->exec = nullptr;
        st = MELT_ERR_CUDA;
      }
      if (graph) cudaGraphDestroy(graph);
    }
  }
  if (st != MELT_OK) {
    cudaStreamSynchronize(stream);  // the upload may still be reading nothing of ours, but be safe
    free_entry(e);
    return st;
  }
  // insert, evicting the least recently used layout
  if ((int)g->cache.size() >= kCacheEntries) {
    auto lru = std::min_element(g->cache.begin(), g->cache.end(),
                                [](const GroupEntry* a, const GroupEntry* b) {
                                  return a->last_use < b->last_use;
                                });
    free_entry(*lru);
    g->cache.erase(lru);
  }
  g->cache.push_back(e);
  *out_entry = e;
  return MELT_OK;
}

}  // namespace

extern "C" {

melt_status melt_group_create(melt_basis* const* bases, int n_bases, int flags, melt_group** out) {
  if (!out || !bases || n_bases < 1 || n_bases > MELT_MAX_GROUPS) return MELT_ERR_ARG;
  if (flags & ~(MELT_GROUP_NO_GRAPH | MELT_GROUP_SHARED)) return MELT_ERR_ARG;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MELT_ERR_CUDA;
  for (int k = 0; k < n_bases; ++k) {
    if (!bases[k] || basis_device(bases[k]) != dev) return MELT_ERR_ARG;
    if (melt_num_outputs(bases[k]) != melt_num_outputs(bases[0])) return MELT_ERR_ARG;
  }
  melt_group* g = new (std::nothrow) melt_group;
  if (!g) return MELT_ERR_OOM;
  g->device = dev;
  g->flags = flags;
  g->bases.assign(bases, bases + n_bases);
  if (cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking) != cudaSuccess) {
    delete g;
    return MELT_ERR_CUDA;
  }
  *out = g;
  return MELT_OK;
}

melt_status melt_forward_grouped(melt_group* g, const float* wave, const int64_t* offsets,
                                 const int64_t* lengths, const int32_t* basis_of, int batch,
                                 float* out, void* stream_v) {
  if (!g || batch < 0 || (batch > 0 && (!lengths || !basis_of || !wave || !out)))
    return MELT_ERR_ARG;
  if (((uintptr_t)wave & 15) || ((uintptr_t)out & 15)) return MELT_ERR_ARG;
  if (batch == 0) return MELT_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MELT_ERR_CUDA;
  if (dev != g->device) return MELT_ERR_ARG;
  for (melt_basis* b : g->bases)
    if (basis_correction(b)) return MELT_ERR_UNSUPPORTED;  // corrections act on contiguous rows
  cudaStream_t stream = (cudaStream_t)stream_v;
  GroupEntry* e = nullptr;
  for (GroupEntry* c : g->cache)
    if (same_layout(c, wave, offsets, lengths, basis_of, batch, out)) {
      e = c;
      break;
    }
  if (!e) {
    const melt_status st = make_entry(g, wave, offsets, lengths, basis_of, batch, out, stream, &e);
    if (st != MELT_OK) return st;
  }
  e->last_use = ++g->tick;
  melt_status st = MELT_OK;
  if (e->exec) {
    if (cudaGraphLaunch(e->exec, stream) != cudaSuccess) st = MELT_ERR_CUDA;
  } else {
    st = launch_all(g, e, stream);
  }
  if (st != MELT_OK) return st;
  if (cudaEventRecord(e->done, stream) != cudaSuccess) return MELT_ERR_CUDA;
  return MELT_OK;
}

melt_status melt_group_autotune(melt_group* g, const float* wave, const int64_t* offsets, const int64_t* lengths,
                                const int32_t* basis_of, int batch, float* out, void* stream_v, int reps,
                                const char* path, int* hit) {
  if (hit) *hit = 0;
  if (!g || reps < 1 || batch < 0 || (batch > 0 && (!lengths || !basis_of || !wave || !out))) return MELT_ERR_ARG;
  if (((uintptr_t)wave & 15) || ((uintptr_t)out & 15)) return MELT_ERR_ARG;
  if (batch == 0) return MELT_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MELT_ERR_CUDA;
  if (dev != g->device) return MELT_ERR_ARG;
  for (melt_basis* b : g->bases)
    if (basis_correction(b)) return MELT_ERR_UNSUPPORTED;
  cudaStream_t stream = (cudaStream_t)stream_v;
  const int nb = (int)g->bases.size();
  // the batch's work lists, without a graph: plans change between launches
  const int flags = g->flags;
  g->flags |= MELT_GROUP_NO_GRAPH;
  GroupEntry* e = nullptr;
  melt_status st = make_entry(g, wave, offsets, lengths, basis_of, batch, out, stream, &e);
  g->flags = flags;
  if (st != MELT_OK) return st;
  // key: device, then each basis's configuration and tile-count class
  char key[4096], part[256], rest[2048];
  int kl = 0;
  if (!device_token(g->device, part, sizeof(part))) st = MELT_ERR_CUDA;
  if (st == MELT_OK) kl = std::snprintf(key, sizeof(key), "melt-group-plan-v1 %s %d", part, nb);
  for (int k = 0; st == MELT_OK && k < nb; ++k) {
    basis_plan_key(g->bases[k], part, sizeof(part));
    kl += std::snprintf(key + kl, sizeof(key) - kl, " | %s %d", part, tile_class(e->count[k]));
    if (kl >= (int)sizeof(key)) st = MELT_ERR_ARG;
  }
  // a cached line: one plan per basis ("-" for a basis without plans)
  bool applied = false;
  if (st == MELT_OK && path && cache_lookup(path, key, rest, sizeof(rest))) {
    std::vector<melt_plan> pl(nb);
    std::vector<char> has(nb, 0);
    const char* r = rest;
    bool ok = true;
    for (int k = 0; ok && k < nb; ++k) {
      while (*r == ' ') ++r;
      if (*r == '-') {
        ++r;
        continue;
      }
      int used = 0;
      ok = parse_plan(r, &pl[k], &used);
      r += used;
      has[k] = 1;
    }
    for (int k = 0; ok && k < nb; ++k)
      if (has[k]) {
        melt_plan cur;
        ok = melt_plan_get(g->bases[k], &cur) == MELT_OK;  // rejects bases without plans
      }
    if (ok) {
      // all or nothing: every plan must fit before any is set
      std::vector<melt_plan> prev(nb);
      for (int k = 0; ok && k < nb; ++k)
        if (has[k]) {
          melt_plan_get(g->bases[k], &prev[k]);
          ok = melt_plan_set(g->bases[k], &pl[k]) == MELT_OK;
        }
      if (!ok)
        for (int k = 0; k < nb; ++k)
          if (has[k]) melt_plan_set(g->bases[k], &prev[k]);
      applied = ok;
    }
  }
  // otherwise tune one basis at a time, timing the whole grouped launch
  std::vector<melt_plan> chosen(nb);
  std::vector<char> tuned(nb, 0);
  if (st == MELT_OK && !applied) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = MELT_ERR_CUDA;
    melt_plan cands[64];
    for (int k = 0; st == MELT_OK && k < nb; ++k) {
      const int n = e->count[k] > 0 ? basis_plan_candidates(g->bases[k], cands, 64) : 0;
      if (n < 1) continue;
      float best_ms = 1e30f;
      int best_i = -1;
      for (int i = 0; st == MELT_OK && i < n; ++i) {
        if (melt_plan_set(g->bases[k], &cands[i]) != MELT_OK) continue;
        st = launch_all(g, e, stream);  // warm-up
        if (st == MELT_OK && cudaEventRecord(e0, stream) != cudaSuccess) st = MELT_ERR_CUDA;
        for (int r = 0; r < reps && st == MELT_OK; ++r) st = launch_all(g, e, stream);
        if (st == MELT_OK && cudaEventRecord(e1, stream) != cudaSuccess) st = MELT_ERR_CUDA;
        if (st == MELT_OK && cudaEventSynchronize(e1) != cudaSuccess) st = MELT_ERR_CUDA;
        float ms = 0.f;
        if (st == MELT_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best_i = i;
        }
      }
      if (st == MELT_OK && best_i >= 0) {
        melt_plan_set(g->bases[k], &cands[best_i]);
        chosen[k] = cands[best_i];
        tuned[k] = 1;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st == MELT_OK) st = melt_group_sync(g, stream);
    if (st == MELT_OK && path) {
      int rl = 0;
      for (int k = 0; k < nb && rl < (int)sizeof(rest); ++k) {
        if (rl) rest[rl++] = ' ';
        if (tuned[k]) rl += format_plan(chosen[k], rest + rl, sizeof(rest) - rl);
        else rl += std::snprintf(rest + rl, sizeof(rest) - rl, "-");
      }
      if (rl < (int)sizeof(rest)) cache_append(path, key, rest);
    }
  }
  // every cached layout (this batch's included; graphs captured with the
  // earlier plans too) is dropped, so the next call plans and captures anew
  cudaStreamSynchronize(stream);
  for (GroupEntry* c : g->cache) free_entry(c);
  g->cache.clear();
  if (st == MELT_OK && hit) *hit = applied ? 1 : 0;
  return st;
}

melt_status melt_group_set_split(melt_group* g, double frac0) {
  if (!g || !(frac0 >= 0.0 && frac0 < 1.0)) return MELT_ERR_ARG;
  g->split = frac0;
  // recorded graphs hold the old split: drop them
  for (GroupEntry* e : g->cache) free_entry(e);
  g->cache.clear();
  return MELT_OK;
}

melt_status melt_group_sync(melt_group* g, void* stream) {
  if (!g) return MELT_ERR_ARG;
  melt_status first = MELT_OK;
  for (melt_basis* b : g->bases) {
    const melt_status st = melt_sync(b, stream);
    if (first == MELT_OK) first = st;
  }
  return first;
}

melt_status melt_group_destroy(melt_group* g) {
  if (!g) return MELT_OK;
  for (GroupEntry* e : g->cache) free_entry(e);
  if (g->capture) cudaStreamDestroy(g->capture);
  delete g;
  return MELT_OK;
}

}  // extern "C"
