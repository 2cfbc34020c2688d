// melt_forward_host: MelT features of a batch held in host memory.
//
// The batch is cut into chunks of whole clips; each chunk's samples are
// copied to a device slot, its tiles run through the forward kernel and its
// features are copied back, all on one of kHostSlots internal streams.  The
// streams take chunks in turn, so the host-to-device copy of one chunk, the
// kernel of another and the device-to-host copy of a third run at the same
// time on the copy engines and the SMs.  The tile list of every chunk (tile
// offsets relative to the chunk's device slot) is planned once per batch
// layout and kept on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "melt_internal.h"

namespace melt {

namespace {
constexpr int kHostSlots = 4;
constexpr int64_t kMinChunkFloats = 1 << 20;   // 4 MB of samples
constexpr int kTargetChunks = 8;

struct Chunk {
  int c0, c1;             // clips [c0, c1)
  int64_t span0, span1;   // host sample range copied (floats, 4-aligned start)
  int64_t row0, rows;     // output rows
  int64_t tile0, tiles;   // tiles in the device list
};
}  // namespace

struct HostPipe {
  int device = 0;
  cudaStream_t streams[kHostSlots] = {};
  cudaEvent_t done[kHostSlots] = {};
  cudaEvent_t start = nullptr;
  float* d_wave[kHostSlots] = {};
  float* d_out[kHostSlots] = {};
  size_t wave_cap = 0, out_cap = 0;  // floats per slot
  TileDesc* d_tiles = nullptr;
  size_t tiles_cap = 0;
  std::vector<TileDesc> h_tiles;
  std::vector<Chunk> chunks;
  // batch layout the plan is for
  int key_batch = -1;
  std::vector<int64_t> key_off, key_len;
};

void host_pipe_free(HostPipe* hp) {
  if (!hp) return;
  for (int i = 0; i < kHostSlots; ++i) {
    if (hp->streams[i]) cudaStreamSynchronize(hp->streams[i]), cudaStreamDestroy(hp->streams[i]);
    if (hp->done[i]) cudaEventDestroy(hp->done[i]);
    cudaFree(hp->d_wave[i]);
    cudaFree(hp->d_out[i]);
  }
  if (hp->start) cudaEventDestroy(hp->start);
  cudaFree(hp->d_tiles);
  delete hp;
}

namespace {

melt_status st_of(cudaError_t e) {
  if (e == cudaSuccess) return MELT_OK;
  return e == cudaErrorMemoryAllocation ? MELT_ERR_OOM : MELT_ERR_CUDA;
}

#define HCUDA(call)                                  \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return st_of(e_);         \
  } while (0)

melt_status pipe_init(HostPipe* hp) {
  for (int i = 0; i < kHostSlots; ++i) {
    HCUDA(cudaStreamCreateWithFlags(&hp->streams[i], cudaStreamNonBlocking));
    HCUDA(cudaEventCreateWithFlags(&hp->done[i], cudaEventDisableTiming));
  }
  HCUDA(cudaEventCreateWithFlags(&hp->start, cudaEventDisableTiming));
  return MELT_OK;
}

bool same_key(const HostPipe* hp, const int64_t* offsets, const int64_t* lengths, int batch) {
  if (hp->key_batch != batch) return false;
  if ((offsets == nullptr) != hp->key_off.empty()) return false;
  if (std::memcmp(hp->key_len.data(), lengths, sizeof(int64_t) * batch) != 0) return false;
  return !offsets || std::memcmp(hp->key_off.data(), offsets, sizeof(int64_t) * batch) == 0;
}

// Chunks and their tile lists for one batch layout; grows device buffers.
melt_status plan_host(melt_basis* b, HostPipe* hp, const int64_t* offsets, const int64_t* lengths,
                      int batch, int n_out) {
  std::vector<int64_t> off(batch);
  int64_t o = 0, total = 0;
  for (int c = 0; c < batch; ++c) {
    if (lengths[c] < 0) return MELT_ERR_ARG;
    off[c] = offsets ? offsets[c] : o;
    if (off[c] < 0 || (off[c] & 3)) return MELT_ERR_ARG;
    if (c > 0 && off[c] < off[c - 1]) return MELT_ERR_ARG;  // chunk spans need ordered clips
    o += (lengths[c] + 3) & ~int64_t(3);
    total += (lengths[c] + 3) & ~int64_t(3);
  }
  const int64_t target = std::max<int64_t>(kMinChunkFloats, total / kTargetChunks + 1);
  hp->chunks.clear();
  hp->h_tiles.clear();
  size_t wave_max = 4, out_max = 4;
  int64_t row = 0;
  for (int c = 0; c < batch;) {
    Chunk ch;
    ch.c0 = c;
    ch.span0 = off[c];
    ch.span1 = off[c];
    ch.row0 = row;
    ch.rows = 0;
    ch.tile0 = (int64_t)hp->h_tiles.size();
    while (c < batch && (c == ch.c0 || ch.span1 - ch.span0 < target)) {
      const int64_t L = lengths[c];
      const int64_t T = basis_frames(b, L);
      // tiles of this clip, offsets relative to the chunk's device slot
      std::vector<TileDesc> tl((size_t)((T + kTileFrames - 1) / kTileFrames) + 1);
      const long long n = plan_clip_tiles(b, off[c] - ch.span0, L, ch.rows, c, 0, tl.data(),
                                          (long long)tl.size());
      if (n < 0) return MELT_ERR_ARG;
      hp->h_tiles.insert(hp->h_tiles.end(), tl.begin(), tl.begin() + n);
      ch.span1 = std::max(ch.span1, off[c] + ((L + 3) & ~int64_t(3)));
      ch.rows += T;
      ++c;
    }
    ch.c1 = c;
    ch.tiles = (int64_t)hp->h_tiles.size() - ch.tile0;
    row += ch.rows;
    wave_max = std::max(wave_max, (size_t)(ch.span1 - ch.span0));
    out_max = std::max(out_max, (size_t)(ch.rows * n_out));
    hp->chunks.push_back(ch);
  }
  for (auto& t : hp->h_tiles)
    if (t.n_frames > kTileFrames || t.n_frames < 1) return MELT_ERR_ARG;
  // device buffers: synchronise the slots before replacing anything they may use
  for (int i = 0; i < kHostSlots; ++i) HCUDA(cudaStreamSynchronize(hp->streams[i]));
  if (wave_max > hp->wave_cap) {
    for (int i = 0; i < kHostSlots; ++i) {
      cudaFree(hp->d_wave[i]);
      hp->d_wave[i] = nullptr;
    }
    hp->wave_cap = 0;
    for (int i = 0; i < kHostSlots; ++i) HCUDA(melt::dev_alloc(&hp->d_wave[i], wave_max * sizeof(float)));
    hp->wave_cap = wave_max;
  }
  if (out_max > hp->out_cap) {
    for (int i = 0; i < kHostSlots; ++i) {
      cudaFree(hp->d_out[i]);
      hp->d_out[i] = nullptr;
    }
    hp->out_cap = 0;
    for (int i = 0; i < kHostSlots; ++i) HCUDA(melt::dev_alloc(&hp->d_out[i], out_max * sizeof(float)));
    hp->out_cap = out_max;
  }
  const size_t nt = std::max<size_t>(hp->h_tiles.size(), 1);
  if (nt > hp->tiles_cap) {
    cudaFree(hp->d_tiles);
    hp->d_tiles = nullptr;
    hp->tiles_cap = 0;
    HCUDA(melt::dev_alloc(&hp->d_tiles, nt * sizeof(TileDesc)));
    hp->tiles_cap = nt;
  }
  HCUDA(cudaMemcpy(hp->d_tiles, hp->h_tiles.data(), hp->h_tiles.size() * sizeof(TileDesc),
                   cudaMemcpyHostToDevice));
  hp->key_batch = batch;
  hp->key_len.assign(lengths, lengths + batch);
  if (offsets) hp->key_off.assign(offsets, offsets + batch); else hp->key_off.clear();
  return MELT_OK;
}

}  // namespace
}  // namespace melt

using namespace melt;

extern "C" melt_status melt_forward_host(melt_basis* b, const float* wave, const int64_t* offsets,
                                         const int64_t* lengths, int batch, float* out,
                                         void* stream_v) {
  if (!b || batch < 0 || (batch > 0 && (!wave || !lengths || !out))) return MELT_ERR_ARG;
  if (batch == 0) return MELT_OK;
  int dev = 0;
  HCUDA(cudaGetDevice(&dev));
  if (dev != basis_device(b)) return MELT_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)stream_v;
  HostPipe*& hp = basis_host_pipe(b);
  if (!hp) {
    hp = new (std::nothrow) HostPipe();
    if (!hp) return MELT_ERR_OOM;
    hp->device = dev;
    const melt_status st = pipe_init(hp);
    if (st != MELT_OK) {
      host_pipe_free(hp);
      hp = nullptr;
      return st;
    }
  }
  const int n_out = melt_num_outputs(b);
  if (!same_key(hp, offsets, lengths, batch)) {
    const melt_status st = plan_host(b, hp, offsets, lengths, batch, n_out);
    if (st != MELT_OK) {
      hp->key_batch = -1;
      return st;
    }
  }
  // every internal stream starts after the work already queued on `stream`
  HCUDA(cudaEventRecord(hp->start, stream));
  for (int i = 0; i < kHostSlots; ++i) HCUDA(cudaStreamWaitEvent(hp->streams[i], hp->start, 0));
  for (size_t k = 0; k < hp->chunks.size(); ++k) {
    const Chunk& ch = hp->chunks[k];
    const int s = (int)(k % kHostSlots);
    cudaStream_t cs = hp->streams[s];
    HCUDA(cudaMemcpyAsync(hp->d_wave[s], wave + ch.span0, (size_t)(ch.span1 - ch.span0) * sizeof(float),
                          cudaMemcpyHostToDevice, cs));
    if (ch.tiles > 0) {
      const melt_status st = launch_forward_tiles(b, hp->d_wave[s], hp->d_tiles + ch.tile0,
                                                  (int)ch.tiles, hp->d_out[s], ch.rows, cs);
      if (st != MELT_OK) return st;
      HCUDA(cudaMemcpyAsync(out + ch.row0 * n_out, hp->d_out[s], (size_t)(ch.rows * n_out) * sizeof(float),
                            cudaMemcpyDeviceToHost, cs));
    }
  }
  // `stream` continues after every chunk is back in host memory
  for (int i = 0; i < kHostSlots; ++i) {
    HCUDA(cudaEventRecord(hp->done[i], hp->streams[i]));
    HCUDA(cudaStreamWaitEvent(stream, hp->done[i], 0));
  }
  return MELT_OK;
}
