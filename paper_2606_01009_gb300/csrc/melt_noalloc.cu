// melt_forward_noalloc: the MelT forward without any allocation at call time.
//
// Who needs it: callers that must not allocate device memory once they are
// running.  Typical cases are a real-time audio thread (cudaMalloc can block
// on driver locks and synchronise the device, which breaks a latency budget),
// a process where another framework's caching allocator has already reserved
// the device memory (a further cudaMalloc may fail although the work fits),
// and embedded deployments that fix their memory footprint at start-up.
// melt_forward allocates its device tile list and pinned staging on first use
// and whenever a larger batch arrives; this variant never does.
//
// How: the per-call scratch the kernels need - the tile list (one 32-byte
// descriptor per 128 frames of a clip) - lives in a file-scope __device__
// array of kMaxTiles entries (512 KiB), which every device that loads the
// library holds until the process exits.  Its device address is looked up
// once per device with cudaGetSymbolAddress; host code never passes the
// symbol itself to a kernel.  The tiles are planned into a file-scope host
// array and copied with cudaMemcpyAsync from that pageable buffer: the driver
// stages the bytes before the call returns, so the host array is free for the
// next call at once, but the copy may first wait for the work already queued
// on the stream.  A pageable copy cannot be replayed from a CUDA graph, so
// the call refuses to run while its stream is being captured.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "melt_internal.h"

using namespace melt;

namespace {

constexpr long long kMaxTiles = 16384;  // 16384 tiles x 128 frames = 2,097,152 frames per call
constexpr int kMaxDevices = 64;

static __device__ __align__(256) TileDesc g_noalloc_tiles[kMaxTiles];

std::mutex g_mu;                           // guards the host array and the per-device table
TileDesc* g_dev_tiles[kMaxDevices] = {};   // device address of g_noalloc_tiles, per device
TileDesc g_host_tiles[kMaxTiles];          // host-side plan of the current call

}  // namespace

extern "C" melt_status melt_forward_noalloc(melt_basis* basis, const float* wave,
                                            const int64_t* offsets, const int64_t* lengths,
                                            int batch, float* out, void* stream_v) {
  if (!basis || batch < 0 || (batch > 0 && (!lengths || !wave || !out))) return MELT_ERR_ARG;
  if (((uintptr_t)wave & 15) || ((uintptr_t)out & 15)) return MELT_ERR_ARG;
  if (batch == 0) return MELT_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MELT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices || dev != basis_device(basis)) return MELT_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)stream_v;
  // the plan is copied from pageable memory, which a captured graph cannot replay
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return MELT_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return MELT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_tiles[dev]) {
    // set-up, once per device, with that device current
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tiles);
    if (e != cudaSuccess || !p) return MELT_ERR_CUDA;
    g_dev_tiles[dev] = static_cast<TileDesc*>(p);
  }
  const long long n = plan_tiles_into(basis, offsets, lengths, batch, g_host_tiles, kMaxTiles);
  if (n < 0) return MELT_ERR_ARG;  // -1: bad offset/length; -2: more than kMaxTiles tiles
  if (n == 0) return MELT_OK;
  int64_t rows = 0;  // the tiles need not be in output-row order
  for (long long i = 0; i < n; ++i) rows = std::max<int64_t>(rows, g_host_tiles[i].out_row + g_host_tiles[i].n_frames);
  // Every field of the n descriptors is written here; nothing in the array
  // has to start at zero.
  if (cudaMemcpyAsync(g_dev_tiles[dev], g_host_tiles, (size_t)n * sizeof(TileDesc),
                      cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return MELT_ERR_CUDA;
  return launch_forward_tiles(basis, wave, g_dev_tiles[dev], (int)n, out, rows, stream);
}
