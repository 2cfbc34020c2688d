// Internal types shared by the host planner and the kernels of libmelt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "melt.h"

namespace melt {

// Frames per tile.  Every kernel works on tiles of up to kTileFrames
// consecutive frames of one clip; 128 is the M extent of one tcgen05 MMA
// (cta_group::1) and of the SIMT kernel's CTA tile.
constexpr int kTileFrames = 128;

// One unit of work: up to kTileFrames consecutive frames of one clip.
struct TileDesc {
  int64_t in_off;     // float index in `wave` of sample 0 of the tile's first frame
  int64_t out_row;    // row of the tile's first frame in the packed output
  int32_t n_frames;   // valid frames in the tile, 1..kTileFrames
  int32_t n_samples;  // samples of the clip from in_off to the clip end (clamped to int32)
  int32_t group;      // basis group of the tile (grouped launch); 0 otherwise
  int32_t clip;       // clip index
};
static_assert(sizeof(TileDesc) == 32, "TileDesc is 32 bytes");

// Error bits latched by kernels in the per-basis device error word.
enum : int { kErrTimeout = 1, kErrBadTile = 2 };

// Parameters of the FP32 SIMT kernel.
struct SimtParams {
  const float* wave;
  const TileDesc* tiles;
  int n_tiles;
  const float* w32;   // [n_fft][2*mp]: interleaved (W_r[m][n], W_i[m][n]) per mel, zero-padded to mp mels
  const float* dct;   // [n_mfcc][n_mels] or nullptr
  float* out;
  int n_fft, hop, n_mels, mp, n_mfcc, n_out;
  float eps;
  int mode;           // 0: log-Mel / MFCC, 1: raw R|I components
};

// Every device allocation and every page-locked host allocation the library
// makes goes through these two calls, which count them (the count is read by
// melt_diag_alloc_count, so a test can show that a call allocated nothing).
cudaError_t dev_alloc_bytes(void** p, size_t bytes);
cudaError_t host_alloc_pinned_bytes(void** p, size_t bytes);
template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc_bytes(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t host_alloc_pinned(T** p, size_t bytes) {
  return host_alloc_pinned_bytes(reinterpret_cast<void**>(p), bytes);
}

// Launch the FP32 SIMT kernel for `p` (grid picked by the caller).
// Persistent launch: as many CTAs as fit on sm_count SMs (at most one per tile).
cudaError_t launch_simt(const SimtParams& p, int mj, int sm_count, cudaStream_t stream);
int simt_smem_bytes(int mj, int n_mels, int n_mfcc);

}  // namespace melt

// ---- helpers shared with the allocation-free entry point (melt_noalloc.cu)
namespace melt {

// Plans the tiles of a batch into dst[0..cap).  Returns the tile count,
// -1 for an invalid offset/length, -2 if more than `cap` tiles are needed.
long long plan_tiles_into(const melt_basis* b, const int64_t* offsets, const int64_t* lengths,
                          int batch, TileDesc* dst, long long cap);

// Launches the basis's forward kernel over `n_tiles` device tile descriptors
// and applies the attached correction to the `rows` output rows (fused in the
// kernel where the layout allows, else as a separate pass).
melt_status launch_forward_tiles(melt_basis* b, const float* wave, const TileDesc* d_tiles,
                                 int n_tiles, float* out, int64_t rows, cudaStream_t stream);

// Both bases' tiles in one persistent CTA-pair launch (the grouped call);
// *launched is false, with nothing enqueued, where the bases' kernels do not
// allow it (then the caller launches them one by one).
// frac0 is the first basis's share of the clusters (0: by tiles x n_fft).
melt_status launch_forward_tiles_pair2(melt_basis* b0, const TileDesc* t0, int n0, melt_basis* b1,
                                       const TileDesc* t1, int n1, const float* wave, float* out, double frac0,
                                       cudaStream_t stream, bool* launched);

// Frames of a clip of `len` samples under basis b: floor((len - N)/H) + 1, 0 if len < N.
int64_t basis_frames(const melt_basis* b, int64_t len);

// Tiles of one clip (samples from float index `off`, output rows from `row`)
// into dst[0..cap).  Returns the tile count, -2 if more than `cap` are needed.
long long plan_clip_tiles(const melt_basis* b, int64_t off, int64_t len, int64_t row, int clip,
                          int group, TileDesc* dst, long long cap);

// Device of the basis (the current device when it was created).
int basis_device(const melt_basis* b);

// Correction MLP attached to the basis (melt_basis_set_correction), or nullptr.
const melt_mlp* basis_correction(const melt_basis* b);

// Layout plans of the basis's tensor-core launch that fit the device, into
// out[0..cap); returns their count (0 for the FP32 form, which has no plans).
int basis_plan_candidates(const melt_basis* b, melt_plan* out, int cap);

// Plan cache files of melt_autotune_file / melt_group_autotune: the device
// name as one token, the basis configuration ("n_fft hop n_mels precision
// n_mfcc hidden bands"), the size class of a tile count (floor(log2)), and
// the seven fields of a plan written / read as text.
bool device_token(int device, char* buf, size_t n);
void basis_plan_key(const melt_basis* b, char* buf, size_t n);
int tile_class(long long tiles);
int format_plan(const melt_plan& p, char* buf, size_t n);
bool parse_plan(const char* s, melt_plan* p, int* used);
// Looks up the line starting with `key` + " : " in the file at `path`;
// copies what follows the colon into rest.  False if the file or line is missing.
bool cache_lookup(const char* path, const char* key, char* rest, size_t n);
// Appends "key : rest\n" to the file at `path` in one write (ignored if it cannot be opened).
void cache_append(const char* path, const char* key, const char* rest);

// Correction MLP (melt_mlp.cu): y = x + W2 GELU(W1 (x - mu)/sd + b1) + b2 over
// n rows of n_in bands; y == x allowed.
melt_status mlp_apply(const melt_mlp* p, const float* x, float* y, long long n, cudaStream_t s);
int mlp_inputs(const melt_mlp* p);
int mlp_device(const melt_mlp* p);
int mlp_hidden(const melt_mlp* p);
// The correction fused in the CTA-pair kernel's epilogue: shapes it supports,
// bytes of one CTA's half of its BF16 weight image, and the repacking of the
// current FP32 parameters into that image (asynchronous on s).
bool mlp_fused_shape_ok(int M, int Hd);
long long mlp_fused_half_bytes(int M, int Hd);
melt_status mlp_fused_image(const melt_mlp* p, void* d_img, cudaStream_t s);

}  // namespace melt

// ---- host-buffer entry point (melt_host.cu): per-basis pipeline state
namespace melt {
struct HostPipe;
// The basis's host pipeline slot (created on first use of melt_forward_host).
HostPipe*& basis_host_pipe(melt_basis* b);
// Release a pipeline (called when its basis is destroyed; NULL is a no-op).
void host_pipe_free(HostPipe* hp);
}  // namespace melt
