// Instantiations of the CTA-pair tensor-core MelT kernel with the correction
// MLP fused in its epilogue (BF16).
#include "melt_diag.h"
#include "melt_tc2_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_pair_mlp(int nch) { return pick_pair_mlp_kernel<>(nch); }

// The fused epilogue's GELU on n values (diagnostic: checked against the exact function).
__global__ void gelu_diag_kernel(const float* h, float* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = gelu_poly(h[i]);
}

// The epilogues' natural log on n values (diagnostic: checked against the exact function).
__global__ void log_diag_kernel(const float* x, float* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fast_ln(x[i]);
}

}  // namespace tc
}  // namespace melt

extern "C" melt_status melt_diag_log(const float* x, float* y, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return MELT_ERR_ARG;
  if (n == 0) return MELT_OK;
  const long long blocks = (n + 255) / 256;
  melt::tc::log_diag_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? MELT_OK : MELT_ERR_CUDA;
}

extern "C" melt_status melt_diag_gelu(const float* h, float* y, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!h || !y))) return MELT_ERR_ARG;
  if (n == 0) return MELT_OK;
  const long long blocks = (n + 255) / 256;
  melt::tc::gelu_diag_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(h, y, n);
  return cudaGetLastError() == cudaSuccess ? MELT_OK : MELT_ERR_CUDA;
}
