// Instantiations of the CTA-pair tensor-core MelT kernel with the correction
// MLP fused in its epilogue (BF16).
#include "melt_tc2_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_pair_mlp(int nch) { return pick_pair_mlp_kernel<>(nch); }

}  // namespace tc
}  // namespace melt
