// Instantiation of the CTA-pair tensor-core MelT kernel with split-BF16
// operands (hi*hi + hi*lo + lo*hi per K-step).
#include "melt_tc2_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_pair_x3() { return pick_pair_x3_kernel<>(); }

}  // namespace tc
}  // namespace melt
