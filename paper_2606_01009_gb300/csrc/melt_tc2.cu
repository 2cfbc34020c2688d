// Instantiations of the CTA-pair tensor-core MelT kernel (BF16).
#include "melt_tc2_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_pair(bool mfcc, int nch, bool dtc) {
  return mfcc ? pick_pair_kernel<true>(nch, dtc) : pick_pair_kernel<false>(nch);
}

GroupKernelFn kernel_for_pair_group() { return melt_tc_pair_group_kernel<1, false, false, MELT_BF16>; }

}  // namespace tc
}  // namespace melt
