// Instantiations of the CTA-pair tensor-core MelT kernel (BF16).
#include "melt_tc2_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_pair(bool mfcc, int nch, bool dtc) {
  return mfcc ? pick_pair_kernel<true>(nch, dtc) : pick_pair_kernel<false>(nch);
}

}  // namespace tc
}  // namespace melt
