// Instantiations of the tensor-core MelT kernel with the MFCC (DCT-II) epilogue.
#include "melt_tc_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_mfcc(int prec, int nch) {
  switch (prec) {
    case MELT_BF16: return pick_kernel<MELT_BF16, true>(nch);
    case MELT_BF16X3: return pick_kernel<MELT_BF16X3, true>(nch);
    default: return nullptr;
  }
}

}  // namespace tc
}  // namespace melt
