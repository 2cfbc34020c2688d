// Instantiations of the tensor-core MelT kernel with the log-Mel epilogue.
#include "melt_tc_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_plain(int prec, int nch, bool stft) {
  if (stft) {
    switch (prec) {
      case MELT_BF16: return melt_tc_kernel<MELT_BF16, 1, false, true>;
      case MELT_BF16X3: return melt_tc_kernel<MELT_BF16X3, 1, false, true>;
      default: return nullptr;
    }
  }
  switch (prec) {
    case MELT_BF16: return pick_kernel<MELT_BF16, false>(nch);
    case MELT_BF16X3: return pick_kernel<MELT_BF16X3, false>(nch);
    default: return nullptr;
  }
}

}  // namespace tc
}  // namespace melt
