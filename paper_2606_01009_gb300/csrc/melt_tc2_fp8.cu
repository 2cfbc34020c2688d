// Instantiations of the CTA-pair tensor-core MelT kernel with FP8 e4m3
// operands (per-row power-of-two scales applied by block-scaled MMAs).
#include "melt_tc2_kernel.cuh"

namespace melt {
namespace tc {

KernelFn kernel_for_pair_fp8(bool mfcc, int nch, bool dtc) { return pick_pair_fp8_kernel<>(mfcc, nch, dtc); }

}  // namespace tc
}  // namespace melt
