/*
 * melt_diag.h - diagnostics of libmelt, outside the feature path.
 */
#ifndef MELT_DIAG_H_
#define MELT_DIAG_H_

#include "melt.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * melt_diag_wait_timeout - exercises the failure path of the library's
 *   bounded waits without faulting the GPU.  Every wait in the kernels (on an
 *   mbarrier, for a copy, a peer or a pipeline stage) gives up after 1 s of
 *   GPU time, latches MELT_ERR_TIMEOUT in the basis, lets its kernel finish
 *   and leaves the context usable.  This call launches one thread that waits
 *   on an mbarrier nothing arrives on, so that path runs: the next melt_sync
 *   on the stream returns MELT_ERR_TIMEOUT (about 1 s later) and clears it.
 *   basis   a basis of the current device (its error word receives the bit)
 *   stream  cudaStream_t as void* (NULL = legacy default stream)
 *   Errors: MELT_ERR_ARG for a NULL basis or one of another device,
 *   MELT_ERR_CUDA if the launch fails.
 */
melt_status melt_diag_wait_timeout(melt_basis* basis, void* stream);

/*
 * melt_diag_gelu - evaluates, on n device floats h, the GELU that the CTA-pair
 *   kernel's fused correction epilogue applies to the hidden layer: GELU(h) =
 *   h Phi(h) (the exact-erf form the model is trained with), computed as
 *   max(h, 0) - |h| Q(|h|), the normal tail Q(t) = 2^(S(t) - t^2 log2(e) / 2)
 *   with a polynomial S.  Stated accuracy against the exact function:
 *   relative error <= 2e-5 for |h| <= 5, absolute error <= 3e-6 everywhere.  The paper
 *   has no counterpart (it evaluates no correction layer); this entry point
 *   lets a test check that bound.
 *   h, y    device float[n] (may be the same array)
 *   stream  cudaStream_t as void*; asynchronous
 *   Errors: MELT_ERR_ARG for n < 0 or NULL pointers, MELT_ERR_CUDA if the launch fails.
 */
melt_status melt_diag_gelu(const float* h, float* y, int64_t n, void* stream);

/*
 * melt_diag_log - evaluates, on n device floats x, the natural log that the
 *   tensor-core kernels' epilogues take of S + eps (Eq. 8): log2(x) from the
 *   hardware approximation with subnormal inputs flushed to zero, times ln 2.
 *   The paper has no counterpart; this entry point lets a test check the
 *   log's error against the exact function over every binade (the parity
 *   bounds assume absolute error <= 2^-21 for x in [0.5, 2] and <= 4 ulp of
 *   the result elsewhere).
 *   x, y    device float[n] (may be the same array); x > 0 normal
 *   stream  cudaStream_t as void*; asynchronous
 *   Errors: MELT_ERR_ARG for n < 0 or NULL pointers, MELT_ERR_CUDA if the launch fails.
 */
melt_status melt_diag_log(const float* x, float* y, int64_t n, void* stream);

/*
 * melt_diag_alloc_count - number of device allocations (cudaMalloc) and
 *   page-locked host allocations (cudaMallocHost) the library has made in
 *   this process so far, over all devices and threads.  The paper has no
 *   counterpart: it lets a test show that an entry point allocated nothing
 *   (the count is the same before and after the call).  Never fails.
 */
long long melt_diag_alloc_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MELT_DIAG_H_ */
