// walk_reject_fp32.cu -- the precision form of the walker step (FP32 offset,
// Kahan sums) for the alternative particle-membrane interactions of App. A
// and B: rejection sampling and the equal-step-length random leap (ERL).
#include "walk_kernel.cuh"
#include "rms_internal.h"

namespace rms {
template cudaError_t launch_walk<float, kInteractRS, false>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                     const Tables<float> &, const WalkerState<float> &,
                                                     const RunCtl &, int64_t, int64_t);
template cudaError_t launch_walk<float, kInteractERL, false>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                      const Tables<float> &, const WalkerState<float> &,
                                                      const RunCtl &, int64_t, int64_t);
}  // namespace rms
