// walk_mt_fp32.cu -- the precision form of the walker step (FP32 offset,
// Kahan sums) with absorbing membranes (Sec. 2.1.3,
// magnetization transfer), for each particle-membrane interaction.
#include "walk_kernel.cuh"
#include "rms_internal.h"

namespace rms {
template cudaError_t launch_walk<float, kInteractEC, true>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                    const Tables<float> &, const WalkerState<float> &,
                                                    const RunCtl &, int64_t, int64_t);
template cudaError_t launch_walk<float, kInteractRS, true>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                    const Tables<float> &, const WalkerState<float> &,
                                                    const RunCtl &, int64_t, int64_t);
template cudaError_t launch_walk<float, kInteractERL, true>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                    const Tables<float> &, const WalkerState<float> &,
                                                    const RunCtl &, int64_t, int64_t);
}  // namespace rms
