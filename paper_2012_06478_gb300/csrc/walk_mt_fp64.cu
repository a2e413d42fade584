// walk_mt_fp64.cu -- the plain form of the walker step (FP64, no FMA
// contraction) with absorbing membranes (Sec. 2.1.3,
// magnetization transfer), for each particle-membrane interaction.
#include "walk_kernel.cuh"
#include "rms_internal.h"

namespace rms {
template cudaError_t launch_walk<double, kInteractEC, true>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                    const Tables<double> &, const WalkerState<double> &,
                                                    const RunCtl &, int64_t, int64_t);
template cudaError_t launch_walk<double, kInteractRS, true>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                    const Tables<double> &, const WalkerState<double> &,
                                                    const RunCtl &, int64_t, int64_t);
template cudaError_t launch_walk<double, kInteractERL, true>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                    const Tables<double> &, const WalkerState<double> &,
                                                    const RunCtl &, int64_t, int64_t);
}  // namespace rms
