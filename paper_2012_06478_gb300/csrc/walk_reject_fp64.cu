// walk_reject_fp64.cu -- the plain form of the walker step (FP64, no FMA
// contraction) for the alternative particle-membrane interactions of App. A
// and B: rejection sampling and the equal-step-length random leap (ERL).
// A unit of its own so that these kernels compile in parallel with the
// elastic-collision ones.
#include "walk_kernel.cuh"
#include "rms_internal.h"

namespace rms {
template cudaError_t launch_walk<double, kInteractRS, false>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                      const Tables<double> &, const WalkerState<double> &,
                                                      const RunCtl &, int64_t, int64_t);
template cudaError_t launch_walk<double, kInteractERL, false>(int, bool, dim3, cudaStream_t, const Geometry &,
                                                       const Tables<double> &, const WalkerState<double> &,
                                                       const RunCtl &, int64_t, int64_t);
}  // namespace rms
