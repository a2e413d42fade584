// walk_fp64.cu -- the plain form of the walker step: FP64 positions and
// phases.  Built with -fmad=false so that every +, -, *, / and sqrt is a
// separately rounded IEEE operation, as in the CPU FP64 reference.
#include "walk_kernel.cuh"
#include "rms_internal.h"

namespace rms {
template cudaError_t launch_walk<double, kInteractEC, false>(int, bool, dim3, cudaStream_t, const Geometry &,
                                         const Tables<double> &, const WalkerState<double> &,
                                         const RunCtl &, int64_t, int64_t);
template int batched_blocks_per_sm<double>(int);
template cudaError_t launch_walk_batched<double>(int, int32_t, cudaStream_t, const ReqDesc<double> *,
                                                const BlockTask *);
int walk_block_size() { return kWalkBlock; }
}  // namespace rms
