// walk_fp32.cu -- the precision form of the walker step: voxel index plus an
// FP32 in-voxel offset, FP32 Kahan-compensated phase and relaxation sums.
// Built with FMA contraction allowed.
#include "walk_kernel.cuh"
#include "rms_internal.h"

namespace rms {
template cudaError_t launch_walk<float, kInteractEC, false>(int, bool, dim3, cudaStream_t, const Geometry &,
                                        const Tables<float> &, const WalkerState<float> &,
                                        const RunCtl &, int64_t, int64_t);
template int batched_blocks_per_sm<float>(int);
template cudaError_t launch_walk_batched<float>(int, int32_t, cudaStream_t, const ReqDesc<float> *,
                                               const BlockTask *);
}  // namespace rms
