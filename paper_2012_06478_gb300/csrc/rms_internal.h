// rms_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "rms_device.cuh"

namespace rms {

template <typename Real, int IM, bool MT>
cudaError_t launch_walk(int n_shapes, bool hash, dim3 grid, cudaStream_t stream, const Geometry &g,
                        const Tables<Real> &t, const WalkerState<Real> &st, const RunCtl &ctl,
                        int64_t k_begin, int64_t k_end);

#define RMS_EXTERN_LAUNCH_WALK(REAL, IM, MT)                                                               \
    extern template cudaError_t launch_walk<REAL, IM, MT>(int, bool, dim3, cudaStream_t, const Geometry &, \
                                                          const Tables<REAL> &, const WalkerState<REAL> &, \
                                                          const RunCtl &, int64_t, int64_t);
RMS_EXTERN_LAUNCH_WALK(double, kInteractEC, false)
RMS_EXTERN_LAUNCH_WALK(double, kInteractRS, false)
RMS_EXTERN_LAUNCH_WALK(double, kInteractERL, false)
RMS_EXTERN_LAUNCH_WALK(float, kInteractEC, false)
RMS_EXTERN_LAUNCH_WALK(float, kInteractRS, false)
RMS_EXTERN_LAUNCH_WALK(float, kInteractERL, false)
RMS_EXTERN_LAUNCH_WALK(double, kInteractEC, true)
RMS_EXTERN_LAUNCH_WALK(double, kInteractRS, true)
RMS_EXTERN_LAUNCH_WALK(double, kInteractERL, true)
RMS_EXTERN_LAUNCH_WALK(float, kInteractEC, true)
RMS_EXTERN_LAUNCH_WALK(float, kInteractRS, true)
RMS_EXTERN_LAUNCH_WALK(float, kInteractERL, true)
#undef RMS_EXTERN_LAUNCH_WALK

template <typename Real>
cudaError_t launch_walk_batched(int ns_bucket, int32_t n_tasks, cudaStream_t stream, const ReqDesc<Real> *reqs,
                                const BlockTask *tasks);
extern template cudaError_t launch_walk_batched<double>(int, int32_t, cudaStream_t, const ReqDesc<double> *,
                                                        const BlockTask *);
extern template cudaError_t launch_walk_batched<float>(int, int32_t, cudaStream_t, const ReqDesc<float> *,
                                                       const BlockTask *);

template <typename Real>
int batched_blocks_per_sm(int ns_bucket);
extern template int batched_blocks_per_sm<double>(int);
extern template int batched_blocks_per_sm<float>(int);

int walk_block_size();

// Message returned by rms_last_error() on the calling thread.
void set_last_error(const char *msg);

}  // namespace rms
