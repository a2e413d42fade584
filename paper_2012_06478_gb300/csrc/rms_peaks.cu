// rms_peaks.cu -- microbenchmarks for the rooflines of the walker step
// (include/rms_peaks.h): the random 2-byte gather rate of a uint16 volume
// (the label lookup of Sec. 2.1.1) and the FP64 add / multiply rate (the
// pipe that bounds the plain FP64 form).  Built with -fmad=false like the
// plain form, so an add is an add and a multiply a multiply.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/rms_peaks.h"
#include "rms_internal.h"

namespace {

constexpr int kBlock = 256;
constexpr int kBlocksPerSM = 8;  // 2048 threads: a full SM
constexpr int kChains = 8;       // independent operations in flight per thread

rms_status fail(rms_status st, const std::string &msg)
{
    rms::set_last_error(msg.c_str());
    return st;
}

// Independent FP64 chains.  OP 0: x += b, 1: x *= b, 2: x = x*b + c.  The
// sum is stored only when it equals an impossible value, so that nothing is
// dead code and nothing is written.
template <int OP>
__global__ void __launch_bounds__(kBlock) fp64_peak_kernel(double b, double c, int64_t iters, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0 + 1e-3 * (double)(threadIdx.x + 7 * i);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (OP == 0)
                x[i] = __dadd_rn(x[i], b);
            else if (OP == 1)
                x[i] = __dmul_rn(x[i], b);
            else
                x[i] = __fma_rn(x[i], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s = __dadd_rn(s, x[i]);
    if (s == -1.0) sink[0] = s;
}

// Random uint16 gathers through the read-only path.  Each thread keeps ILP
// linear congruential streams (multiplier 1664525, increment 1013904223 --
// Knuth / Numerical Recipes); the top log2(volume) bits of a state are the
// element index.  DEP: one stream whose next state also adds the label just
// read, so each address waits for the previous load (one gather in flight
// per thread, as along a walker's face events).
template <int ILP, bool DEP>
__global__ void __launch_bounds__(kBlock) gather_peak_kernel(const uint16_t *__restrict__ vol, uint32_t shift,
                                                             int64_t iters, uint32_t *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) x[i] = (tid * ILP + i) * 2654435761u + 12345u;
    uint32_t acc = 0, lab = 0;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < ILP; ++i) {
            if (DEP) {
                x[i] = (x[i] + lab) * 1664525u + 1013904223u;
                lab = __ldg(vol + (x[i] >> shift));
                acc += lab;
            } else {
                x[i] = x[i] * 1664525u + 1013904223u;
                acc += __ldg(vol + (x[i] >> shift));
            }
        }
    }
    if (acc == 0xFFFFFFFFu) sink[0] = acc;
}

__global__ void fill_kernel(uint16_t *vol, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        vol[i] = (uint16_t)(((uint64_t)i * 0x9E3779B97F4A7C15ULL) >> 54);  // pseudo-random labels < 1024
}

struct Buffers {
    void *vol = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Buffers()
    {
        if (vol) cudaFree(vol);
        if (sink) cudaFree(sink);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

}  // namespace

extern "C" rms_status rms_device_sm_count(int32_t *sm_count)
{
    if (!sm_count) return fail(RMS_E_INVALID_ARG, "null pointer");
    int dev = 0, n = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
    *sm_count = n;
    return RMS_OK;
}

extern "C" rms_status rms_measure_peak(int32_t kind, int64_t volume_elems, double target_ms, int32_t reps,
                                       void *stream, double *rate, double *ms)
{
    if (kind < RMS_PEAK_FP64_ADD || kind > RMS_PEAK_GATHER_DEP) return fail(RMS_E_INVALID_ARG, "unknown peak kind");
    if (!(target_ms > 0.0) || target_ms > 10000.0 || reps < 1 || reps > 1000)
        return fail(RMS_E_INVALID_ARG, "target_ms in (0, 1e4] and reps in 1..1000");
    const bool gather = kind >= RMS_PEAK_GATHER;
    int log2v = 0;
    if (gather) {
        if (volume_elems < (1 << 10) || volume_elems > (1LL << 31) || (volume_elems & (volume_elems - 1)))
            return fail(RMS_E_INVALID_ARG, "volume_elems must be a power of two in [2^10, 2^31]");
        while ((1LL << log2v) < volume_elems) ++log2v;
    }
    int32_t sms = 0;
    rms_status st = rms_device_sm_count(&sms);
    if (st != RMS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Buffers buf;
    cudaError_t e = cudaMalloc(&buf.sink, 64);
    if (e == cudaSuccess && gather) e = cudaMalloc(&buf.vol, (size_t)volume_elems * sizeof(uint16_t));
    if (e == cudaErrorMemoryAllocation) return fail(RMS_E_OOM, "rms_measure_peak: device allocation failed");
    if (e == cudaSuccess) e = cudaEventCreate(&buf.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&buf.e1);
    if (e != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
    if (gather) {
        fill_kernel<<<sms * 4, kBlock, 0, s>>>((uint16_t *)buf.vol, volume_elems);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
    }
    const dim3 grid((unsigned)(sms * kBlocksPerSM));
    const int ilp = kind == RMS_PEAK_GATHER_DEP ? 1 : kChains;
    const double ops_per_iter = (double)grid.x * kBlock * (gather ? ilp : kChains);
    const uint32_t shift = (uint32_t)(32 - log2v);
    auto launch = [&](int64_t iters) {
        switch (kind) {
        case RMS_PEAK_FP64_ADD:
            fp64_peak_kernel<0><<<grid, kBlock, 0, s>>>(1e-9, 0.0, iters, (double *)buf.sink);
            break;
        case RMS_PEAK_FP64_MUL:
            fp64_peak_kernel<1><<<grid, kBlock, 0, s>>>(0.99999999999, 0.0, iters, (double *)buf.sink);
            break;
        case RMS_PEAK_FP64_FMA:
            fp64_peak_kernel<2><<<grid, kBlock, 0, s>>>(0.5, 0.5, iters, (double *)buf.sink);
            break;
        case RMS_PEAK_GATHER:
            gather_peak_kernel<kChains, false><<<grid, kBlock, 0, s>>>((const uint16_t *)buf.vol, shift, iters,
                                                                      (uint32_t *)buf.sink);
            break;
        default:
            gather_peak_kernel<1, true><<<grid, kBlock, 0, s>>>((const uint16_t *)buf.vol, shift, iters,
                                                               (uint32_t *)buf.sink);
            break;
        }
    };
    auto timed = [&](int64_t iters, float *out_ms) -> cudaError_t {
        cudaError_t err = cudaEventRecord(buf.e0, s);
        if (err != cudaSuccess) return err;
        launch(iters);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = cudaEventRecord(buf.e1, s)) != cudaSuccess) return err;
        if ((err = cudaEventSynchronize(buf.e1)) != cudaSuccess) return err;
        return cudaEventElapsedTime(out_ms, buf.e0, buf.e1);
    };
    // calibrate: a short launch (also the warm-up that brings the volume
    // into L2 when it fits), then scale the iteration count to target_ms
    float t = 0.0f;
    int64_t iters = 64;
    if ((e = timed(iters, &t)) != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
    if ((e = timed(iters, &t)) != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
    iters = std::max<int64_t>(16, std::min<int64_t>((int64_t)1 << 30, (int64_t)(iters * target_ms / std::max(t, 1e-3f))));
    if ((e = timed(iters, &t)) != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));  // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        if ((e = timed(iters, &t)) != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
        best = std::min(best, t);
    }
    if (rate) *rate = ops_per_iter * (double)iters / (best * 1e-3);
    if (ms) *ms = best;
    return RMS_OK;
}
