// rms_handles.h -- the library's handle types and the stages of a run,
// shared by the C ABI (rms_api.cu) and the serving loop (rms_serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rms.h"
#include "rms_device.cuh"

// A host-side NVTX range for the lifetime of the object (header-only NVTX
// v3: no link dependency, and a no-op unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct rms_substrate {
    int device = 0;
    int32_t nx = 0, ny = 0, nz = 0;
    double voxel_um = 0;
    int32_t periodic[3] = {1, 1, 1};
    int32_t L = 0;
    std::vector<double> D, T2, T1, kappa;
    std::vector<double> rho;  // surface relaxivity per pair (empty: no absorbing membrane)
    std::vector<double> conc; // spin concentration per label (empty: all equal)
    double lambda = -1.0;     // exponent of (c2/c1) in the generalised Eq. 3 (< 0: optimal)
    int32_t perm_model = RMS_PERM_KAPPA;
    uint64_t *d_acc = nullptr;  // per label start acceptance threshold (nullptr: always)
    std::vector<uint8_t> dead;
    uint16_t *d_labels = nullptr;
    double *d_D = nullptr, *d_T2 = nullptr, *d_T1 = nullptr, *d_kappa = nullptr, *d_rho = nullptr;
    uint8_t *d_dead = nullptr;
    int32_t *d_ok = nullptr;  // raster list of non-dead voxels (nullptr: none dead)
    int64_t n_ok = 0;
    std::atomic<int> refs{0};
};

struct rms_sequence {
    rms_substrate *sub = nullptr;
    double dt = 0;
    int64_t n_steps = 0;
    int32_t S = 0, n_dirs = 0, n_b = 0, n_rec = 0;
    int32_t any_relax = 0;
    int32_t has_mode = 0;
    std::vector<int64_t> rec_steps;  // host copy of the recording steps
    double *d_s64 = nullptr, *d_dtR64 = nullptr, *d_wG64 = nullptr;
    float *d_s32 = nullptr, *d_dtR32 = nullptr, *d_wG32 = nullptr;
    uint32_t *d_T = nullptr;
    uint32_t *d_Tmt = nullptr;  // saturation thresholds (nullptr: no absorbing membrane)
    uint8_t *d_flags = nullptr, *d_mode = nullptr;
    int32_t *d_rec_of = nullptr;
    double *d_dirs = nullptr, *d_b = nullptr, *d_bs = nullptr, *d_q = nullptr;
    double *d_trig = nullptr;  // azimuth table (FP64 form)
    std::atomic<int> refs{0};
};

struct rms_run_handle {
    rms_sequence *seq = nullptr;
    int64_t W = 0, w_begin = 0;
    uint64_t seed = 0;
    int32_t precision = RMS_FP64;
    uint32_t flags = 0;
    int32_t interaction = RMS_EC;
    cudaStream_t stream = nullptr;
    int32_t n_blocks = 0;
    char *d_state = nullptr;  // one allocation for the walker state
    rms::WalkerState<double> st64{};
    rms::WalkerState<float> st32{};
    // RMS_MORTON: the second state buffer the re-bucketing gathers into, and
    // the sort buffers (keys, slots, tile histograms, scan block sums)
    char *d_state_alt = nullptr;
    rms::WalkerState<double> st64_alt{};
    rms::WalkerState<float> st32_alt{};
    char *d_sort = nullptr;
    int32_t sort_shift = 0, sort_passes = 0;
    double *d_mom_partial = nullptr, *d_mom = nullptr;
    double *d_mom_chunk = nullptr;  // first-level moment sums [rec][chunk of 256 blocks][22]
    // d_S: the unnormalised sums [combo][2] + (alpha sum, 0), then the
    // normalised signal in the same layout (normalised_S)
    double *d_ro_partial = nullptr, *d_S = nullptr;
    int32_t *d_status = nullptr;
    int32_t *h_cancel = nullptr, *d_cancel = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    int32_t n_combo = 0, n_chunks = 0;
};

namespace rms {

constexpr int kWalkBlockSize = 128;  // walkers per block of the walk kernels

rms_status fail(rms_status st, const std::string &msg);

#define RMS_CUDA(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return ::rms::fail(e_ == cudaErrorMemoryAllocation ? RMS_E_OOM : RMS_E_CUDA,          \
                               std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

#define RMS_TRY(expr)            \
    do {                         \
        rms_status st_ = (expr); \
        if (st_ < 0) return st_; \
    } while (0)

// The normalised signal [combo][2] + (alpha sum, 0) of a finalised run.
inline double *normalised_S(const rms_run_handle *r) { return r->d_S + 2 * (size_t)(r->n_combo + 1); }

template <typename Real>
size_t layout_state(WalkerState<Real> &st, char *base, int64_t W, int S, bool hash, bool f32, bool counts,
                    bool wid = false);

// Run flags that select the verification kernel (checksum, invariant checks, counts).
constexpr uint32_t kVerifyFlags = RMS_TRAJ_HASH | RMS_CHECKED | RMS_COUNTS;

// Stages of a run, each enqueued on r->stream.
rms_status run_setup(rms_run_handle *r, bool with_cancel_and_events);  // allocate, lay out
rms_status run_init(rms_run_handle *r);                               // Sec. 2.2 item 1
rms_status run_walk(rms_run_handle *r, int64_t k0, int64_t k1);       // steps (k0, k1]
rms_status run_finalize(rms_run_handle *r);                           // moments, read-out
void run_free(rms_run_handle *r, bool sync);
size_t run_state_bytes(const rms_sequence *q, int64_t W, int32_t precision, uint32_t flags);
// RMS_MORTON (rms_morton.cu): the key's coordinate shift and radix passes for
// a volume, the sort buffers' bytes, and the re-bucketing enqueued on r->stream.
void morton_plan(int32_t nx, int32_t ny, int32_t nz, int32_t *shift, int32_t *passes);
size_t morton_scratch_bytes(int64_t W);
rms_status run_rebucket(rms_run_handle *r);
template <typename Real>
ReqDesc<Real> run_desc(rms_run_handle *r);

}  // namespace rms
