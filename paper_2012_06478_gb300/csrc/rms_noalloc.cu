// rms_noalloc.cu -- a signal read-out that allocates no device memory.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree (or any
// allocating library routine) at the point where they want the signal.
// Typical cases are a serving loop that shares the GPU with other streams
// (cudaMalloc and cudaFree can synchronise the whole device and stall them),
// and a host application whose device memory is owned by its own fixed-size
// pool or arena and that may not take memory outside it.  Such a caller keeps
// its walker data in its own buffers and gets S(b, g) without the library
// asking the driver for memory.
//
// How: the per-chunk partial sums live in one file-scope __device__ array of
// fixed size (RMS_NOALLOC_SCRATCH_BYTES).  The CUDA runtime loads the
// library's device code on a device lazily, at its first use there, and the
// array's memory is taken then and held until the process exits.  Host code
// cannot use the array's name as a device address, so the first call on each
// device looks up the address with cudaGetSymbolAddress (with that device
// current) and caches it with the identity of the device's current context;
// that first call should therefore happen before any stream capture.  A new
// context on the device (after cudaDeviceReset, say) has a new copy of the
// array at a new address: the next call sees the changed context identity
// and looks the address up again.
// Every call shares the array and it keeps the last call's contents: each
// call writes every partial it later reads, so nothing needs clearing, but
// calls that overlap on the GPU (different streams, or different host
// threads on the same device) race on it and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/rms.h"
#include "rms_internal.h"

namespace {

constexpr int64_t kScratchDoubles = RMS_NOALLOC_SCRATCH_BYTES / 8;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_ptr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};  // context identity the address belongs to

// The driver's identity of the calling thread's current context (0 if it
// cannot be had), through the runtime's driver entry points so that the
// library needs no link to the driver library.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)f;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

constexpr int kBlock = 128;
constexpr int kTile = 64;
constexpr int kMaxShapes = 8;

rms_status fail(rms_status st, const char *msg)
{
    rms::set_last_error(msg);
    return st;
}

// Partial sums of alpha cos(phi) and -alpha sin(phi) (Eq. 7), phi = q g.Phi_s,
// q = sqrt(b / b_s), alpha = exp(-A), over walkers [chunk*per, (chunk+1)*per)
// for every (shape, direction, b) combination; the extra combination n_combo
// holds the sum of alpha.  phase is (W, S, 3) row-major, A is (W).
__global__ void __launch_bounds__(kBlock)
noalloc_partial_kernel(const double *phase, const double *A, int64_t W, int32_t S, const double *b_s,
                       const double *dirs, int32_t n_dirs, const double *b, int32_t n_b, int32_t n_combo,
                       int64_t per, double *part)
{
    __shared__ double sP[kTile][kMaxShapes * 3];
    __shared__ double sAl[kTile];
    const int combo = blockIdx.x * kBlock + threadIdx.x;
    int s = 0;
    double q = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (combo < n_combo) {
        const int ib = combo % n_b;
        const int gi = (combo / n_b) % n_dirs;
        s = combo / (n_b * n_dirs);
        q = b_s[s] > 0.0 ? sqrt(b[ib] / b_s[s]) : 0.0;
        g0 = dirs[3 * gi];
        g1 = dirs[3 * gi + 1];
        g2 = dirs[3 * gi + 2];
    }
    const int64_t w0 = (int64_t)blockIdx.y * per;
    const int64_t w1 = min(W, w0 + per);
    double re = 0.0, im = 0.0;
    for (int64_t base = w0; base < w1; base += kTile) {
        const int nt = (int)min((int64_t)kTile, w1 - base);
        for (int e = threadIdx.x; e < nt * (S * 3 + 1); e += kBlock) {
            const int j = e / (S * 3 + 1), k = e % (S * 3 + 1);
            if (k < S * 3)
                sP[j][k] = phase[(base + j) * S * 3 + k];
            else
                sAl[j] = exp(-A[base + j]);
        }
        __syncthreads();
        if (combo < n_combo) {
            for (int j = 0; j < nt; ++j) {
                const double phi = q * (g0 * sP[j][3 * s] + g1 * sP[j][3 * s + 1] + g2 * sP[j][3 * s + 2]);
                double sn, cs;
                sincos(phi, &sn, &cs);
                re += sAl[j] * cs;
                im += -(sAl[j] * sn);
            }
        } else if (combo == n_combo) {
            for (int j = 0; j < nt; ++j) re += sAl[j];
        }
        __syncthreads();
    }
    if (combo <= n_combo) {
        part[((int64_t)blockIdx.y * (n_combo + 1) + combo) * 2 + 0] = re;
        part[((int64_t)blockIdx.y * (n_combo + 1) + combo) * 2 + 1] = im;
    }
}

__device__ __forceinline__ void neumaier(double &sum, double &comp, double x)
{
    const double t = sum + x;
    if (fabs(sum) >= fabs(x))
        comp += (sum - t) + x;
    else
        comp += (x - t) + sum;
    sum = t;
}

// Fixed-order sums over chunks; every thread also sums the alpha column in
// the same order, so all of them divide by the same total.
__global__ void noalloc_reduce_kernel(const double *part, int64_t n_chunks, int32_t n_combo, double *S_re,
                                      double *S_im, double *alpha_sum)
{
    const int combo = blockIdx.x * blockDim.x + threadIdx.x;
    if (combo >= n_combo) return;
    double as = 0, ac = 0, rs = 0, rc = 0, is = 0, ic = 0;
    for (int64_t k = 0; k < n_chunks; ++k) {
        neumaier(as, ac, part[(k * (n_combo + 1) + n_combo) * 2]);
        neumaier(rs, rc, part[(k * (n_combo + 1) + combo) * 2 + 0]);
        neumaier(is, ic, part[(k * (n_combo + 1) + combo) * 2 + 1]);
    }
    const double a = as + ac;
    S_re[combo] = (rs + rc) / a;
    S_im[combo] = (is + ic) / a;
    if (combo == 0 && alpha_sum) *alpha_sum = a;
}

// The scratch array's device address on the current device: looked up once
// per device and context (the first call, and again after the device's
// context has changed; a context whose identity cannot be read is looked up
// every time).
rms_status scratch_ptr(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(RMS_E_INVALID_ARG, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long ctx = current_context_id();
    if (!g_ptr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return fail(RMS_E_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "no address");
        if (ctx == 0) ctx = current_context_id();  // the lookup may have made the context current
        g_ptr[dev] = (double *)p;
        g_ctx[dev] = ctx;
    }
    *out = g_ptr[dev];
    return RMS_OK;
}

}  // namespace

extern "C" rms_status rms_readout_noalloc(const double *phase, const double *A, int64_t n_walkers, int32_t n_shapes,
                                          const double *b_s, int32_t n_dirs, const double *dirs, int32_t n_b,
                                          const double *b, double *S_re, double *S_im, double *alpha_sum,
                                          void *stream)
{
    if (!phase || !A || !b_s || !dirs || !b || !S_re || !S_im)
        return fail(RMS_E_INVALID_ARG, "rms_readout_noalloc: null pointer");
    if (n_walkers < 1 || n_shapes < 1 || n_shapes > kMaxShapes || n_dirs < 1 || n_b < 1)
        return fail(RMS_E_INVALID_ARG, "rms_readout_noalloc: n_walkers, n_dirs, n_b >= 1 and n_shapes in 1..8");
    const int64_t n_combo = (int64_t)n_shapes * n_dirs * n_b;
    const int64_t per_chunk = 2 * (n_combo + 1);  // doubles one walker chunk needs
    if (n_combo > (1 << 30) || per_chunk > kScratchDoubles)
        return fail(RMS_E_INVALID_ARG,
                    "rms_readout_noalloc: n_shapes*n_dirs*n_b too large for the fixed scratch "
                    "(needs 2*(n_shapes*n_dirs*n_b + 1) <= RMS_NOALLOC_SCRATCH_BYTES/8)");
    double *scratch = nullptr;
    rms_status st = scratch_ptr(&scratch);
    if (st != RMS_OK) return st;
    // as many walker chunks as fit (at most one per 4096 walkers)
    int64_t n_chunks = (n_walkers + 4095) / 4096;
    const int64_t cap = kScratchDoubles / per_chunk;
    if (n_chunks > cap) n_chunks = cap;
    if (n_chunks > 65535) n_chunks = 65535;
    const int64_t per = (n_walkers + n_chunks - 1) / n_chunks;
    n_chunks = (n_walkers + per - 1) / per;
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid((unsigned)((n_combo + 1 + kBlock - 1) / kBlock), (unsigned)n_chunks);
    noalloc_partial_kernel<<<grid, kBlock, 0, s>>>(phase, A, n_walkers, n_shapes, b_s, dirs, n_dirs, b, n_b,
                                                   (int32_t)n_combo, per, scratch);
    noalloc_reduce_kernel<<<(unsigned)((n_combo + 127) / 128), 128, 0, s>>>(scratch, n_chunks, (int32_t)n_combo,
                                                                             S_re, S_im, alpha_sum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RMS_E_CUDA, cudaGetErrorString(e));
    return RMS_OK;
}
