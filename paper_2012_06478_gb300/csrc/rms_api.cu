// rms_api.cu -- the C ABI (include/rms.h): substrate, sequence and run
// handles, the set-up kernels that build the per-label and per-pair tables,
// walker initialisation, the moment and signal reductions and the read-out.
//
// Built with -fmad=false: the tables (step lengths, relaxation rates,
// permeation thresholds, waveform weights) and the read-out are evaluated
// with the same separately rounded FP64 operations as the CPU reference.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rms.h"
#include "rms_device.cuh"
#include "rms_handles.h"
#include "rms_internal.h"

using namespace rms;

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

rms_status rms::fail(rms_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}


void rms::set_last_error(const char *msg) { g_last_error = msg; }

extern "C" int rms_version(void) { return 10000; }
extern "C" const char *rms_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------ handles

// ------------------------------------------------------------------ set-up kernels

__global__ void max_label_kernel(const uint16_t *lab, int64_t n, uint32_t *out)
{
    uint32_t m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (uint32_t)lab[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Raster list of the voxels whose label is not dead (Sec. 2.2 item 1):
// per-block counts, one scan, then an ordered fill.
constexpr int kOkBlock = 1024;

__global__ void ok_count_kernel(const uint16_t *lab, int64_t n, const uint8_t *dead, int32_t *cnt)
{
    __shared__ int32_t s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kOkBlock + threadIdx.x;
    const int ok = i < n && !dead[lab[i]];
    const int wc = __popc(__ballot_sync(0xffffffffu, ok));
    if ((threadIdx.x & 31) == 0 && wc) atomicAdd(&s, wc);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = s;
}

__global__ void exclusive_scan_kernel(int32_t *cnt, int64_t n, int64_t *total)
{
    // single block; serial over chunks of blockDim.x, each chunk scanned in shared memory
    __shared__ int64_t buf[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t x = i < n ? cnt[i] : 0;
        buf[threadIdx.x] = x;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            const int64_t y = threadIdx.x >= (unsigned)off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < n) cnt[i] = (int32_t)(carry + buf[threadIdx.x] - x);
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void ok_fill_kernel(const uint16_t *lab, int64_t n, const uint8_t *dead, const int32_t *start,
                               int32_t *list)
{
    __shared__ int32_t warp_base[kOkBlock / 32];
    const int64_t i = (int64_t)blockIdx.x * kOkBlock + threadIdx.x;
    const int ok = i < n && !dead[lab[i]];
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_base[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int k = 0; k < kOkBlock / 32; ++k) {
            const int32_t c = warp_base[k];
            warp_base[k] = acc;
            acc += c;
        }
    }
    __syncthreads();
    if (ok) list[start[blockIdx.x] + warp_base[wid] + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
}

// Eq. 1 (d = 3): ds = sqrt((6 D) dt); s = ds / l_p.  Eq. 5: dt / T per label.
__global__ void label_tables_kernel(int32_t L, const double *D, const double *T2, const double *T1, double dt,
                                    double voxel, double *s64, float *s32, double *dtR64, float *dtR32)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L) return;
    const double ds = sqrt((6.0 * D[c]) * dt);
    const double s = ds / voxel;
    s64[c] = s;
    s32[c] = (float)s;
    const double r2 = isinf(T2[c]) ? 0.0 : dt / T2[c];
    const double r1 = isinf(T1[c]) ? 0.0 : dt / T1[c];
    dtR64[c] = r2;
    dtR64[L + c] = r1;
    dtR64[2 * L + c] = 0.0;
    dtR32[c] = (float)r2;
    dtR32[L + c] = (float)r1;
    dtR32[2 * L + c] = 0.0f;
}

// Eq. 3: P_{1->2} = (kappa ds1 C / D1) / (1 + (kappa/2)(ds1/D1 + ds2/D2) C),
// C = C_3 = 2/3 (Eq. 2b), evaluated as ((kappa ds1)/D1) C over
// 1 + ((kappa/2)((ds1/D1) + (ds2/D2))) C.  The walker crosses when a uniform
// 32-bit word is below T = min(floor(P 2^32), 2^32 - 1).
__global__ void pair_tables_kernel(int32_t L, const double *D, const double *kappa, const uint8_t *dead,
                                   double dt, uint32_t *T, int32_t *warn)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * L) return;
    const int a = (int)(idx / L), b = (int)(idx % L);
    const double k = kappa[idx];
    uint32_t thr = 0u;
    if (a != b && !dead[a] && !dead[b] && k > 0.0) {
        const double C = 2.0 / 3.0;
        const double ds1 = sqrt((6.0 * D[a]) * dt);
        const double ds2 = sqrt((6.0 * D[b]) * dt);
        const double num = ((k * ds1) / D[a]) * C;
        const double den = 1.0 + ((k / 2.0) * ((ds1 / D[a]) + (ds2 / D[b]))) * C;
        const double P = num / den;
        if (P > 1.0) atomicOr(warn, 1);
        if (P >= 1.0) {
            thr = 0xFFFFFFFFu;
        } else if (P > 0.0) {
            const double x = floor(P * 4294967296.0);
            thr = x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
        }
    }
    T[idx] = thr;
}

// Sec. 2.1.3 (magnetization transfer): saturation thresholds
// T_mt = floor(P_MT 2^32) for a walker of label a meeting an absorbing
// membrane towards label b, P_MT = (rho ds_a / D_a) C_3.  A membrane into a
// dead label counts; none inside a label.
__global__ void mt_tables_kernel(int32_t L, const double *D, const double *rho, const uint8_t *dead, double dt,
                                 uint32_t *Tmt, int32_t *warn)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * L) return;
    const int a = (int)(idx / L), b = (int)(idx % L);
    const double r = rho[idx];
    uint32_t thr = 0u;
    if (a != b && !dead[a] && r > 0.0) {
        const double C = 2.0 / 3.0;
        const double ds1 = sqrt((6.0 * D[a]) * dt);
        const double P = ((r * ds1) / D[a]) * C;
        if (P > 1.0) atomicOr(warn, 1);
        if (P >= 1.0) {
            thr = 0xFFFFFFFFu;
        } else if (P > 0.0) {
            const double x = floor(P * 4294967296.0);
            thr = x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
        }
    }
    Tmt[idx] = thr;
}

// The azimuth table: (cos, sin) of the centres (2j + 1) 2^-11 pi/4 of the
// 1024 parts of [0, pi/4].
__global__ void trig_table_kernel(double *trig)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kTrigParts) return;
    const double th = ((double)(2 * j + 1) * 0x1p-11) * 0.78539816339744830962;
    double sn, cs;
    poly_sincos(th, sn, cs);
    trig[2 * j] = cs;
    trig[2 * j + 1] = sn;
}

// Per step: weights dt G_{s,k}, the step flags and the recording index.
__global__ void step_tables_kernel(int64_t N, int32_t S, double dt, const double *G, const int64_t *rec,
                                   int32_t n_rec, double *wG64, float *wG32, uint8_t *flags, int32_t *rec_of)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // 0-based step index
    if (k >= N) return;
    uint8_t f = 0;
    for (int s = 0; s < S; ++s) {
        const double w = dt * G[(int64_t)s * N + k];
        wG64[(int64_t)s * N + k] = w;
        wG32[(int64_t)s * N + k] = (float)w;
        if (w != 0.0) f |= 1u;
    }
    // binary search of step k+1 among the recording steps
    int lo = 0, hi = n_rec;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (rec[mid] < k + 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    int32_t r = -1;
    if (lo < n_rec && rec[lo] == k + 1) {
        r = lo;
        f |= 2u;
    }
    flags[k] = f;
    rec_of[k] = r;
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

// b of a unit waveform: b_s = dt sum_{j=1..N} F_{j-1}^2, F_j = F_{j-1} + dt G_j
// (compensated sum); then q = sqrt(b / b_s), the amplitude giving b.  One
// block per shape: the block stages the waveform through shared memory in
// coalesced chunks and thread 0 takes the recurrence in step order -- the
// CPU reference's operations in its order, so b_s is the same to the bit.
// (Read straight from global memory, each step waited for its load: 34 ms
// for N = 1e5, most of a sequence's set-up.)
constexpr int kBvThreads = 256;
constexpr int kBvChunk = 2048;

__global__ void __launch_bounds__(kBvThreads) bvalue_kernel(int64_t N, int32_t S, double dt, const double *G,
                                                            int32_t n_b, const double *b, double *bs_out, double *q)
{
    const int s = blockIdx.x;
    if (s >= S) return;  // block-uniform
    __shared__ double sg[kBvChunk];
    const double *g = G + (int64_t)s * N;
    double F = 0.0, sum = 0.0, comp = 0.0;  // thread 0's
    for (int64_t base = 0; base < N; base += kBvChunk) {
        const int n = (int)min((int64_t)kBvChunk, N - base);
        for (int i = threadIdx.x; i < n; i += kBvThreads) sg[i] = g[base + i];
        __syncthreads();
        if (threadIdx.x == 0)
            for (int i = 0; i < n; ++i) {
                neumaier(sum, comp, F * F);
                F = F + dt * sg[i];
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double bs = dt * (sum + comp);
        bs_out[s] = bs;
        for (int i = 0; i < n_b; ++i) q[s * n_b + i] = bs > 0.0 ? sqrt(b[i] / bs) : 0.0;
    }
}

// ------------------------------------------------------------------ init (Sec. 2.2 item 1)

template <typename Real>
__global__ void init_kernel(Geometry g, const int32_t *ok_list, int64_t n_ok, const uint64_t *acc,
                            WalkerState<Real> st, RunCtl ctl, bool hash)
{
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= ctl.n_walkers) return;
    const uint64_t w = (uint64_t)(ctl.w_begin + li);
    // attempt j: INIT calls 2j, 2j + 1; with spin concentrations the start in
    // label l is kept iff word 1 of call 2j + 1 is below acc[l] (density ~ c)
    U4 x, y;
    int64_t vox = 0;
    bool ok = false;
    for (uint32_t j = 0; j < kMaxInit && !ok; ++j) {
        x = draw(ctl.seed, w, 0u, kTagInit, 2u * j);
        y = draw(ctl.seed, w, 0u, kTagInit, 2u * j + 1u);
        const uint64_t r = ((uint64_t)x.x << 32) | (uint64_t)x.y;
        const int64_t idx = (int64_t)__umul64hi(r, (uint64_t)n_ok);
        vox = ok_list ? (int64_t)ok_list[idx] : idx;
        ok = acc == nullptr || (uint64_t)y.y < acc[g.labels[vox]];
    }
    if (!ok) atomicOr(ctl.status, kErrInit);
    const int32_t ix = (int32_t)(vox % g.nx);
    const int32_t iy = (int32_t)((vox / g.nx) % g.ny);
    const int32_t iz = (int32_t)(vox / ((int64_t)g.nx * g.ny));
    const double o[3] = {u01(x.z), u01(x.w), u01(y.x)};
    const int32_t i0[3] = {ix, iy, iz};
    for (int a = 0; a < 3; ++a) {
        st.o[a][li] = (Real)o[a];
        st.o0[a][li] = (Real)o[a];
        st.i0[a][li] = i0[a];
        st.di[a][li] = 0;
    }
    st.c[li] = g.labels[vox];
    st.A[li] = Real(0);
    if (st.A_c) st.A_c[li] = Real(0);
    for (int k = 0; k < ctl.n_shapes * 3; ++k) {
        st.phase[(int64_t)k * ctl.n_walkers + li] = Real(0);
        if (st.phase_c) st.phase_c[(int64_t)k * ctl.n_walkers + li] = Real(0);
    }
    if (hash) st.hash[li] = 0ull;
    if (st.counts)
        for (int a = 0; a < 3; ++a) st.counts[(int64_t)a * ctl.n_walkers + li] = 0;
    if (st.wid) st.wid[li] = (int32_t)li;
}

// ------------------------------------------------------------------ reductions

// Moments, first level: the per-block partials of recording step r, blocks
// c*kMomChunk ..., staged through shared memory with coalesced loads (the
// partials of one recording step are contiguous), each of the 22 sums taken
// in block order with compensation.  Block index = r * n_mchunks + c.
constexpr int kMomChunk = 256;

__global__ void __launch_bounds__(256) moments_chunk_kernel(const double *part, int32_t n_blocks, int32_t n_mchunks,
                                                            double *out)
{
    __shared__ double tile[kMomChunk * kMoments];
    const int64_t r = blockIdx.x / n_mchunks;
    const int32_t c = blockIdx.x % n_mchunks;
    const int32_t b0 = c * kMomChunk;
    const int32_t nb = min(kMomChunk, n_blocks - b0);
    const double *src = part + (r * n_blocks + b0) * kMoments;
    for (int e = threadIdx.x; e < nb * kMoments; e += blockDim.x) tile[e] = src[e];
    __syncthreads();
    if (threadIdx.x < kMoments) {
        double sum = 0.0, comp = 0.0;
        for (int b = 0; b < nb; ++b) neumaier(sum, comp, tile[b * kMoments + threadIdx.x]);
        out[(int64_t)blockIdx.x * kMoments + threadIdx.x] = sum + comp;
    }
}

// Moments, second level: fixed-order compensated sum of the n_blocks
// partials of each recording step (here the first level's chunk sums).
__global__ void moments_reduce_kernel(const double *part, int32_t n_rec, int32_t n_blocks, double *out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_rec * kMoments) return;
    const int r = idx / kMoments, m = idx % kMoments;
    double s = 0.0, c = 0.0;
    for (int b = 0; b < n_blocks; ++b) neumaier(s, c, part[((int64_t)r * n_blocks + b) * kMoments + m]);
    out[idx] = s + c;
}

// Read-out (Eq. 7): for every (shape, direction, b) combination the sums of
// alpha cos(phi) and -alpha sin(phi) over a chunk of walkers, phi = q (g . Phi_s),
// alpha = exp(-A).  One thread per combination; the walkers of the chunk are
// staged through shared memory in tiles.  The extra combination n_combo
// carries the sum of alpha.
constexpr int kRoBlock = 128;
constexpr int kRoTile = 64;
constexpr int64_t kRoChunk = 4096;

template <typename Real>
__global__ void __launch_bounds__(kRoBlock)
readout_kernel(const Real *phase, const Real *phase_c, const Real *A, const Real *A_c, int64_t W, int32_t S,
               const double *q, const double *dirs, int32_t n_dirs, int32_t n_b, int32_t n_combo,
               double *part)
{
    __shared__ double sP[kRoTile][kMaxShapes * 3];
    __shared__ double sAl[kRoTile];
    const int combo = blockIdx.y * kRoBlock + threadIdx.x;  // grid: x = walker chunk, y = combination group
    int s = 0;
    double qq = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (combo < n_combo) {
        const int ib = combo % n_b;
        const int gi = (combo / n_b) % n_dirs;
        s = combo / (n_b * n_dirs);
        qq = q[s * n_b + ib];
        g0 = dirs[3 * gi];
        g1 = dirs[3 * gi + 1];
        g2 = dirs[3 * gi + 2];
    }
    const int64_t w0 = (int64_t)blockIdx.x * kRoChunk;
    const int64_t w1 = min(W, w0 + kRoChunk);
    double re = 0.0, im = 0.0;
    for (int64_t base = w0; base < w1; base += kRoTile) {
        const int nt = (int)min((int64_t)kRoTile, w1 - base);
        for (int e = threadIdx.x; e < nt * (S * 3 + 1); e += kRoBlock) {
            const int j = e % nt, k = e / nt;
            const int64_t w = base + j;
            if (k < S * 3) {
                double p = (double)phase[(int64_t)k * W + w];
                if (phase_c) p = p - (double)phase_c[(int64_t)k * W + w];
                sP[j][k] = p;
            } else {
                double a = (double)A[w];
                if (A_c) a = a - (double)A_c[w];
                sAl[j] = exp(-a);
            }
        }
        __syncthreads();
        if (combo < n_combo) {
            for (int j = 0; j < nt; ++j) {
                const double phi = qq * (g0 * sP[j][3 * s] + g1 * sP[j][3 * s + 1] + g2 * sP[j][3 * s + 2]);
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
        part[((int64_t)blockIdx.x * (n_combo + 1) + combo) * 2 + 0] = re;
        part[((int64_t)blockIdx.x * (n_combo + 1) + combo) * 2 + 1] = im;
    }
}

// A float widened to double, exactly, on the integer ALU for normal values
// and zeros (the FP64 pipe is GB300's scarce one); subnormals, infinities and
// NaNs take the hardware conversion, out of line so that it is not evaluated
// speculatively beside the integer path.
static __device__ __noinline__ double f2d_hw(float x) { return (double)x; }
__device__ __forceinline__ double f2d(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu;
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    if (e == 0u) {
        if ((b & 0x7FFFFFu) == 0u) return __longlong_as_double((long long)sign);  // +-0
        return f2d_hw(x);
    }
    if (e == 0xFFu) return f2d_hw(x);
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29)));
}

// The FP32 form's read-out: the same sums over the same chunks in the same
// order, with each term alpha e^{-i phi} evaluated in single precision --
// the phase staged as the float nearest to its compensated value, phi =
// q (g . Phi_s) and sincosf in FP32, alpha rounded to float -- and summed in
// FP64 (the term widened exactly).  With P = q sum_i |g_i| |Phi_i| every term
// is within about (6 P + 4) 2^-24 alpha of its FP64 value, so S is within
// (6 P + 4) 2^-24 of the FP64 read-out of the same walkers (7.4e-6 at
// P = 20 rad), far inside the form's 1e-3 bar on S; the per-walker terms do
// not depend on the walkers' order or chunking.  b = 0 (q = 0) takes alpha
// in FP64, so S(b = 0) = 1 exactly, and the sum of alpha stays FP64.
__global__ void __launch_bounds__(kRoBlock)
readout_f32_kernel(const float *phase, const float *phase_c, const float *A, const float *A_c, int64_t W, int32_t S,
                   const double *q, const double *dirs, int32_t n_dirs, int32_t n_b, int32_t n_combo, double *part)
{
    __shared__ float sP[kRoTile][kMaxShapes * 3];
    __shared__ float sAl[kRoTile];
    __shared__ double sAlD[kRoTile];
    const int combo = blockIdx.y * kRoBlock + threadIdx.x;
    int s = 0;
    float qq = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    if (combo < n_combo) {
        const int ib = combo % n_b;
        const int gi = (combo / n_b) % n_dirs;
        s = combo / (n_b * n_dirs);
        qq = (float)q[s * n_b + ib];
        g0 = (float)dirs[3 * gi];
        g1 = (float)dirs[3 * gi + 1];
        g2 = (float)dirs[3 * gi + 2];
    }
    const int64_t w0 = (int64_t)blockIdx.x * kRoChunk;
    const int64_t w1 = min(W, w0 + kRoChunk);
    double re = 0.0, im = 0.0;
    for (int64_t base = w0; base < w1; base += kRoTile) {
        const int nt = (int)min((int64_t)kRoTile, w1 - base);
        for (int e = threadIdx.x; e < nt * (S * 3 + 1); e += kRoBlock) {
            const int j = e % nt, k = e / nt;
            const int64_t w = base + j;
            if (k < S * 3) {
                sP[j][k] = (float)((double)phase[(int64_t)k * W + w] - (double)phase_c[(int64_t)k * W + w]);
            } else {
                // kSaturatedF (saturated): exp underflows to 0
                const double al = exp(-((double)A[w] - (double)A_c[w]));
                sAlD[j] = al;
                sAl[j] = (float)al;
            }
        }
        __syncthreads();
        if (combo < n_combo && qq != 0.0f) {
            for (int j = 0; j < nt; ++j) {
                const float gp = fmaf(g2, sP[j][3 * s + 2], fmaf(g1, sP[j][3 * s + 1], g0 * sP[j][3 * s]));
                float sn, cs;
                sincosf(qq * gp, &sn, &cs);
                re += f2d(sAl[j] * cs);
                im += f2d(-(sAl[j] * sn));
            }
        } else if (combo <= n_combo) {  // b = 0, and the sum of alpha
            for (int j = 0; j < nt; ++j) re += sAlD[j];
        }
        __syncthreads();
    }
    if (combo <= n_combo) {
        part[((int64_t)blockIdx.x * (n_combo + 1) + combo) * 2 + 0] = re;
        part[((int64_t)blockIdx.x * (n_combo + 1) + combo) * 2 + 1] = im;
    }
}

__global__ void readout_reduce_kernel(const double *part, int32_t n_chunks, int32_t n_combo, double *out)
{
    const int combo = blockIdx.x * blockDim.x + threadIdx.x;
    if (combo > n_combo) return;
    double rs = 0, rc = 0, is = 0, ic = 0;
    for (int k = 0; k < n_chunks; ++k) {
        neumaier(rs, rc, part[((int64_t)k * (n_combo + 1) + combo) * 2 + 0]);
        neumaier(is, ic, part[((int64_t)k * (n_combo + 1) + combo) * 2 + 1]);
    }
    out[combo * 2 + 0] = rs + rc;
    out[combo * 2 + 1] = is + ic;
}

// S = sum alpha e^{-i phi} / sum alpha from the unnormalised sums, which stay
// as they are (rms_read_partials returns them for combining walker shards).
__global__ void normalise_kernel(const double *sums, int32_t n_combo, double *S)
{
    const int combo = blockIdx.x * blockDim.x + threadIdx.x;
    if (combo > n_combo) return;
    const double asum = sums[n_combo * 2];
    if (combo == n_combo) {
        S[combo * 2 + 0] = asum;
        S[combo * 2 + 1] = 0.0;
        return;
    }
    S[combo * 2 + 0] = sums[combo * 2 + 0] / asum;
    S[combo * 2 + 1] = sums[combo * 2 + 1] / asum;
}

// The counter-based generator, one thread per (counter, key) pair.
__global__ void philox_words_kernel(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U4 r = philox4x32_10(U4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}, key[2 * i],
                               key[2 * i + 1]);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

// Final per-walker state in array-of-structures form, FP64.
template <typename Real>
__global__ void export_kernel(WalkerState<Real> st, int64_t W, int32_t S, bool hash, int32_t *i, double *o,
                              int32_t *i0, double *o0, int32_t *c, double *A, double *phase, uint64_t *h)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // slot
    if (w >= W) return;
    const int64_t u = st.wid ? (int64_t)st.wid[w] : w;  // walker: the output row
    if (u < 0 || u >= W) return;  // never, for a valid order (the read calls check the status first)
    for (int a = 0; a < 3; ++a) {
        i[3 * u + a] = st.i0[a][w] + st.di[a][w];
        o[3 * u + a] = (double)st.o[a][w];
        i0[3 * u + a] = st.i0[a][w];
        o0[3 * u + a] = (double)st.o0[a][w];
    }
    c[u] = st.c[w];
    if (st.A_c)  // FP32 form: Kahan sum; kSaturatedF marks a saturated walker
        A[u] = (float)st.A[w] >= kSaturatedF ? (double)INFINITY : (double)st.A[w] - (double)st.A_c[w];
    else
        A[u] = (double)st.A[w];
    for (int k = 0; k < S * 3; ++k) {
        double p = (double)st.phase[(int64_t)k * W + w];
        if (st.phase_c) p = p - (double)st.phase_c[(int64_t)k * W + w];
        phase[u * S * 3 + k] = p;
    }
    h[u] = hash ? st.hash[w] : 0ull;
}

// ------------------------------------------------------------------ substrate

template <typename T>
static rms_status upload(T **dst, const T *src, size_t n, cudaStream_t s, bool src_on_device = false)
{
    RMS_CUDA(cudaMallocAsync((void **)dst, sizeof(T) * (n ? n : 1), s));
    if (n)
        RMS_CUDA(cudaMemcpyAsync(*dst, src, sizeof(T) * n,
                                 src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return RMS_OK;
}


static void free_substrate(rms_substrate *s, cudaStream_t st)
{
    cudaFreeAsync(s->d_labels, st);
    cudaFreeAsync(s->d_D, st);
    cudaFreeAsync(s->d_T2, st);
    cudaFreeAsync(s->d_T1, st);
    cudaFreeAsync(s->d_kappa, st);
    if (s->d_rho) cudaFreeAsync(s->d_rho, st);
    if (s->d_acc) cudaFreeAsync(s->d_acc, st);
    cudaFreeAsync(s->d_dead, st);
    if (s->d_ok) cudaFreeAsync(s->d_ok, st);
}

__global__ void label_hist_kernel(const uint16_t *labels, int64_t n, unsigned long long *count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(count + labels[i], 1ull);
}

// App. C.2: walkers start with density proportional to the spin
// concentration -- a uniform start in label l is kept iff a 32-bit word is
// below acc[l] = floor(c_l / c_max 2^32).  Rejects contrasts whose
// acceptance rate (the volume mean of c / c_max) is below 1/200, for which
// kMaxInit draws could run out.
static rms_status concentration_tables(rms_substrate *s, int64_t nvox, cudaStream_t st)
{
    const int L = s->L;
    unsigned long long *d_cnt = nullptr;
    RMS_CUDA(cudaMallocAsync((void **)&d_cnt, sizeof(unsigned long long) * L, st));
    RMS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * L, st));
    label_hist_kernel<<<1024, 256, 0, st>>>(s->d_labels, nvox, d_cnt);
    RMS_CUDA(cudaGetLastError());
    std::vector<unsigned long long> cnt(L);
    RMS_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(unsigned long long) * L, cudaMemcpyDeviceToHost, st));
    RMS_CUDA(cudaFreeAsync(d_cnt, st));
    RMS_CUDA(cudaStreamSynchronize(st));
    double cmax = 0.0, sum_cv = 0.0, sum_v = 0.0;
    for (int l = 0; l < L; ++l)
        if (!s->dead[l] && s->conc[l] > cmax) cmax = s->conc[l];
    std::vector<uint64_t> acc(L, 0);
    for (int l = 0; l < L; ++l) {
        if (s->dead[l]) continue;
        acc[l] = (uint64_t)std::floor((s->conc[l] / cmax) * 4294967296.0);
        sum_cv += s->conc[l] * (double)cnt[l];
        sum_v += (double)cnt[l];
    }
    if (sum_v > 0.0 && sum_cv / (cmax * sum_v) < 1.0 / 200.0)
        return fail(RMS_E_INVALID_ARG, "spin concentration contrast too large: volume mean of c / c_max < 1/200");
    RMS_TRY(upload(&s->d_acc, acc.data(), (size_t)L, st));
    return RMS_OK;
}

static rms_status create_substrate_impl(const rms_substrate_desc *d, rms_substrate *s)
{
    NvtxRange range("rms: substrate upload and tables");
    cudaStream_t st = (cudaStream_t)d->stream;
    const int64_t nvox = (int64_t)d->nx * d->ny * d->nz;
    const int L = d->n_labels;
    s->nx = d->nx;
    s->ny = d->ny;
    s->nz = d->nz;
    s->voxel_um = d->voxel_um;
    for (int a = 0; a < 3; ++a) s->periodic[a] = d->periodic[a] ? 1 : 0;
    s->L = L;
    s->D.assign(d->D, d->D + L);
    s->T2.assign(L, INFINITY);
    s->T1.assign(L, INFINITY);
    if (d->T2) s->T2.assign(d->T2, d->T2 + L);
    if (d->T1) s->T1.assign(d->T1, d->T1 + L);
    if (d->kappa)
        s->kappa.assign(d->kappa, d->kappa + (size_t)L * L);
    else
        s->kappa.assign((size_t)L * L, d->kappa_scalar);
    if (d->rho) s->rho.assign(d->rho, d->rho + (size_t)L * L);
    if (d->conc) s->conc.assign(d->conc, d->conc + L);
    s->lambda = d->lambda;
    s->perm_model = d->perm_model;
    if (s->perm_model != RMS_PERM_KAPPA && s->perm_model != RMS_PERM_BAXTER)
        return fail(RMS_E_INVALID_ARG, "perm_model must be RMS_PERM_KAPPA or RMS_PERM_BAXTER");
    if (!(s->lambda <= 1.0)) return fail(RMS_E_INVALID_ARG, "lambda must be <= 1 (< 0: the optimal lambda)");
    s->dead.assign(L, 0);
    if (d->dead)
        for (int c = 0; c < L; ++c) s->dead[c] = d->dead[c] ? 1 : 0;
    for (int c = 0; c < L; ++c) {
        if (!(s->D[c] > 0.0) || !std::isfinite(s->D[c]))
            return fail(RMS_E_INVALID_ARG, "D must be finite and > 0 for every label");
        if (!(s->T2[c] > 0.0) || !(s->T1[c] > 0.0))
            return fail(RMS_E_INVALID_ARG, "T1 and T2 must be > 0 (INFINITY for none)");
    }
    for (size_t k = 0; k < s->kappa.size(); ++k)
        if (!(s->kappa[k] >= 0.0) || !std::isfinite(s->kappa[k]))
            return fail(RMS_E_INVALID_ARG, "kappa must be finite and >= 0");
    for (size_t k = 0; k < s->rho.size(); ++k)
        if (!(s->rho[k] >= 0.0) || !std::isfinite(s->rho[k]))
            return fail(RMS_E_INVALID_ARG, "rho must be finite and >= 0");
    for (size_t k = 0; k < s->conc.size(); ++k)
        if (!s->dead[k] && (!(s->conc[k] > 0.0) || !std::isfinite(s->conc[k])))
            return fail(RMS_E_INVALID_ARG, "conc must be finite and > 0 for every live label (mark c = 0 dead)");
    RMS_TRY(upload(&s->d_labels, d->labels, (size_t)nvox, st, d->labels_on_device != 0));
    RMS_TRY(upload(&s->d_D, s->D.data(), L, st));
    RMS_TRY(upload(&s->d_T2, s->T2.data(), L, st));
    RMS_TRY(upload(&s->d_T1, s->T1.data(), L, st));
    RMS_TRY(upload(&s->d_kappa, s->kappa.data(), (size_t)L * L, st));
    if (!s->rho.empty()) RMS_TRY(upload(&s->d_rho, s->rho.data(), (size_t)L * L, st));
    RMS_TRY(upload(&s->d_dead, s->dead.data(), L, st));
    // every label must be < L
    uint32_t *d_max = nullptr;
    RMS_CUDA(cudaMallocAsync((void **)&d_max, sizeof(uint32_t), st));
    RMS_CUDA(cudaMemsetAsync(d_max, 0, sizeof(uint32_t), st));
    max_label_kernel<<<1024, 256, 0, st>>>(s->d_labels, nvox, d_max);
    RMS_CUDA(cudaGetLastError());
    uint32_t mx = 0;
    RMS_CUDA(cudaMemcpyAsync(&mx, d_max, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RMS_CUDA(cudaFreeAsync(d_max, st));
    RMS_CUDA(cudaStreamSynchronize(st));
    if ((int64_t)mx >= L) return fail(RMS_E_INVALID_ARG, "a label value is >= n_labels");
    if (!s->conc.empty()) RMS_TRY(concentration_tables(s, nvox, st));
    bool any_dead = false;
    for (int c = 0; c < L; ++c) any_dead |= s->dead[c] != 0;
    if (!any_dead) {
        s->n_ok = nvox;
    } else {
        const int64_t nblk = (nvox + kOkBlock - 1) / kOkBlock;
        int32_t *d_cnt = nullptr;
        int64_t *d_tot = nullptr;
        RMS_CUDA(cudaMallocAsync((void **)&d_cnt, sizeof(int32_t) * nblk, st));
        RMS_CUDA(cudaMallocAsync((void **)&d_tot, sizeof(int64_t), st));
        ok_count_kernel<<<(unsigned)nblk, kOkBlock, 0, st>>>(s->d_labels, nvox, s->d_dead, d_cnt);
        exclusive_scan_kernel<<<1, 1024, 0, st>>>(d_cnt, nblk, d_tot);
        int64_t tot = 0;
        RMS_CUDA(cudaMemcpyAsync(&tot, d_tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        RMS_CUDA(cudaStreamSynchronize(st));
        if (tot == 0) {
            cudaFreeAsync(d_cnt, st);
            cudaFreeAsync(d_tot, st);
            return fail(RMS_E_INVALID_ARG, "every voxel is dead");
        }
        RMS_CUDA(cudaMallocAsync((void **)&s->d_ok, sizeof(int32_t) * tot, st));
        ok_fill_kernel<<<(unsigned)nblk, kOkBlock, 0, st>>>(s->d_labels, nvox, s->d_dead, d_cnt, s->d_ok);
        RMS_CUDA(cudaGetLastError());
        RMS_CUDA(cudaFreeAsync(d_cnt, st));
        RMS_CUDA(cudaFreeAsync(d_tot, st));
        s->n_ok = tot;
    }
    RMS_CUDA(cudaStreamSynchronize(st));
    return RMS_OK;
}

extern "C" rms_status rms_create_substrate(const rms_substrate_desc *d, rms_substrate **out)
{
    if (!d || !out || !d->labels || !d->D) return fail(RMS_E_INVALID_ARG, "null descriptor field");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || (int64_t)d->nx * d->ny * d->nz >= (1ll << 31))
        return fail(RMS_E_INVALID_ARG, "grid size out of range");
    if (!(d->voxel_um > 0.0) || !std::isfinite(d->voxel_um)) return fail(RMS_E_INVALID_ARG, "voxel_um must be > 0");
    if (d->n_labels < 1 || d->n_labels > 65536) return fail(RMS_E_INVALID_ARG, "n_labels out of range");
    rms_substrate *s = new (std::nothrow) rms_substrate();
    if (!s) return fail(RMS_E_OOM, "host allocation");
    cudaGetDevice(&s->device);
    rms_status r = create_substrate_impl(d, s);
    if (r < 0) {
        free_substrate(s, (cudaStream_t)d->stream);
        cudaStreamSynchronize((cudaStream_t)d->stream);
        delete s;
        return r;
    }
    *out = s;
    return RMS_OK;
}

extern "C" rms_status rms_destroy_substrate(rms_substrate *s)
{
    if (!s) return RMS_OK;
    if (s->refs.load() > 0) return fail(RMS_E_BUSY, "substrate still used by a sequence");
    cudaDeviceSynchronize();
    free_substrate(s, 0);
    cudaStreamSynchronize(0);
    delete s;
    return RMS_OK;
}

// ------------------------------------------------------------------ sequence

// Bernoulli threshold: min(floor(P 2^32), 2^32 - 1); 0 for P <= 0.
static uint32_t threshold_of(double P)
{
    if (!(P > 0.0)) return 0u;
    if (P >= 1.0) return 0xFFFFFFFFu;
    const double x = std::floor(P * 4294967296.0);
    return x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
}

// (c_to / c_from)^lambda seen from the walker's side: lambda fixed (the
// label of lower index is side 1, the other side uses 1 - lambda) or, for
// lambda < 0, the minimiser of alpha_lambda (App. C.2).
static double conc_factor(double c_from, double c_to, double D_from, double D_to, double lambda, bool side1)
{
    const double lam = lambda < 0.0 ? 1.0 / (1.0 + (c_to * std::sqrt(D_to)) / (c_from * std::sqrt(D_from)))
                                    : (side1 ? lambda : 1.0 - lambda);
    return std::pow(c_to / c_from, lam);
}

// Permeation thresholds with spin concentrations (App. C.2, the generalised
// Eq. 3 with the finite-step correction kappa = kappa0 / (1 - alpha_lambda))
// or by Baxter's rule (App. C.3, P = c2 sqrt(D2) / (c1 sqrt(D1)), at most 1;
// kappa > 0 marks the permeable pairs).  Computed on the host because the
// generalised form needs pow: this unit is built with -ffp-contract=off and
// the operations follow the order written, so the thresholds are the same
// bits as any IEEE evaluation of that order with the same libm.
static void host_pair_tables(const rms_substrate *sub, double dt, std::vector<uint32_t> &T, bool &warn)
{
    const int L = sub->L;
    const double C = 2.0 / 3.0;
    std::vector<double> ds(L);
    for (int c = 0; c < L; ++c) ds[c] = std::sqrt((6.0 * sub->D[c]) * dt);
    T.assign((size_t)L * L, 0u);
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b) {
            const double k = sub->kappa[(size_t)a * L + b];
            if (a == b || sub->dead[a] || sub->dead[b] || !(k > 0.0)) continue;
            const double ca = sub->conc.empty() ? 1.0 : sub->conc[a];
            const double cb = sub->conc.empty() ? 1.0 : sub->conc[b];
            double P;
            if (sub->perm_model == RMS_PERM_BAXTER) {
                P = (cb * std::sqrt(sub->D[b])) / (ca * std::sqrt(sub->D[a]));
            } else {
                const double fab = conc_factor(ca, cb, sub->D[a], sub->D[b], sub->lambda, a < b);
                const double fba = conc_factor(cb, ca, sub->D[b], sub->D[a], sub->lambda, b < a);
                const double num = (((k * ds[a]) / sub->D[a]) * fab) * C;
                const double den = 1.0 + ((k / 2.0) * (((ds[a] / sub->D[a]) * fab) + ((ds[b] / sub->D[b]) * fba))) * C;
                P = num / den;
                if (P > 1.0) warn = true;
            }
            T[(size_t)a * L + b] = threshold_of(P);
        }
}

static void free_sequence(rms_sequence *q, cudaStream_t st)
{
    void *p[] = {q->d_s64, q->d_dtR64, q->d_wG64, q->d_s32, q->d_dtR32, q->d_wG32, q->d_T, q->d_Tmt,
                 q->d_flags, q->d_mode, q->d_rec_of, q->d_dirs, q->d_b, q->d_bs, q->d_q, q->d_trig};
    for (void *x : p)
        if (x) cudaFreeAsync(x, st);
}

static rms_status set_sequence_impl(rms_substrate *sub, const rms_sequence_desc *d, rms_sequence *q,
                                    bool *warn)
{
    NvtxRange range("rms: sequence tables");
    cudaStream_t st = 0;
    const int L = sub->L;
    const int64_t N = d->n_steps;
    const int S = d->n_shapes;
    q->sub = sub;
    q->dt = d->dt_ms;
    q->n_steps = N;
    q->S = S;
    q->n_dirs = d->n_dirs;
    q->n_b = d->n_b;
    q->n_rec = d->n_rec;
    q->rec_steps.assign(d->rec_steps, d->rec_steps + d->n_rec);
    for (int c = 0; c < L; ++c) {
        if (sub->dead[c]) continue;
        if (std::sqrt((6.0 * sub->D[c]) * d->dt_ms) >= sub->voxel_um)
            return fail(RMS_E_STEP_TOO_LARGE, "step length sqrt(6 D dt) >= voxel size for label " + std::to_string(c));
        if (!std::isinf(sub->T2[c]) || !std::isinf(sub->T1[c])) q->any_relax = 1;
    }
    for (int i = 0; i < d->n_rec; ++i) {
        if (d->rec_steps[i] < 1 || d->rec_steps[i] > N || (i > 0 && d->rec_steps[i] <= d->rec_steps[i - 1]))
            return fail(RMS_E_INVALID_ARG, "rec_steps must be strictly increasing in [1, n_steps]");
    }
    for (int i = 0; i < d->n_b; ++i)
        if (!(d->b[i] >= 0.0)) return fail(RMS_E_INVALID_ARG, "b-values must be >= 0");
    if (d->mode)
        for (int64_t k = 0; k < N; ++k)
            if (d->mode[k] > 2) return fail(RMS_E_INVALID_ARG, "mode values are 0, 1 or 2");
    RMS_CUDA(cudaMallocAsync((void **)&q->d_s64, sizeof(double) * L, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_s32, sizeof(float) * L, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_dtR64, sizeof(double) * 3 * L, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_dtR32, sizeof(float) * 3 * L, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_T, sizeof(uint32_t) * (size_t)L * L, st));
    if (sub->d_rho) RMS_CUDA(cudaMallocAsync((void **)&q->d_Tmt, sizeof(uint32_t) * (size_t)L * L, st));
    const size_t nG = (size_t)S * (N ? N : 1);
    RMS_CUDA(cudaMallocAsync((void **)&q->d_wG64, sizeof(double) * nG, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_wG32, sizeof(float) * nG, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_flags, N ? N : 1, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_rec_of, sizeof(int32_t) * (N ? N : 1), st));
    if (d->mode) {
        RMS_TRY(upload(&q->d_mode, d->mode, (size_t)N, st));
        q->has_mode = 1;
    }
    RMS_TRY(upload(&q->d_dirs, d->dirs, (size_t)3 * d->n_dirs, st));
    RMS_TRY(upload(&q->d_b, d->b, (size_t)d->n_b, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_bs, sizeof(double) * S, st));
    RMS_CUDA(cudaMallocAsync((void **)&q->d_trig, sizeof(double) * 2 * kTrigParts, st));
    trig_table_kernel<<<kTrigParts / 128, 128, 0, st>>>(q->d_trig);
    RMS_CUDA(cudaMallocAsync((void **)&q->d_q, sizeof(double) * S * d->n_b, st));
    double *d_G = nullptr;
    int64_t *d_rec = nullptr;
    int32_t *d_warn = nullptr;
    RMS_TRY(upload(&d_G, d->G, (size_t)S * N, st));
    RMS_TRY(upload(&d_rec, d->rec_steps, (size_t)d->n_rec, st));
    RMS_CUDA(cudaMallocAsync((void **)&d_warn, sizeof(int32_t), st));
    RMS_CUDA(cudaMemsetAsync(d_warn, 0, sizeof(int32_t), st));
    label_tables_kernel<<<(L + 127) / 128, 128, 0, st>>>(L, sub->d_D, sub->d_T2, sub->d_T1, d->dt_ms, sub->voxel_um,
                                                           q->d_s64, q->d_s32, q->d_dtR64, q->d_dtR32);
    const int64_t LL = (int64_t)L * L;
    pair_tables_kernel<<<(unsigned)((LL + 255) / 256), 256, 0, st>>>(L, sub->d_D, sub->d_kappa, sub->d_dead,
                                                                      d->dt_ms, q->d_T, d_warn);
    if (sub->d_rho)
        mt_tables_kernel<<<(unsigned)((LL + 255) / 256), 256, 0, st>>>(L, sub->d_D, sub->d_rho, sub->d_dead,
                                                                        d->dt_ms, q->d_Tmt, d_warn);
    std::vector<uint32_t> hostT;  // lives until the stream synchronisation below
    bool host_warn = false;
    if (!sub->conc.empty() || sub->perm_model == RMS_PERM_BAXTER) {
        host_pair_tables(sub, d->dt_ms, hostT, host_warn);
        RMS_CUDA(cudaMemcpyAsync(q->d_T, hostT.data(), sizeof(uint32_t) * hostT.size(), cudaMemcpyHostToDevice, st));
    }
    if (N > 0)
        step_tables_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, S, d->dt_ms, d_G, d_rec, d->n_rec,
                                                                         q->d_wG64, q->d_wG32, q->d_flags,
                                                                         q->d_rec_of);
    bvalue_kernel<<<(unsigned)std::max(S, 1), kBvThreads, 0, st>>>(N, S, d->dt_ms, d_G, d->n_b, q->d_b, q->d_bs,
                                                                    q->d_q);
    RMS_CUDA(cudaGetLastError());
    int32_t w = 0;
    RMS_CUDA(cudaMemcpyAsync(&w, d_warn, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RMS_CUDA(cudaFreeAsync(d_G, st));
    RMS_CUDA(cudaFreeAsync(d_rec, st));
    RMS_CUDA(cudaFreeAsync(d_warn, st));
    RMS_CUDA(cudaStreamSynchronize(st));
    *warn = w != 0 || host_warn;
    return RMS_OK;
}

extern "C" rms_status rms_set_sequence(rms_substrate *sub, const rms_sequence_desc *d, rms_sequence **out)
{
    if (!sub || !d || !out) return fail(RMS_E_INVALID_ARG, "null argument");
    *out = nullptr;
    if (!(d->dt_ms > 0.0) || !std::isfinite(d->dt_ms)) return fail(RMS_E_INVALID_ARG, "dt must be > 0");
    if (d->n_steps < 0 || d->n_steps > 2000000000ll) return fail(RMS_E_INVALID_ARG, "n_steps out of range");
    if (d->n_shapes < 1 || d->n_shapes > kMaxShapes) return fail(RMS_E_INVALID_ARG, "n_shapes must be 1..8");
    if (d->n_dirs < 1 || d->n_b < 1 || (int64_t)d->n_shapes * d->n_dirs * d->n_b > 8000000)
        return fail(RMS_E_INVALID_ARG, "n_shapes * n_dirs * n_b must be in 1..8e6");
    if ((d->n_steps > 0 && !d->G) || d->n_dirs < 1 || !d->dirs || d->n_b < 1 || !d->b || d->n_rec < 0 ||
        (d->n_rec > 0 && !d->rec_steps))
        return fail(RMS_E_INVALID_ARG, "missing waveform, directions, b-values or recording steps");
    rms_sequence *q = new (std::nothrow) rms_sequence();
    if (!q) return fail(RMS_E_OOM, "host allocation");
    bool warn = false;
    rms_status r = set_sequence_impl(sub, d, q, &warn);
    if (r < 0) {
        free_sequence(q, 0);
        cudaStreamSynchronize(0);
        delete q;
        return r;
    }
    sub->refs.fetch_add(1);
    *out = q;
    if (warn) {
        g_last_error = "some permeation probability of Eq. 3 exceeded 1 and was clamped";
        return RMS_W_PROB_RANGE;
    }
    return RMS_OK;
}

extern "C" rms_status rms_sequence_bvalues(const rms_sequence *q, double *bs)
{
    if (!q || !bs) return fail(RMS_E_INVALID_ARG, "null argument");
    RMS_CUDA(cudaMemcpy(bs, q->d_bs, sizeof(double) * q->S, cudaMemcpyDeviceToHost));
    return RMS_OK;
}

extern "C" rms_status rms_destroy_sequence(rms_sequence *q)
{
    if (!q) return RMS_OK;
    if (q->refs.load() > 0) return fail(RMS_E_BUSY, "sequence still used by a run");
    cudaDeviceSynchronize();
    free_sequence(q, 0);
    cudaStreamSynchronize(0);
    q->sub->refs.fetch_sub(1);
    delete q;
    return RMS_OK;
}

// ------------------------------------------------------------------ run

template <typename Real>
size_t rms::layout_state(WalkerState<Real> &st, char *base, int64_t W, int S, bool hash, bool f32, bool counts,
                         bool wid)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return p;
    };
    for (int a = 0; a < 3; ++a) st.o[a] = (Real *)take(sizeof(Real) * W);
    for (int a = 0; a < 3; ++a) st.o0[a] = (Real *)take(sizeof(Real) * W);
    for (int a = 0; a < 3; ++a) st.i0[a] = (int32_t *)take(sizeof(int32_t) * W);
    for (int a = 0; a < 3; ++a) st.di[a] = (int32_t *)take(sizeof(int32_t) * W);
    st.c = (int32_t *)take(sizeof(int32_t) * W);
    st.A = (Real *)take(sizeof(Real) * W);
    st.A_c = f32 ? (Real *)take(sizeof(Real) * W) : nullptr;
    st.phase = (Real *)take(sizeof(Real) * W * S * 3);
    st.phase_c = f32 ? (Real *)take(sizeof(Real) * W * S * 3) : nullptr;
    st.hash = hash ? (uint64_t *)take(sizeof(uint64_t) * W) : nullptr;
    st.counts = counts ? (int32_t *)take(sizeof(int32_t) * 3 * W) : nullptr;
    st.wid = wid ? (int32_t *)take(sizeof(int32_t) * W) : nullptr;
    return off;
}

template <typename Real>
ReqDesc<Real> rms::run_desc(rms_run_handle *r)
{
    rms_sequence *q = r->seq;
    rms_substrate *sub = q->sub;
    ReqDesc<Real> d{};
    d.g = Geometry{sub->d_labels, sub->nx, sub->ny, sub->nz, sub->periodic[0], sub->periodic[1], sub->periodic[2],
                   sub->voxel_um, (float)sub->voxel_um};
    if constexpr (std::is_same<Real, float>::value) {
        d.t = Tables<float>{q->d_s32, q->d_dtR32, q->d_T, q->d_Tmt, sub->L, q->d_wG32, q->d_flags, q->d_rec_of,
                            q->d_mode, q->any_relax, q->d_trig};
        d.st = r->st32;
    } else {
        d.t = Tables<double>{q->d_s64, q->d_dtR64, q->d_T, q->d_Tmt, sub->L, q->d_wG64, q->d_flags, q->d_rec_of,
                             q->d_mode, q->any_relax, q->d_trig};
        d.st = r->st64;
    }
    d.ctl.seed = r->seed;
    d.ctl.w_begin = r->w_begin;
    d.ctl.n_walkers = r->W;
    d.ctl.n_steps = q->n_steps;
    d.ctl.n_shapes = q->S;
    d.ctl.n_rec = q->n_rec;
    d.ctl.status = r->d_status;
    d.ctl.checked = (r->flags & RMS_CHECKED) != 0;
    d.ctl.cancel = r->d_cancel;
    d.ctl.mom_partial = r->d_mom_partial;
    d.ctl.n_blocks = r->n_blocks;
    round_keys(r->seed, d.ctl.rk);
    return d;
}
template ReqDesc<float> rms::run_desc<float>(rms_run_handle *);
template ReqDesc<double> rms::run_desc<double>(rms_run_handle *);

template <typename Real>
static rms_status init_impl(rms_run_handle *r)
{
    const ReqDesc<Real> d = run_desc<Real>(r);
    const unsigned ib = (unsigned)((r->W + 255) / 256);
    init_kernel<Real><<<ib, 256, 0, r->stream>>>(d.g, r->seq->sub->d_ok, r->seq->sub->n_ok, r->seq->sub->d_acc, d.st,
                                                  d.ctl, (r->flags & kVerifyFlags) != 0);
    RMS_CUDA(cudaGetLastError());
    return RMS_OK;
}

rms_status rms::run_init(rms_run_handle *r)
{
    return r->precision == RMS_FP32 ? init_impl<float>(r) : init_impl<double>(r);
}

template <typename Real>
static rms_status walk_impl(rms_run_handle *r, int64_t k0, int64_t k1)
{
    const ReqDesc<Real> d = run_desc<Real>(r);
    const bool hash = (r->flags & kVerifyFlags) != 0;  // the verification kernel
    const dim3 grid((unsigned)r->n_blocks);
    const int S = r->seq->S;
#define RMS_WALK(IM, MT) \
    RMS_CUDA((launch_walk<Real, IM, MT>(S, hash, grid, r->stream, d.g, d.t, d.st, d.ctl, k0, k1)))
    const bool mt = d.t.Tmt != nullptr;
    switch (r->interaction) {
    case RMS_RS:
        if (mt) RMS_WALK(kInteractRS, true); else RMS_WALK(kInteractRS, false);
        break;
    case RMS_ERL:
        if (mt) RMS_WALK(kInteractERL, true); else RMS_WALK(kInteractERL, false);
        break;
    default:
        if (mt) RMS_WALK(kInteractEC, true); else RMS_WALK(kInteractEC, false);
    }
#undef RMS_WALK
    return RMS_OK;
}

rms_status rms::run_walk(rms_run_handle *r, int64_t k0, int64_t k1)
{
    NvtxRange range("rms: walk slice");
    return r->precision == RMS_FP32 ? walk_impl<float>(r, k0, k1) : walk_impl<double>(r, k0, k1);
}

static int32_t mom_chunks(int32_t n_blocks) { return (n_blocks + kMomChunk - 1) / kMomChunk; }

// Moment sums, the read-out and the normalisation, enqueued on the run's stream.
template <typename Real>
static rms_status finalize_impl(rms_run_handle *r)
{
    rms_sequence *q = r->seq;
    cudaStream_t s = r->stream;
    const WalkerState<Real> st = run_desc<Real>(r).st;
    if (q->n_rec > 0) {
        const int32_t nmc = mom_chunks(r->n_blocks);
        moments_chunk_kernel<<<(unsigned)((int64_t)q->n_rec * nmc), 256, 0, s>>>(r->d_mom_partial, r->n_blocks, nmc,
                                                                              r->d_mom_chunk);
        moments_reduce_kernel<<<(q->n_rec * kMoments + 127) / 128, 128, 0, s>>>(r->d_mom_chunk, q->n_rec, nmc,
                                                                                r->d_mom);
        RMS_CUDA(cudaGetLastError());
    }
    const dim3 rgrid((unsigned)r->n_chunks, (unsigned)((r->n_combo + 1 + kRoBlock - 1) / kRoBlock));
    if constexpr (std::is_same<Real, float>::value)
        readout_f32_kernel<<<rgrid, kRoBlock, 0, s>>>(st.phase, st.phase_c, st.A, st.A_c, r->W, q->S, q->d_q,
                                                      q->d_dirs, q->n_dirs, q->n_b, r->n_combo, r->d_ro_partial);
    else
        readout_kernel<Real><<<rgrid, kRoBlock, 0, s>>>(st.phase, st.phase_c, st.A, st.A_c, r->W, q->S, q->d_q,
                                                        q->d_dirs, q->n_dirs, q->n_b, r->n_combo, r->d_ro_partial);
    readout_reduce_kernel<<<(r->n_combo + 1 + 127) / 128, 128, 0, s>>>(r->d_ro_partial, r->n_chunks, r->n_combo,
                                                                       r->d_S);
    normalise_kernel<<<(r->n_combo + 1 + 127) / 128, 128, 0, s>>>(r->d_S, r->n_combo, normalised_S(r));
    RMS_CUDA(cudaGetLastError());
    return RMS_OK;
}

rms_status rms::run_finalize(rms_run_handle *r)
{
    NvtxRange range("rms: moments and read-out");
    return r->precision == RMS_FP32 ? finalize_impl<float>(r) : finalize_impl<double>(r);
}

void rms::run_free(rms_run_handle *r, bool sync)
{
    cudaStream_t s = r->stream;
    void *p[] = {r->d_state, r->d_state_alt, r->d_sort, r->d_mom_partial, r->d_mom_chunk, r->d_mom, r->d_ro_partial,
                 r->d_S, r->d_status};
    for (void *x : p)
        if (x) cudaFreeAsync(x, s);
    if (sync || r->h_cancel) cudaStreamSynchronize(s);
    if (r->h_cancel) cudaFreeHost(r->h_cancel);
    if (r->ev_start) cudaEventDestroy(r->ev_start);
    if (r->ev_end) cudaEventDestroy(r->ev_end);
}

size_t rms::run_state_bytes(const rms_sequence *q, int64_t W, int32_t precision, uint32_t flags)
{
    WalkerState<double> s64{};
    WalkerState<float> s32{};
    const bool hash = (flags & kVerifyFlags) != 0;
    const int64_t nb = (W + kWalkBlockSize - 1) / kWalkBlockSize;
    const int64_t nc = (W + kRoChunk - 1) / kRoChunk;
    const int64_t ncombo = (int64_t)q->S * q->n_dirs * q->n_b;
    const bool cnt = (flags & RMS_COUNTS) != 0;
    const bool mort = (flags & RMS_MORTON) != 0;
    size_t b = precision == RMS_FP32 ? layout_state<float>(s32, nullptr, W, q->S, hash, true, cnt, mort)
                                     : layout_state<double>(s64, nullptr, W, q->S, hash, false, cnt, mort);
    if (mort) b = 2 * b + morton_scratch_bytes(W);  // second state buffer and sort buffers
    b += sizeof(double) * ((size_t)std::max(q->n_rec, 1) * nb * kMoments + (size_t)std::max(q->n_rec, 1) * kMoments +
                           (size_t)std::max(q->n_rec, 1) * mom_chunks((int32_t)nb) * kMoments +
                           2 * (size_t)(ncombo + 1) * nc + 4 * (size_t)(ncombo + 1));
    return b;
}

// Allocate the run's device memory (stream-ordered) and lay out the state.
rms_status rms::run_setup(rms_run_handle *r, bool with_cancel_and_events)
{
    rms_sequence *q = r->seq;
    cudaStream_t s = r->stream;
    const bool hash = (r->flags & kVerifyFlags) != 0;
    const bool f32 = r->precision == RMS_FP32;
    r->n_blocks = (int32_t)((r->W + walk_block_size() - 1) / walk_block_size());
    r->n_combo = q->S * q->n_dirs * q->n_b;
    r->n_chunks = (int32_t)((r->W + kRoChunk - 1) / kRoChunk);
    const bool cnt = (r->flags & RMS_COUNTS) != 0;
    const bool mort = (r->flags & RMS_MORTON) != 0;
    const size_t bytes = f32 ? layout_state<float>(r->st32, nullptr, r->W, q->S, hash, true, cnt, mort)
                             : layout_state<double>(r->st64, nullptr, r->W, q->S, hash, false, cnt, mort);
    RMS_CUDA(cudaMallocAsync((void **)&r->d_state, bytes, s));
    if (f32)
        layout_state<float>(r->st32, r->d_state, r->W, q->S, hash, true, cnt, mort);
    else
        layout_state<double>(r->st64, r->d_state, r->W, q->S, hash, false, cnt, mort);
    if (mort) {
        RMS_CUDA(cudaMallocAsync((void **)&r->d_state_alt, bytes, s));
        if (f32)
            layout_state<float>(r->st32_alt, r->d_state_alt, r->W, q->S, hash, true, cnt, true);
        else
            layout_state<double>(r->st64_alt, r->d_state_alt, r->W, q->S, hash, false, cnt, true);
        RMS_CUDA(cudaMallocAsync((void **)&r->d_sort, morton_scratch_bytes(r->W), s));
        morton_plan(q->sub->nx, q->sub->ny, q->sub->nz, &r->sort_shift, &r->sort_passes);
    }
    const size_t nmp = (size_t)std::max(q->n_rec, 1) * r->n_blocks * kMoments;
    RMS_CUDA(cudaMallocAsync((void **)&r->d_mom_partial, sizeof(double) * nmp, s));
    // zero: a run that ends before some recording steps reports zero sums for them
    RMS_CUDA(cudaMemsetAsync(r->d_mom_partial, 0, sizeof(double) * nmp, s));
    RMS_CUDA(cudaMallocAsync((void **)&r->d_mom, sizeof(double) * std::max(q->n_rec, 1) * kMoments, s));
    RMS_CUDA(cudaMallocAsync((void **)&r->d_mom_chunk,
                             sizeof(double) * std::max(q->n_rec, 1) * mom_chunks(r->n_blocks) * kMoments, s));
    RMS_CUDA(cudaMallocAsync((void **)&r->d_ro_partial, sizeof(double) * 2 * (size_t)(r->n_combo + 1) * r->n_chunks, s));
    RMS_CUDA(cudaMallocAsync((void **)&r->d_S, sizeof(double) * 4 * (r->n_combo + 1), s));
    RMS_CUDA(cudaMallocAsync((void **)&r->d_status, sizeof(int32_t), s));
    RMS_CUDA(cudaMemsetAsync(r->d_status, 0, sizeof(int32_t), s));
    if (with_cancel_and_events) {
        RMS_CUDA(cudaHostAlloc((void **)&r->h_cancel, sizeof(int32_t), cudaHostAllocMapped));
        *r->h_cancel = 0;
        RMS_CUDA(cudaHostGetDevicePointer((void **)&r->d_cancel, r->h_cancel, 0));
        RMS_CUDA(cudaEventCreate(&r->ev_start));
        RMS_CUDA(cudaEventCreate(&r->ev_end));
    }
    return RMS_OK;
}

// Resume: per-walker state from host arrays (the layouts rms_read_walkers
// writes).  The FP32 form splits each double into its float and the Kahan
// compensation (float - double), so the compensated value is the double's
// to within float rounding of the difference; a saturated walker (+inf)
// keeps kSaturatedF.
template <typename Real>
__global__ void import_kernel(WalkerState<Real> st, int64_t W, int32_t S, const int32_t *i, const double *o,
                              const int32_t *i0, const double *o0, const int32_t *c, const double *A,
                              const double *phase, const uint64_t *hash)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    constexpr bool f32 = std::is_same<Real, float>::value;
    for (int a = 0; a < 3; ++a) {
        st.o[a][w] = (Real)o[3 * w + a];
        st.o0[a][w] = (Real)o0[3 * w + a];
        st.i0[a][w] = i0[3 * w + a];
        st.di[a][w] = i[3 * w + a] - i0[3 * w + a];
    }
    st.c[w] = c[w];
    const double a = A[w];
    if constexpr (f32) {
        if (isinf(a)) {
            st.A[w] = kSaturatedF;
            st.A_c[w] = 0.0f;
        } else {
            const float hi = (float)a;
            st.A[w] = hi;
            st.A_c[w] = (float)((double)hi - a);
        }
    } else {
        st.A[w] = a;
    }
    for (int k = 0; k < S * 3; ++k) {
        const double p = phase[(int64_t)w * S * 3 + k];
        const int s = k / 3, ax = k % 3;
        const int64_t at = ((int64_t)s * 3 + ax) * W + w;
        if constexpr (f32) {
            const float hi = (float)p;
            st.phase[at] = hi;
            st.phase_c[at] = (float)((double)hi - p);
        } else {
            st.phase[at] = p;
        }
    }
    if (st.hash) st.hash[w] = hash ? hash[w] : 0ull;
    if (st.counts)
        for (int k = 0; k < 3; ++k) st.counts[(int64_t)k * W + w] = 0;
    if (st.wid) st.wid[w] = (int32_t)w;
}

// Upload a stored state and seed the moment partials with the sums of the
// recording steps it has passed (into block 0's slot: the fixed-order sum
// over blocks then returns them unchanged).
static rms_status run_import(rms_run_handle *r, const rms_run_state *from)
{
    rms_sequence *q = r->seq;
    cudaStream_t s = r->stream;
    const int64_t W = r->W;
    const int S = q->S;
    int32_t *d_i = nullptr, *d_i0 = nullptr, *d_c = nullptr;
    double *d_o = nullptr, *d_o0 = nullptr, *d_A = nullptr, *d_ph = nullptr;
    uint64_t *d_h = nullptr;
    RMS_TRY(upload(&d_i, from->i, (size_t)3 * W, s));
    RMS_TRY(upload(&d_i0, from->i0, (size_t)3 * W, s));
    RMS_TRY(upload(&d_o, from->o, (size_t)3 * W, s));
    RMS_TRY(upload(&d_o0, from->o0, (size_t)3 * W, s));
    RMS_TRY(upload(&d_c, from->c, (size_t)W, s));
    RMS_TRY(upload(&d_A, from->A, (size_t)W, s));
    RMS_TRY(upload(&d_ph, from->phase, (size_t)3 * S * W, s));
    if (from->hash) RMS_TRY(upload(&d_h, from->hash, (size_t)W, s));
    const unsigned nb = (unsigned)((W + 255) / 256);
    if (r->precision == RMS_FP32)
        import_kernel<float><<<nb, 256, 0, s>>>(r->st32, W, S, d_i, d_o, d_i0, d_o0, d_c, d_A, d_ph, d_h);
    else
        import_kernel<double><<<nb, 256, 0, s>>>(r->st64, W, S, d_i, d_o, d_i0, d_o0, d_c, d_A, d_ph, d_h);
    RMS_CUDA(cudaGetLastError());
    if (from->moments)
        for (int rr = 0; rr < q->n_rec; ++rr)
            if (q->rec_steps[rr] <= from->step)
                RMS_CUDA(cudaMemcpyAsync(r->d_mom_partial + (size_t)rr * r->n_blocks * kMoments, from->moments + 22 * rr,
                                         sizeof(double) * kMoments, cudaMemcpyHostToDevice, s));
    void *tmp[] = {d_i, d_i0, d_c, d_o, d_o0, d_A, d_ph, d_h};
    for (void *x : tmp)
        if (x) RMS_CUDA(cudaFreeAsync(x, s));
    RMS_CUDA(cudaStreamSynchronize(s));  // the host arrays may go once this returns
    return RMS_OK;
}

// Set up, then initialise (or resume) and enqueue steps (k_first, k_last].
static rms_status run_impl(rms_run_handle *r, int32_t spl, const rms_run_state *from, int64_t k_first,
                           int64_t k_last)
{
    NvtxRange range("rms: run");
    RMS_TRY(run_setup(r, true));
    if (from)
        RMS_TRY(run_import(r, from));
    else
        RMS_TRY(run_init(r));
    RMS_CUDA(cudaEventRecord(r->ev_start, r->stream));
    for (int64_t k0 = k_first; k0 < k_last; k0 += spl) {
        if (r->flags & RMS_MORTON) RMS_TRY(run_rebucket(r));
        RMS_TRY(run_walk(r, k0, std::min<int64_t>(k_last, k0 + spl)));
    }
    RMS_CUDA(cudaEventRecord(r->ev_end, r->stream));
    return run_finalize(r);
}

extern "C" rms_status rms_run(rms_sequence *q, const rms_run_desc *d, rms_run_handle **out)
{
    return rms_run_range(q, d, nullptr, 0, out);
}

extern "C" rms_status rms_run_range(rms_sequence *q, const rms_run_desc *d, const rms_run_state *from,
                                    int64_t step_end, rms_run_handle **out)
{
    if (!q || !d || !out) return fail(RMS_E_INVALID_ARG, "null argument");
    *out = nullptr;
    const int64_t k_first = from ? from->step : 0;
    const int64_t k_last = step_end > 0 ? step_end : q->n_steps;
    if (from && (!from->i || !from->o || !from->i0 || !from->o0 || !from->c || !from->A ||
                 (q->S > 0 && !from->phase)))
        return fail(RMS_E_INVALID_ARG, "resume state: null array");
    if (k_first < 0 || k_first > k_last || k_last > q->n_steps || step_end < 0)
        return fail(RMS_E_INVALID_ARG, "need 0 <= from->step <= step_end <= n_steps (step_end 0: n_steps)");
    if (d->n_walkers < 1 || d->n_walkers > (1ll << 31) - 1 || d->walker_begin < 0)
        return fail(RMS_E_INVALID_ARG, "n_walkers must be in [1, 2^31) and walker_begin >= 0");
    if (d->precision != RMS_FP64 && d->precision != RMS_FP32)
        return fail(RMS_E_INVALID_ARG, "precision must be RMS_FP64 or RMS_FP32");
    if (d->flags & ~(kVerifyFlags | RMS_MORTON)) return fail(RMS_E_INVALID_ARG, "unknown flag");
    if (d->steps_per_launch < 0) return fail(RMS_E_INVALID_ARG, "steps_per_launch must be >= 0");
    if (d->interaction != RMS_EC && d->interaction != RMS_RS && d->interaction != RMS_ERL)
        return fail(RMS_E_INVALID_ARG, "interaction must be RMS_EC, RMS_RS or RMS_ERL");
    rms_run_handle *r = new (std::nothrow) rms_run_handle();
    if (!r) return fail(RMS_E_OOM, "host allocation");
    r->seq = q;
    r->W = d->n_walkers;
    r->w_begin = d->walker_begin;
    r->seed = d->seed;
    r->precision = d->precision;
    r->flags = d->flags;
    r->interaction = d->interaction;
    r->stream = (cudaStream_t)d->stream;
    int32_t spl = d->steps_per_launch;
    if (spl == 0) {
        // about 2e9 walker-steps per launch (a few tens of ms); 8e9 with Morton
        // re-bucketing, which runs once per launch (locality holds that long)
        const int64_t target = ((r->flags & RMS_MORTON) ? 8000000000ll : 2000000000ll) / std::max<int64_t>(r->W, 1);
        spl = (int32_t)std::max<int64_t>(64, std::min<int64_t>(target, std::max<int64_t>(q->n_steps, 1)));
    }
    rms_status st = run_impl(r, spl, from, k_first, k_last);
    if (st < 0) {
        run_free(r, true);
        delete r;
        return st;
    }
    q->refs.fetch_add(1);
    *out = r;
    return RMS_OK;
}

extern "C" rms_status rms_run_query(rms_run_handle *r)
{
    if (!r) return fail(RMS_E_INVALID_ARG, "null run");
    cudaError_t e = cudaStreamQuery(r->stream);
    if (e == cudaErrorNotReady) return RMS_E_NOT_READY;
    RMS_CUDA(e);
    return RMS_OK;
}

extern "C" rms_status rms_cancel(rms_run_handle *r)
{
    if (!r) return fail(RMS_E_INVALID_ARG, "null run");
    *(volatile int32_t *)r->h_cancel = 1;
    return RMS_OK;
}

static rms_status finish(rms_run_handle *r)
{
    RMS_CUDA(cudaStreamSynchronize(r->stream));
    if (*(volatile int32_t *)r->h_cancel) return fail(RMS_E_CANCELLED, "run was cancelled");
    int32_t status = 0;
    RMS_CUDA(cudaMemcpy(&status, r->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (status & kErrInvariant)
        return fail(RMS_E_DEVICE, "a walker invariant broke (RMS_CHECKED); device status " + std::to_string(status));
    if (status & kErrOrder)
        return fail(RMS_E_DEVICE, "the walker re-ordering (RMS_MORTON) gave a slot out of range; device status " +
                                      std::to_string(status));
    if (status & ~kWarnLeaps) return fail(RMS_E_DEVICE, "device status " + std::to_string(status));
    if (status & kWarnLeaps) {
        set_last_error("an ERL step found no admissible direction in RMS_MAX_LEAPS draws; "
                       "that walker stayed for the step");
        return RMS_W_LEAP_LIMIT;
    }
    return RMS_OK;
}

extern "C" rms_status rms_read_signal(rms_run_handle *r, double *S_re, double *S_im, double *moments, double *alpha_sum)
{
    if (!r) return fail(RMS_E_INVALID_ARG, "null run");
    const rms_status fin = finish(r);
    if (fin < 0) return fin;
    std::vector<double> S((size_t)2 * (r->n_combo + 1));
    RMS_CUDA(cudaMemcpy(S.data(), normalised_S(r), sizeof(double) * S.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < r->n_combo; ++k) {
        if (S_re) S_re[k] = S[2 * k];
        if (S_im) S_im[k] = S[2 * k + 1];
    }
    if (alpha_sum) *alpha_sum = S[2 * r->n_combo];
    if (moments && r->seq->n_rec > 0)
        RMS_CUDA(cudaMemcpy(moments, r->d_mom, sizeof(double) * r->seq->n_rec * kMoments, cudaMemcpyDeviceToHost));
    return fin;
}

extern "C" rms_status rms_read_partials(rms_run_handle *r, double *num_re, double *num_im, double *alpha_sum,
                                        double *moments)
{
    if (!r) return fail(RMS_E_INVALID_ARG, "null run");
    const rms_status fin = finish(r);
    if (fin < 0) return fin;
    std::vector<double> S((size_t)2 * (r->n_combo + 1));
    RMS_CUDA(cudaMemcpy(S.data(), r->d_S, sizeof(double) * S.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < r->n_combo; ++k) {
        if (num_re) num_re[k] = S[2 * k];
        if (num_im) num_im[k] = S[2 * k + 1];
    }
    if (alpha_sum) *alpha_sum = S[2 * r->n_combo];
    if (moments && r->seq->n_rec > 0)
        RMS_CUDA(cudaMemcpy(moments, r->d_mom, sizeof(double) * r->seq->n_rec * kMoments, cudaMemcpyDeviceToHost));
    return fin;
}

extern "C" rms_status rms_normalise_partials(int64_t n_combo, const double *num_re, const double *num_im,
                                             double alpha_sum, double *S_re, double *S_im)
{
    if (n_combo < 0 || (n_combo > 0 && (!num_re || !num_im || !S_re || !S_im)))
        return fail(RMS_E_INVALID_ARG, "rms_normalise_partials: n_combo >= 0 and non-null arrays");
    for (int64_t k = 0; k < n_combo; ++k) {
        S_re[k] = num_re[k] / alpha_sum;
        S_im[k] = num_im[k] / alpha_sum;
    }
    return RMS_OK;
}

extern "C" rms_status rms_philox4x32_10(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out,
                                        void *stream)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(RMS_E_INVALID_ARG, "rms_philox4x32_10: bad arguments");
    if (n == 0) return RMS_OK;
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7FFFFFFF) return fail(RMS_E_INVALID_ARG, "rms_philox4x32_10: n too large");
    philox_words_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(ctr, key, n, out);
    RMS_CUDA(cudaGetLastError());
    return RMS_OK;
}

extern "C" rms_status rms_read_walkers(rms_run_handle *r, int32_t *i, double *o, int32_t *i0, double *o0, int32_t *c,
                                       double *A, double *phase, uint64_t *hash)
{
    if (!r) return fail(RMS_E_INVALID_ARG, "null run");
    const rms_status fin = finish(r);
    if (fin < 0) return fin;
    const int64_t W = r->W;
    const int S = r->seq->S;
    cudaStream_t s = r->stream;
    char *buf = nullptr;
    const size_t bi = sizeof(int32_t) * 3 * W, bo = sizeof(double) * 3 * W, bc = sizeof(int32_t) * W,
                 bA = sizeof(double) * W, bp = sizeof(double) * 3 * S * W, bh = sizeof(uint64_t) * W;
    // every sub-buffer starts on a 256-byte boundary
    const size_t sizes[8] = {bi, bi, bo, bo, bc, bA, bp, bh};
    size_t offs[8], total = 0;
    for (int k = 0; k < 8; ++k) {
        offs[k] = total;
        total += (sizes[k] + 255) & ~size_t(255);
    }
    RMS_CUDA(cudaMallocAsync((void **)&buf, total, s));
    int32_t *di = (int32_t *)(buf + offs[0]), *di0 = (int32_t *)(buf + offs[1]);
    double *dO = (double *)(buf + offs[2]), *dO0 = (double *)(buf + offs[3]);
    int32_t *dc = (int32_t *)(buf + offs[4]);
    double *dA = (double *)(buf + offs[5]);
    double *dp = (double *)(buf + offs[6]);
    uint64_t *dh = (uint64_t *)(buf + offs[7]);
    const unsigned nb = (unsigned)((W + 255) / 256);
    const bool hsh = (r->flags & kVerifyFlags) != 0;
    if (r->precision == RMS_FP32)
        export_kernel<float><<<nb, 256, 0, s>>>(r->st32, W, S, hsh, di, dO, di0, dO0, dc, dA, dp, dh);
    else
        export_kernel<double><<<nb, 256, 0, s>>>(r->st64, W, S, hsh, di, dO, di0, dO0, dc, dA, dp, dh);
    RMS_CUDA(cudaGetLastError());
    struct {
        void *h;
        const void *d;
        size_t n;
    } cp[] = {{i, di, bi}, {i0, di0, bi}, {o, dO, bo}, {o0, dO0, bo}, {c, dc, bc}, {A, dA, bA}, {phase, dp, bp},
              {hash, dh, bh}};
    for (auto &x : cp)
        if (x.h) RMS_CUDA(cudaMemcpyAsync(x.h, x.d, x.n, cudaMemcpyDeviceToHost, s));
    RMS_CUDA(cudaFreeAsync(buf, s));
    RMS_CUDA(cudaStreamSynchronize(s));
    return fin;
}

extern "C" rms_status rms_read_counts(rms_run_handle *r, int64_t *counts)
{
    if (!r || !counts) return fail(RMS_E_INVALID_ARG, "null argument");
    const rms_status fin = finish(r);
    if (fin < 0) return fin;
    const int32_t *d = r->precision == RMS_FP32 ? r->st32.counts : r->st64.counts;
    if (!d) return fail(RMS_E_INVALID_ARG, "the run was made without RMS_COUNTS");
    std::vector<int32_t> h((size_t)3 * r->W), wid;
    RMS_CUDA(cudaMemcpy(h.data(), d, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost));
    const int32_t *dw = r->precision == RMS_FP32 ? r->st32.wid : r->st64.wid;
    if (dw) {  // RMS_MORTON: slot -> walker
        wid.resize((size_t)r->W);
        RMS_CUDA(cudaMemcpy(wid.data(), dw, sizeof(int32_t) * wid.size(), cudaMemcpyDeviceToHost));
    }
    for (int64_t w = 0; w < r->W; ++w) {
        const int64_t u = dw ? wid[(size_t)w] : w;
        for (int a = 0; a < 3; ++a) counts[3 * u + a] = h[(size_t)a * r->W + w];
    }
    return fin;
}

extern "C" rms_status rms_read_slots(rms_run_handle *r, int32_t *walker_of_slot)
{
    if (!r || !walker_of_slot) return fail(RMS_E_INVALID_ARG, "null argument");
    const rms_status fin = finish(r);
    if (fin < 0) return fin;
    const int32_t *dw = r->precision == RMS_FP32 ? r->st32.wid : r->st64.wid;
    if (dw) {
        RMS_CUDA(cudaMemcpy(walker_of_slot, dw, sizeof(int32_t) * (size_t)r->W, cudaMemcpyDeviceToHost));
    } else {
        for (int64_t w = 0; w < r->W; ++w) walker_of_slot[w] = (int32_t)w;
    }
    return fin;
}

extern "C" rms_status rms_run_step_time_ms(rms_run_handle *r, float *ms)
{
    if (!r || !ms) return fail(RMS_E_INVALID_ARG, "null argument");
    RMS_CUDA(cudaEventSynchronize(r->ev_end));
    RMS_CUDA(cudaEventElapsedTime(ms, r->ev_start, r->ev_end));
    return RMS_OK;
}

extern "C" rms_status rms_destroy_run(rms_run_handle *r)
{
    if (!r) return RMS_OK;
    cudaStreamSynchronize(r->stream);
    run_free(r, true);
    r->seq->refs.fetch_sub(1);
    delete r;
    return RMS_OK;
}
