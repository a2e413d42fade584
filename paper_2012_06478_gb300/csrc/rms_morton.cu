// rms_morton.cu -- walkers re-bucketed in Morton order of their voxel
// between step launches (the staging of large label volumes: the label volume
// is the lookup table of Sec. 2.1.1, and walkers that sit next to each other
// in memory then look up neighbouring labels, so a warp's gathers share
// sectors and the blocks resident at one time touch a small part of the
// volume).
//
// A walker's random streams depend only on (seed, walker id, step), so the
// order of the walkers in memory changes no trajectory: the state carries the
// walker id of each slot (WalkerState::wid) and the step kernel draws with it.
// Only the order of the FP64 sums over walkers changes.
//
// The order: a stable least-significant-digit radix sort, 8 bits per pass, of
// the Morton code (bits of x, y, z interleaved) of the walker's wrapped voxel
// coordinates shifted right so that each coordinate keeps at most 8 bits.
// Each pass is a per-tile digit histogram, an exclusive scan of the
// histograms in digit-major order and a stable scatter in which every tile
// ranks its items by warp match and a per-digit scan over its warps.  Then
// every state array is gathered into the second state buffer, which becomes
// the live one.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "rms_handles.h"
#include "rms_internal.h"

namespace rms {

constexpr int kSortTile = 1024;     // items per tile = threads per block, one item each
constexpr int kScanBlock = 1024;    // threads per block of the scan kernels
constexpr int kScanPer = 8;         // items per thread of the scan kernels
constexpr int kScanSpan = kScanBlock * kScanPer;

// The low 10 bits of x moved to every third bit (bit i -> bit 3i).
__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

template <typename Real>
__global__ void morton_key_kernel(WalkerState<Real> st, int64_t W, int32_t nx, int32_t ny, int32_t nz, int32_t shift,
                                  uint32_t *key, int32_t *slot)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W) return;
    const int32_t N[3] = {nx, ny, nz};
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int32_t q = (st.i0[a][i] + st.di[a][i]) % N[a];
        if (q < 0) q += N[a];
        c[a] = (uint32_t)q >> shift;
    }
    key[i] = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
    slot[i] = (int32_t)i;
}

// Digit counts of tile blockIdx.x, stored digit-major: hist[d * n_tiles + tile].
__global__ void __launch_bounds__(kSortTile) sort_hist_kernel(const uint32_t *key, int64_t n, int32_t shift,
                                                              uint32_t *hist, int64_t n_tiles)
{
    __shared__ uint32_t h[256];
    if (threadIdx.x < 256) h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kSortTile + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
    __syncthreads();
    if (threadIdx.x < 256) hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Inclusive scan of v over the block (blockDim.x = kScanBlock); returns the
// block total in *total.
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t *warp_tot, uint32_t *total)
{
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wp] = v;
    __syncthreads();
    if (wp == 0) {
        uint32_t t = warp_tot[lane];  // kScanBlock / 32 = 32 warps
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    if (wp > 0) v += warp_tot[wp - 1];
    *total = warp_tot[31];
    __syncthreads();  // warp_tot may be reused by the caller
    return v;
}

// Block b's sum of a[b*kScanSpan, (b+1)*kScanSpan).
__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const uint32_t *a, int64_t M, uint32_t *bsum)
{
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanSpan + (int64_t)threadIdx.x * kScanPer;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < M) s += a[base + k];
    uint32_t tot;
    block_inclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Exclusive scan of the nb block sums, in place (one block).
__global__ void __launch_bounds__(kScanBlock) scan_bsum_kernel(uint32_t *bsum, int64_t nb)
{
    __shared__ uint32_t wt[32];
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t tot;
        const uint32_t inc = block_inclusive_scan(v, wt, &tot);
        if (i < nb) bsum[i] = carry + inc - v;
        carry += tot;
    }
}

// Exclusive scan of a in place, block b starting from bsum[b].
__global__ void __launch_bounds__(kScanBlock) scan_apply_kernel(uint32_t *a, int64_t M, const uint32_t *bsum)
{
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanSpan + (int64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < M ? a[base + k] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_inclusive_scan(s, wt, &tot) - s + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < M) a[base + k] = run;
        run += v[k];
    }
}

// Stable scatter of tile blockIdx.x: an item goes to the scanned offset of its
// digit for this tile plus the number of items of the same digit before it
// in the tile (earlier warps, then lower lanes of its own warp).
__global__ void __launch_bounds__(kSortTile) sort_scatter_kernel(const uint32_t *kin, const int32_t *vin,
                                                                 uint32_t *kout, int32_t *vout, int64_t n,
                                                                 int32_t shift, const uint32_t *offs, int64_t n_tiles)
{
    __shared__ uint32_t cnt[kSortTile / 32][256];
    for (int t = threadIdx.x; t < (kSortTile / 32) * 256; t += kSortTile) (&cnt[0][0])[t] = 0u;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kSortTile + threadIdx.x;
    const bool valid = i < n;  // the invalid items are the last lanes of the last tile
    const uint32_t k = valid ? kin[i] : 0u;
    const uint32_t d = (k >> shift) & 255u;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0xFFFFu);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0u) cnt[wp][d] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < 256) {
        uint32_t run = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
        for (int w = 0; w < kSortTile / 32; ++w) {
            const uint32_t c = cnt[w][threadIdx.x];
            cnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    if (valid) {
        const uint32_t pos = cnt[wp][d] + rank;
        if ((int64_t)pos < n) {  // always, for a consistent histogram; never written out of bounds
            kout[pos] = k;
            vout[pos] = vin[i];
        }
    }
}

// Slot j of the new order takes the walker in slot perm[j] of the old one.
// A slot index out of range (a broken sort) is reported (kErrOrder) and never
// dereferenced.
template <typename Real>
__global__ void permute_kernel(WalkerState<Real> src, WalkerState<Real> dst, const int32_t *perm, int64_t W,
                               int32_t S, int32_t *status)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= W) return;
    const int64_t p = perm[j];
    if (p < 0 || p >= W) {
        atomicOr(status, kErrOrder);
        return;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dst.o[a][j] = src.o[a][p];
        dst.o0[a][j] = src.o0[a][p];
        dst.i0[a][j] = src.i0[a][p];
        dst.di[a][j] = src.di[a][p];
    }
    dst.c[j] = src.c[p];
    dst.A[j] = src.A[p];
    if (src.A_c) dst.A_c[j] = src.A_c[p];
    for (int k = 0; k < S * 3; ++k) {
        dst.phase[(int64_t)k * W + j] = src.phase[(int64_t)k * W + p];
        if (src.phase_c) dst.phase_c[(int64_t)k * W + j] = src.phase_c[(int64_t)k * W + p];
    }
    if (src.hash) dst.hash[j] = src.hash[p];
    if (src.counts)
        for (int k = 0; k < 3; ++k) dst.counts[(int64_t)k * W + j] = src.counts[(int64_t)k * W + p];
    dst.wid[j] = src.wid[p];
}

static int bit_length(uint32_t x) { return x ? 32 - __builtin_clz(x) : 0; }

void morton_plan(int32_t nx, int32_t ny, int32_t nz, int32_t *shift, int32_t *passes)
{
    const uint32_t nmax = (uint32_t)std::max(nx, std::max(ny, nz));
    const int bits = bit_length(nmax - 1u);  // bits of the largest coordinate
    const int s = std::max(0, bits - 8);
    *shift = s;
    *passes = (3 * (bits - s) + 7) / 8;
}

// The sort buffers of W walkers, carved from one allocation (base nullptr:
// sizes only): keys and slots twice (ping-pong between passes), the tile
// histograms [256][n_tiles] and the scan's block sums, each 256-byte aligned.
struct SortBuffers {
    uint32_t *key[2];
    int32_t *val[2];
    uint32_t *hist, *bsum;
    int64_t n_tiles, M, nb;
    size_t bytes;
};

static SortBuffers sort_buffers(char *base, int64_t W)
{
    SortBuffers b{};
    b.n_tiles = (W + kSortTile - 1) / kSortTile;
    b.M = 256 * b.n_tiles;
    b.nb = (b.M + kScanSpan - 1) / kScanSpan;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return q;
    };
    for (int i = 0; i < 2; ++i) b.key[i] = (uint32_t *)take(sizeof(uint32_t) * W);
    for (int i = 0; i < 2; ++i) b.val[i] = (int32_t *)take(sizeof(int32_t) * W);
    b.hist = (uint32_t *)take(sizeof(uint32_t) * b.M);
    b.bsum = (uint32_t *)take(sizeof(uint32_t) * b.nb);
    b.bytes = off;
    return b;
}

size_t morton_scratch_bytes(int64_t W) { return sort_buffers(nullptr, W).bytes; }

template <typename Real>
static rms_status rebucket_impl(rms_run_handle *r, WalkerState<Real> &st, WalkerState<Real> &alt)
{
    if (r->sort_passes <= 0) return RMS_OK;  // one voxel: nothing to order
    cudaStream_t s = r->stream;
    const int64_t W = r->W;
    const SortBuffers b = sort_buffers(r->d_sort, W);
    uint32_t *const *key = b.key;
    int32_t *const *val = b.val;
    uint32_t *hist = b.hist, *bsum = b.bsum;
    const int64_t n_tiles = b.n_tiles, M = b.M, nb = b.nb;

    const rms_substrate *sub = r->seq->sub;
    const unsigned g256 = (unsigned)((W + 255) / 256);
    morton_key_kernel<Real><<<g256, 256, 0, s>>>(st, W, sub->nx, sub->ny, sub->nz, r->sort_shift, key[0], val[0]);
    RMS_CUDA(cudaGetLastError());
    int cur = 0;
    for (int pass = 0; pass < r->sort_passes; ++pass) {
        const int32_t sh = 8 * pass;
        sort_hist_kernel<<<(unsigned)n_tiles, kSortTile, 0, s>>>(key[cur], W, sh, hist, n_tiles);
        scan_reduce_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(hist, M, bsum);
        scan_bsum_kernel<<<1, kScanBlock, 0, s>>>(bsum, nb);
        scan_apply_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(hist, M, bsum);
        sort_scatter_kernel<<<(unsigned)n_tiles, kSortTile, 0, s>>>(key[cur], val[cur], key[cur ^ 1], val[cur ^ 1],
                                                                    W, sh, hist, n_tiles);
        RMS_CUDA(cudaGetLastError());
        cur ^= 1;
    }
    permute_kernel<Real><<<g256, 256, 0, s>>>(st, alt, val[cur], W, r->seq->S, r->d_status);
    RMS_CUDA(cudaGetLastError());
    std::swap(st, alt);
    std::swap(r->d_state, r->d_state_alt);
    return RMS_OK;
}

rms_status run_rebucket(rms_run_handle *r)
{
    NvtxRange range("rms: Morton re-bucketing");
    return r->precision == RMS_FP32 ? rebucket_impl<float>(r, r->st32, r->st32_alt)
                                    : rebucket_impl<double>(r, r->st64, r->st64_alt);
}

}  // namespace rms
