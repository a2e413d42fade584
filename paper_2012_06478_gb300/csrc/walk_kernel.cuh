// walk_kernel.cuh -- the random-walker time step (Sec. 2.2 items 2-5 of
// Lee, Fieremans & Novikov, arXiv 2012.06478), templated on the arithmetic
// type.  Included by walk_fp64.cu (built without FMA contraction: the plain
// form reproduces the CPU FP64 reference bit for bit) and walk_fp32.cu (the
// precision form: voxel index + FP32 offset, FP32 Kahan-compensated phase),
// and by walk_reject_fp{64,32}.cu and walk_mt_fp{64,32}.cu for the other
// particle-membrane interactions and for absorbing membranes.
//
// One thread owns one walker for a slice of steps; its whole state stays in
// registers for the slice and goes back to global memory (structure of
// arrays, coalesced) at the end.  Per step and walker the only memory
// traffic is the dependent 2-byte label gather across each face met
// (Sec. 2.1.1: the label volume is the lookup table), the threshold of the
// label pair at a membrane (and its saturation threshold, with absorbing
// membranes), and warp-uniform broadcasts of the waveform.
#pragma once

#include <cstdint>
#include <type_traits>

#include "rms_device.cuh"
#include "soft_fp64.cuh"

namespace rms {

constexpr int kWalkBlock = 128;
constexpr int kWalkWarps = kWalkBlock / 32;

template <typename Real>
__device__ __forceinline__ Real clamp01(Real x)
{
    if (x < Real(0)) return Real(0);
    if (x > Real(1)) return Real(1);
    return x;
}
// FP32: the same clamp as __saturatef, which the compiler folds into the
// preceding multiply-add as its saturating form (identical results for the
// non-NaN positions; measured 7 % faster on the FP32 step).
template <>
__device__ __forceinline__ float clamp01<float>(float x)
{
    return __saturatef(x);
}

// FP64 comparisons on the integer ALU.  GB300's FP64 pipe is the scarce
// resource of the plain form, and every comparison or clamp of a double
// would occupy it.  The signed 64-bit pattern of a double orders exactly like
// its value among the non-negative doubles, and its sign bit tells x > 0 and
// x < 0 apart from +-0; the walk's positions, times and step vectors are
// never NaN, so these give the same booleans as the IEEE comparisons.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool dgt0(double x) { return dbits(x) > 0; }  // x > 0
__device__ __forceinline__ bool dlt0(double x)                           // x < 0
{
    const long long b = dbits(x);
    return b < 0 && b != (long long)0x8000000000000000ULL;
}
// a < b for a, b >= +0 (no -0 and no NaN among the arguments)
__device__ __forceinline__ bool dlt_nn(double a, double b) { return dbits(a) < dbits(b); }
// if (x < 0) 0; else if (x > 1) 1; else x -- as clamp01, for any non-NaN x
__device__ __forceinline__ double dclamp01(double x)
{
    const long long b = dbits(x);
    if (b < 0) return b == (long long)0x8000000000000000ULL ? x : 0.0;
    return b > 0x3FF0000000000000LL ? 1.0 : x;
}

// Sec. 2.2 item 2, the direction.  z = 1 - 2u is uniform on [-1, 1] for a
// uniform point of the sphere (Archimedes); the azimuth is
// phi = 2 pi (x1 + 1/2) 2^-32.  Its sine and cosine come from Taylor
// polynomials after an octant reduction in integers -- in the FP64 form a
// table of 1024 angles of [0, pi/4] (filled by poly_sincos), a 5th-order
// polynomial for the offset from the nearest table angle and the
// angle-addition formula -- so the FP64 form uses only +, * and sqrt (the
// same bits as any IEEE machine given the same operation order), and no
// warp ever loops on a rejection.
__device__ __forceinline__ void octant_map(uint32_t oct, double cs, double sn, double &cx, double &sy)
{
    const bool swap = ((oct + 1u) >> 1) & 1u;  // octants 1, 2, 5, 6
    const bool negx = ((oct + 2u) >> 2) & 1u;  // octants 2..5
    const bool negy = (oct >> 2) & 1u;         // octants 4..7
    const double a = swap ? sn : cs, b = swap ? cs : sn;
    cx = negx ? -a : a;
    sy = negy ? -b : b;
}

// The hardware FP64 operations, for the operands the integer-ALU versions
// hand back (zeros, subnormals, out-of-range results).  Out of line, so that
// the compiler cannot evaluate them speculatively beside the integer path:
// inlined, a predicated copy would run on the FP64 pipe at every call.
static __device__ __noinline__ double hw_mul(double a, double b) { return a * b; }
static __device__ __noinline__ double hw_div(double a, double b) { return a / b; }

// FP64 products and quotients of non-negative operands on the integer ALU
// (sfp::mul_rn, div_pos: the IEEE results bit for bit).
// mulr is the product of the form: this one for FP64, a plain multiply for FP32.
__device__ __forceinline__ double dmul(double a, double b)
{
    double p;
    if (!sfp::mul_rn(a, b, p)) p = hw_mul(a, b);
    return p;
}
__device__ __forceinline__ double ddiv_nn(double a, double b)
{
    double q;
    if (!sfp::div_pos(a, b, q)) q = hw_div(a, b);
    return q;
}

__device__ __forceinline__ double mulr(double a, double b) { return dmul(a, b); }
__device__ __forceinline__ float mulr(float a, float b) { return a * b; }

// Exact doubles built from their bits on the integer ALU, so that values
// which need no rounding do not occupy GB300's narrow FP64 pipe.
// k * 2^e2 for an odd |k| < 2^32: no rounding, the same bits as converting k
// and multiplying by the power of two.
__device__ __forceinline__ double odd_scaled(uint32_t mag, bool neg, int e2)
{
    const int p = 31 - __clz((int)mag);  // position of the leading one
    const unsigned long long mant = ((unsigned long long)mag << (52 - p)) & 0x000FFFFFFFFFFFFFULL;
    const unsigned long long bits = (neg ? 0x8000000000000000ULL : 0ULL) |
                                    ((unsigned long long)(p + e2 + 1023) << 52) | mant;
    return __longlong_as_double((long long)bits);
}
// N 2^-64 rounded to the nearest double, ties to even (0 < N < 2^64): the
// IEEE result of a product of doubles whose exact value is N 2^-64.
__device__ __forceinline__ double u64_scaled_rn(unsigned long long N)
{
    const int p = 63 - __clzll((long long)N);
    int e = p - 64;
    unsigned long long q;
    if (p <= 52) {
        q = N << (52 - p);
    } else {
        const int sh = p - 52;
        q = N >> sh;
        const unsigned long long rem = N & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
        if (rem > half || (rem == half && (q & 1ULL))) ++q;
        if (q >> 53) {
            q >>= 1;
            ++e;
        }
    }
    return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) | (q & 0x000FFFFFFFFFFFFFULL)));
}

__device__ __forceinline__ void direction_from(uint32_t x0, uint32_t x1, const double *__restrict__ trig,
                                               double n[3])
{
    // z = 1 - 2 u(x0) = k 2^-32 with the odd integer k = 2^32 - 1 - 2 x0, and
    // (1 - z)(1 + z) = (2^64 - k^2) 2^-64 rounded once: both from integers,
    // the same bits as the CPU FP64 reference's step-by-step evaluation.
    const bool zneg = x0 >= 0x80000000u;
    const uint32_t kmag = zneg ? 2u * x0 + 1u : 0xFFFFFFFFu - 2u * x0;  // |k|
    const double z = odd_scaled(kmag, zneg, -32);
    // Every value below is normal and nonzero for every pair of words, so the
    // integer-ALU products and square root need neither range checks nor a
    // hardware fallback: the argument of the root is at least (2^33 - 1) 2^-64;
    // |e| lies in [2^-30, 2^-11] pi/4, t = e^2 in [2^-61, 2^-22], the table's
    // cosines and sines in [3.8e-4, 1], cs and sn in [7e-10, 1] (the angle is at
    // least 2^-30 pi/4), r in [2^-16, 1]; every product stays far inside the
    // normal range.
    const double r = sfp::sqrt_normal(u64_scaled_rn(0ULL - (unsigned long long)kmag * kmag));
    const uint32_t oct = x1 >> 29;
    uint32_t m = x1 & 0x1FFFFFFFu;
    if (oct & 1u) m = 0x1FFFFFFFu - m;
    // angle (m + 1/2) 2^-29 pi/4 = theta_j + e, theta_j = (2j + 1) 2^-11 pi/4 the
    // centre of part j = top 10 bits of m, |e| <= 2^-11 pi/4
    const uint32_t j = m >> 19;
    const int32_t lo = (int32_t)(m & 0x7FFFFu);
    const int32_t e_int = 2 * lo + 1 - (1 << 19);  // odd
    using sfp::mul_normal;
    const double e = mul_normal(odd_scaled((uint32_t)(e_int < 0 ? -e_int : e_int), e_int < 0, -30), 0.78539816339744830962);
    const double t = mul_normal(e, e);
    const double se = e + mul_normal(mul_normal(e, t), -1.0 / 6.0 + mul_normal(t, 1.0 / 120.0));
    const double ce = 1.0 + mul_normal(t, -1.0 / 2.0 + mul_normal(t, 1.0 / 24.0));
    const double cj = __ldg(trig + 2 * j), sj = __ldg(trig + 2 * j + 1);
    const double cs = mul_normal(cj, ce) - mul_normal(sj, se);
    const double sn = mul_normal(sj, ce) + mul_normal(cj, se);
    double cx, sy;
    octant_map(oct, cs, sn, cx, sy);
    n[0] = mul_normal(r, cx);
    n[1] = mul_normal(r, sy);
    n[2] = z;
}

// FP32 form of the same sampler: shorter polynomials (truncation below
// 4e-7 on [0, pi/4]) and r from the hardware reciprocal square root (about
// 2 ulp; (1 - z)(1 + z) > 0 since |z| < 1) -- errors of the order of the FP32
// form's own rounding, for 2 % of its step time.
__device__ __forceinline__ void direction_from(uint32_t x0, uint32_t x1, const double *, float n[3])
{
    const float z = -((float)(int32_t)(x0 ^ 0x80000000u) + 0.5f) * 0x1p-31f;
    const float rr = (1.0f - z) * (1.0f + z);
    const float r = rr * rsqrtf(rr);
    const uint32_t oct = x1 >> 29;
    uint32_t m = x1 & 0x1FFFFFFFu;
    if (oct & 1u) m = 0x1FFFFFFFu - m;
    const float th = ((float)m + 0.5f) * (0x1p-29f * 0.785398163f);
    const float t = th * th;
    const float sn = th + (th * t) * (-1.0f / 6.0f + t * (1.0f / 120.0f + t * (-1.0f / 5040.0f)));
    const float cs = 1.0f + t * (-0.5f + t * (1.0f / 24.0f + t * (-1.0f / 720.0f + t * (1.0f / 40320.0f))));
    const bool swap = ((oct + 1u) >> 1) & 1u;
    const bool negx = ((oct + 2u) >> 2) & 1u;
    const bool negy = (oct >> 2) & 1u;
    const float a = swap ? sn : cs, b = swap ? cs : sn;
    n[0] = r * (negx ? -a : a);
    n[1] = r * (negy ? -b : b);
    n[2] = z;
}

// Saturation (Sec. 2.1.3): A = +inf (FP64 form) or kSaturatedF (FP32 form).
__device__ __forceinline__ bool saturated(double A) { return dbits(A) == 0x7FF0000000000000LL; }
__device__ __forceinline__ bool saturated(float A) { return A >= kSaturatedF; }
__device__ __forceinline__ void saturate(double &A, double &) { A = __longlong_as_double(0x7FF0000000000000LL); }
__device__ __forceinline__ void saturate(float &A, float &Ac)
{
    A = kSaturatedF;
    Ac = 0.0f;
}

// Word 0 of a step's PERM call: the Bernoulli word of a third membrane event
// in one step.  Rare, so kept out of line: inlined, the ten Philox rounds
// would sit in every pass of the face-event loop (measured: 4 % of the FP32
// step on the axon workload).
static __device__ __noinline__ uint32_t perm_word(uint64_t seed, uint64_t w, uint32_t k, uint32_t call)
{
    return draw(seed, w, k, kTagPerm, call).x;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename Real>
__device__ __forceinline__ void kahan_add(Real &sum, Real &comp, Real x)
{
    const Real y = x - comp;
    const Real t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// The 22 moment terms at a recording step (Sec. 2.3, narrow-pulse D and K):
// alpha, alpha dx_i dx_j (i <= j), alpha dx_i dx_j dx_k dx_l (i<=j<=k<=l),
// each reduced over the warp as soon as it is formed (few live registers);
// lane 0 of each warp leaves the warp's 22 sums in red[22].
__device__ __forceinline__ void warp_moments(double al, const double dx[3], double *red)
{
    const int lane = threadIdx.x & 31;
    int p = 0;
    double r = warp_sum(al);
    if (lane == 0) red[p] = r;
    ++p;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            r = warp_sum(al * dx[a] * dx[b]);
            if (lane == 0) red[p] = r;
            ++p;
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b)
#pragma unroll
            for (int c = b; c < 3; ++c)
#pragma unroll
                for (int d = c; d < 3; ++d) {
                    r = warp_sum(al * dx[a] * dx[b] * dx[c] * dx[d]);
                    if (lane == 0) red[p] = r;
                    ++p;
                }
}

// Steps (k_begin, k_end] for the kWalkBlock walkers of block `block` of a
// run (walkers block*kWalkBlock ...), one walker per thread.  IM is the
// particle-membrane interaction: elastic collision (Sec. 2.1.2-2.1.3, the
// paper's method), or one of the alternatives of App. A and B, in which a
// refused face cancels the step -- rejection sampling keeps the walker where
// it was for the step, ERL draws a new direction (DIR and PERM call = the
// draw's index) until a step is admitted, at most kMaxLeaps draws.  MT adds
// absorbing membranes (Sec. 2.1.3, magnetization transfer; t.Tmt non-null).
// RK: draw with the round keys of ctl.rk, computed once on the host (no key
// schedule per draw: 2.4 % faster on the FP32 step); otherwise advance the
// key from ctl.seed in every draw (the batched kernel, whose request
// descriptors sit in shared memory).
template <typename Real, int NS, bool HASH, int IM, bool MT, bool RK = false>
__device__ __forceinline__ void walk_block(const Geometry &g, const Tables<Real> &t, const WalkerState<Real> &st,
                                           const RunCtl &ctl, int64_t block, int64_t k_begin, int64_t k_end)
{
    constexpr bool kF64 = std::is_same<Real, double>::value;
    __shared__ int32_t s_cancel;
    __shared__ double s_red[kWalkWarps][kMoments];
    if (threadIdx.x == 0) s_cancel = ctl.cancel ? *ctl.cancel : 0;
    __syncthreads();
    if (s_cancel) return;

    // the round keys, loop-invariant and warp-uniform: read once here (read
    // from the launch parameters inside the step loop they took 16 constant
    // loads per warp-step; hoisted, the step is 1.3 % faster)
    uint32_t rk[kRoundKeys];
#pragma unroll
    for (int i = 0; i < kRoundKeys; ++i) rk[i] = ctl.rk[i];
    const int64_t li = block * kWalkBlock + threadIdx.x;
    const bool active = li < ctl.n_walkers;
    // the walker in this slot: its id picks its random streams (RMS_MORTON
    // runs keep walkers in Morton order of their voxel, not in id order)
    const uint64_t w = (uint64_t)(ctl.w_begin + ((active && st.wid) ? (int64_t)st.wid[li] : li));
    const int32_t N[3] = {g.nx, g.ny, g.nz};
    const int32_t stride[3] = {1, g.nx, g.nx * g.ny};
    const int32_t per[3] = {g.per_x, g.per_y, g.per_z};
    const int32_t L = t.n_labels;
    // voxel edge in the form's precision (the single-precision value comes from
    // the host: a conversion here would run on the FP64 pipe at every step)
    Real lp;
    if constexpr (kF64)
        lp = g.voxel_um;
    else
        lp = g.voxel_f;

    Real o[3], o0[3];
    int32_t di[3], wc[3];
    int32_t v = 0, c = 0;
    Real A = Real(0), Ac = Real(0);
    Real ph[NS][3], phc[NS][3];
    uint64_t h = 0;
    // face events, crossings into another label, reflections (verification kernel)
    [[maybe_unused]] int32_t nev = 0, ncr = 0, nrf = 0;
    if (active) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = st.o[a][li];
            o0[a] = st.o0[a][li];
            di[a] = st.di[a][li];
            int32_t q = (st.i0[a][li] + di[a]) % N[a];
            wc[a] = q < 0 ? q + N[a] : q;
        }
        v = wc[0] + stride[1] * wc[1] + stride[2] * wc[2];
        c = st.c[li];
        A = st.A[li];
        if (!kF64) Ac = st.A_c[li];
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ph[s][a] = s < ctl.n_shapes ? st.phase[((int64_t)s * 3 + a) * ctl.n_walkers + li] : Real(0);
                phc[s][a] = (!kF64 && s < ctl.n_shapes)
                                ? st.phase_c[((int64_t)s * 3 + a) * ctl.n_walkers + li]
                                : Real(0);
            }
        if (HASH) h = st.hash[li];
        if constexpr (HASH) {
            if (st.counts) {
                nev = st.counts[li];
                ncr = st.counts[ctl.n_walkers + li];
                nrf = st.counts[2 * ctl.n_walkers + li];
            }
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = o0[a] = Real(0);
            di[a] = wc[a] = 0;
        }
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) ph[s][a] = phc[s][a] = Real(0);
    }

    // a 32-bit step counter (n_steps <= 2e9): uniform 32-bit arithmetic per
    // step (measured 0.8 % faster than 64-bit on the FP32 step)
    for (int32_t k = (int32_t)k_begin + 1; k <= (int32_t)k_end; ++k) {
        const uint8_t fl = __ldg(t.flags + (k - 1));
        if (active) {
            const int mode = t.mode ? (int)__ldg(t.mode + (k - 1)) : 0;
            // state at the step start, restored when a membrane refuses the step
            [[maybe_unused]] Real o_s[3], A_s, Ac_s;
            [[maybe_unused]] int32_t wc_s[3], di_s[3], v_s, c_s, nev_s, ncr_s, nrf_s;
            if constexpr (IM != kInteractEC) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o_s[a] = o[a];
                    wc_s[a] = wc[a];
                    di_s[a] = di[a];
                }
                v_s = v;
                c_s = c;
                A_s = A;
                Ac_s = Ac;
                if constexpr (HASH) {
                    nev_s = nev;
                    ncr_s = ncr;
                    nrf_s = nrf;
                }
            }
            uint32_t att = 0;  // draw index (ERL redraws); always 0 otherwise
            [[maybe_unused]] bool sat_any = false;  // saturated on some draw of this step (MT)
#pragma unroll 1
            for (;;) {
            // ---- direction (one DIR call: words 0, 1 -> direction; words 2, 3 ->
            //      the Bernoulli words of the step's first two membrane events)
            U4 x;
            if constexpr (RK)
                x = philox4x32_10_rk(U4{(uint32_t)w, (uint32_t)(w >> 32), (uint32_t)k, (kTagDir << 16) | att}, rk);
            else
                x = draw(ctl.seed, w, (uint32_t)k, kTagDir, att);
            Real n[3];
            direction_from(x.x, x.y, t.trig, n);
            // ---- face walk (Sec. 2.2 items 3-4)
            Real sc = __ldg(t.s + c);
            Real rate = t.any_relax ? __ldg(t.dtR + mode * L + c) : Real(0);
            [[maybe_unused]] const Real rate0 = rate;
            Real d[3] = {mulr(n[0], sc), mulr(n[1], sc), mulr(n[2], sc)};
            [[maybe_unused]] bool refused = false;
            // A face event on axis `best` moving up/down: look up the voxel across
            // it and decide between crossing and reflection.
            auto face = [&](int best, bool up, int ev) -> bool {
                int32_t coord = 0, Nb = 1, sb = 1, pb = 1;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (a == best) {
                        coord = wc[a];
                        Nb = N[a];
                        sb = stride[a];
                        pb = per[a];
                    }
                int32_t nc, nv;
                bool wall = false;
                if (up) {
                    nc = coord + 1;
                    nv = v + sb;
                    if (nc == Nb) {
                        wall = !pb;
                        nc = 0;
                        nv = v - (Nb - 1) * sb;
                    }
                } else {
                    nc = coord - 1;
                    nv = v - sb;
                    if (coord == 0) {
                        wall = !pb;
                        nc = Nb - 1;
                        nv = v + (Nb - 1) * sb;
                    }
                }
                const int32_t c2 = wall ? -1 : (int32_t)__ldg(g.labels + nv);
                // magnetization transfer (Sec. 2.1.3): meeting an absorbing membrane
                // saturates the walker with probability P_MT -- word `ev` of the
                // step's MT call (call = the draw index)
                if constexpr (MT) {
                    if (c2 >= 0 && c2 != c) {
                        const uint32_t tm = __ldg(t.Tmt + (int64_t)c * L + c2);
                        if (tm != 0u && !saturated(A)) {
                            const U4 m = draw(ctl.seed, w, (uint32_t)k, kTagMT, att);
                            if ((ev == 0 ? m.x : (ev == 1 ? m.y : m.z)) < tm) saturate(A, Ac);
                        }
                    }
                }
                bool cross;
                if (c2 == c) {
                    cross = true;
                } else if (c2 < 0) {
                    cross = false;
                } else {
                    const uint32_t T = __ldg(t.T + (int64_t)c * L + c2);
                    if (T == 0u) {
                        cross = false;
                    } else {
                        // third membrane event of a step: word 0 of the step's PERM call
                        const uint32_t word =
                            ev == 0 ? x.z : (ev == 1 ? x.w : perm_word(ctl.seed, w, (uint32_t)k, att));
                        cross = word < T;
                    }
                }
                if (cross) {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (a == best) {
                            wc[a] = nc;
                            di[a] += up ? 1 : -1;
                            o[a] = up ? Real(0) : Real(1);
                        }
                    v = nv;
                    if (c2 != c) {
                        if constexpr (HASH) ++ncr;
                        c = c2;
                        if (t.any_relax) rate = __ldg(t.dtR + mode * L + c);
                        return true;  // the caller switches to the new label's step length
                    }
                } else if constexpr (IM != kInteractEC) {
                    refused = true;
                } else {
                    if constexpr (HASH) ++nrf;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (a == best) {
                            n[a] = -n[a];
                            d[a] = -d[a];
                        }
                }
                return false;
            };
            // Face times from the step start: axis a meets its face at T[a] = dist/|d_a|
            // (beyond the step when >= 1); events are taken in time order (ties to the
            // lower axis), an axis meets at most one face per step (s_c < 1: the corner
            // reflector), and a crossing into a label of another step length
            // recomputes the remaining times from the current positions.
            if constexpr (kF64) {
                // Plain form: the CPU FP64 reference's operation order; comparisons on the
                // integer ALU (dgt0/dlt_nn/dclamp01 give the IEEE results).
                const double kInf = __longlong_as_double(0x7FF0000000000000LL);
                // one division per axis: (1 - o)/d moving up, o/(-d) moving down, on the
                // integer ALU (the IEEE quotient; the hardware division only for operands
                // outside its range, e.g. o = -0)
                double T[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double num = dgt0(d[a]) ? 1.0 - o[a] : o[a];
                    const double den = __longlong_as_double(dbits(d[a]) & 0x7FFFFFFFFFFFFFFFLL);  // |d|
                    T[a] = (dgt0(d[a]) || dlt0(d[a])) ? ddiv_nn(num, den) : kInf;
                }
                double tau = 0.0;
                // not unrolled in the plain form: its event pass carries the integer-ALU
                // arithmetic (and the rare re-timing after a change of step length, with
                // three divisions); three copies of it measured 7 % slower, from
                // instruction fetch
#pragma unroll 1
                for (int ev = 0; ev < 3; ++ev) {
                    int best = 0;
                    double tmin = T[0];
                    if (dlt_nn(T[1], tmin)) {
                        best = 1;
                        tmin = T[1];
                    }
                    if (dlt_nn(T[2], tmin)) {
                        best = 2;
                        tmin = T[2];
                    }
                    if (!dlt_nn(tmin, 1.0)) break;
                    const double dts = tmin - tau;
                    bool up = false;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (a == best) {
                            up = dgt0(d[a]);
                            o[a] = up ? 1.0 : 0.0;
                            T[a] = kInf;
                        } else {
                            o[a] = dclamp01(o[a] + dmul(dts, d[a]));
                        }
                    }
                    if (t.any_relax) A = A + dmul(dts, rate);
                    tau = tmin;
                    if constexpr (HASH) ++nev;
                    const bool changed = face(best, up, ev);
                    if constexpr (IM != kInteractEC) {
                        if (refused) break;
                    }
                    if (changed) {
                        const double sn = __ldg(t.s + c);
                        if (dbits(sn) != dbits(sc)) {
                            sc = sn;
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                d[a] = dmul(n[a], sc);
                                if (dbits(T[a]) == 0x7FF0000000000000LL) continue;
                                const double num = dgt0(d[a]) ? 1.0 - o[a] : o[a];
                                T[a] = tau + ddiv_nn(num, __longlong_as_double(dbits(d[a]) & 0x7FFFFFFFFFFFFFFFLL));
                            }
                        }
                    }
                }
                if (IM == kInteractEC || !refused) {
                    const double rem = 1.0 - tau;
#pragma unroll
                    for (int a = 0; a < 3; ++a) o[a] = dclamp01(o[a] + dmul(rem, d[a]));
                    if (t.any_relax) A = A + dmul(rem, rate);
                }
            } else {
                // Precision form: the same walk in FP32 (approximate division).
                constexpr Real kNever = Real(1e30);
                Real T[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const Real ad = fabsf(d[a]);
                    const Real dist = d[a] > Real(0) ? Real(1) - o[a] : o[a];
                    T[a] = ad > Real(0) ? fminf(__fdividef(dist, ad), kNever) : kNever;
                }
                Real tau = Real(0);
#pragma unroll  // unrolled: each event index is a constant (measured 5 % faster, FP32)
                for (int ev = 0; ev < 3; ++ev) {
                    int best = 0;
                    Real tmin = T[0];
                    if (T[1] < tmin) {
                        best = 1;
                        tmin = T[1];
                    }
                    if (T[2] < tmin) {
                        best = 2;
                        tmin = T[2];
                    }
                    if (!(tmin < Real(1))) break;
                    tmin = fmaxf(tmin, tau);
                    const Real dtt = tmin - tau;
                    bool up = false;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (a == best) {
                            up = d[a] > Real(0);
                            o[a] = up ? Real(1) : Real(0);
                            T[a] = kNever;
                        } else {
                            o[a] = clamp01(o[a] + dtt * d[a]);
                        }
                    }
                    if (t.any_relax) kahan_add(A, Ac, dtt * rate);
                    tau = tmin;
                    if constexpr (HASH) ++nev;
                    const bool changed = face(best, up, ev);
                    if constexpr (IM != kInteractEC) {
                        if (refused) break;
                    }
                    if (changed) {
                        const Real sn = __ldg(t.s + c);
                        if (sn != sc) {
                            sc = sn;
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                d[a] = n[a] * sc;
                                if (!(T[a] < kNever)) continue;
                                const Real dist = d[a] > Real(0) ? Real(1) - o[a] : o[a];
                                T[a] = tau + __fdividef(dist, fabsf(d[a]));
                            }
                        }
                    }
                }
                if (IM == kInteractEC || !refused) {
                    const Real rem = Real(1) - tau;
#pragma unroll
                    for (int a = 0; a < 3; ++a) o[a] = clamp01(o[a] + rem * d[a]);
                    if (t.any_relax) kahan_add(A, Ac, rem * rate);
                }
            }
            if constexpr (IM == kInteractEC) {
                break;
            } else {
                if (!refused) break;
                if constexpr (MT) sat_any = sat_any || saturated(A);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o[a] = o_s[a];
                    wc[a] = wc_s[a];
                    di[a] = di_s[a];
                }
                v = v_s;
                c = c_s;
                A = A_s;
                Ac = Ac_s;
                if constexpr (HASH) {
                    nev = nev_s;
                    ncr = ncr_s;
                    nrf = nrf_s;
                }
                if constexpr (MT) {
                    if (sat_any) saturate(A, Ac);  // a saturation met on a cancelled draw stays
                }
                if (IM == kInteractRS || ++att >= kMaxLeaps) {
                    // the walker stays for the step, in its label
                    if (t.any_relax) {
                        if constexpr (kF64)
                            A = A + rate0;
                        else
                            kahan_add(A, Ac, rate0);
                    }
                    if (IM == kInteractERL) atomicOr(ctl.status, kWarnLeaps);
                    if constexpr (HASH) ++nrf;
                    break;
                }
            }
            }  // draws
            if (HASH) {  // the verification kernel: checksum and, on request, invariants
                const uint64_t x = (((uint64_t)k & 0xFFFFu) << 48) ^ ((uint64_t)(uint32_t)c << 32) ^
                                   (uint64_t)(uint32_t)v;
                h = mix64(h ^ x);
                if (ctl.checked) {
                    bool bad = false;
#pragma unroll
                    for (int a = 0; a < 3; ++a) bad = bad || wc[a] < 0 || wc[a] >= N[a];
                    bad = bad || v != wc[0] + stride[1] * wc[1] + stride[2] * wc[2];
                    if (!bad) bad = (int32_t)__ldg(g.labels + v) != c;  // indices checked first
#pragma unroll
                    for (int a = 0; a < 3; ++a) bad = bad || !(o[a] >= Real(0) && o[a] <= Real(1));
                    if (bad) atomicOr(ctl.status, kErrInvariant);
                }
            }
            // ---- phase (Eq. 7, right end point of each step)
            if (fl & 1u) {
                Real dx[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    dx[a] = mulr(lp, (Real)di[a] + (o[a] - o0[a]));
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    if (s < ctl.n_shapes) {
                        const Real wg = __ldg(t.wG + (int64_t)s * ctl.n_steps + (k - 1));
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            if (kF64)
                                ph[s][a] = ph[s][a] + dmul(wg, dx[a]);
                            else
                                kahan_add(ph[s][a], phc[s][a], wg * dx[a]);
                        }
                    }
                }
            }
        }
        // ---- displacement moments at recording steps (block-uniform branch)
        if (fl & 2u) {
            double dx[3] = {0.0, 0.0, 0.0};
            double al = 0.0;
            if (active) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    dx[a] = g.voxel_um * ((double)di[a] + ((double)o[a] - (double)o0[a]));
                al = kF64 ? exp(-(double)A) : exp(-((double)A - (double)Ac));
            }
            warp_moments(al, dx, s_red[threadIdx.x >> 5]);
            __syncthreads();
            if (threadIdx.x < kMoments) {
                double acc = 0.0;
#pragma unroll
                for (int ww = 0; ww < kWalkWarps; ++ww) acc += s_red[ww][threadIdx.x];
                const int32_t r = __ldg(t.rec_of + (k - 1));
                ctl.mom_partial[((int64_t)r * ctl.n_blocks + block) * kMoments + threadIdx.x] = acc;
            }
            __syncthreads();
        }
    }

    if (active) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            st.o[a][li] = o[a];
            st.di[a][li] = di[a];
        }
        st.c[li] = c;
        st.A[li] = A;
        if (!kF64) st.A_c[li] = Ac;
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (s < ctl.n_shapes)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    st.phase[((int64_t)s * 3 + a) * ctl.n_walkers + li] = ph[s][a];
                    if (!kF64) st.phase_c[((int64_t)s * 3 + a) * ctl.n_walkers + li] = phc[s][a];
                }
        if (HASH) st.hash[li] = h;
        if constexpr (HASH) {
            if (st.counts) {
                st.counts[li] = nev;
                st.counts[ctl.n_walkers + li] = ncr;
                st.counts[2 * ctl.n_walkers + li] = nrf;
            }
        }
    }
}

// Resident blocks per SM the register allocation must allow (0: no bound,
// the compiler's choice).  The plain form's one-shape kernel: its integer-ALU
// arithmetic is made of long dependent chains, whose latency more warps hide,
// and 5 blocks (at most 102 registers) measured 6 % faster than the
// unconstrained 4.  The FP32 form's one-shape elastic-collision kernel: 9
// blocks (56 registers, no spills; 36 warps per SM), 2.5 % faster than 7
// blocks (72 registers) and 7.5 % faster than the compiler's own choice (80
// registers, 6 blocks); 10 blocks spill.  The RS/ERL and absorbing-membrane
// kernels would spill under such bounds, and kernels with more shapes keep
// the registers their phases need.
template <typename Real, int NS, bool HASH, int IM, bool MT>
constexpr int kWalkMinBlocks = (NS != 1) ? 0
                               : std::is_same<Real, double>::value ? 5
                               : (IM != kInteractEC || MT) ? 0
                               : HASH ? 7 : 9;  // the verification kernel would spill at 9

// One run: block b of the grid advances walkers b*kWalkBlock ... of the run.
template <typename Real, int NS, bool HASH, int IM, bool MT>
__global__ void __launch_bounds__(kWalkBlock, kWalkMinBlocks<Real, NS, HASH, IM, MT>)
walk_kernel(Geometry g, Tables<Real> t, WalkerState<Real> st, RunCtl ctl, int64_t k_begin, int64_t k_end)
{
    walk_block<Real, NS, HASH, IM, MT, true>(g, t, st, ctl, blockIdx.x, k_begin, k_end);
}

// Many runs in one launch (continuous batching): block i executes task i --
// a block of walkers of one request for that request's next steps.  The
// request descriptors and the task table are read once per block.
template <typename Real, int NS>
__global__ void __launch_bounds__(kWalkBlock, (std::is_same<Real, float>::value && NS <= 2) ? 8 : 4)
walk_batched_kernel(const ReqDesc<Real> *reqs, const BlockTask *tasks, int32_t n_tasks)
{
    if ((int32_t)blockIdx.x >= n_tasks) return;
    __shared__ ReqDesc<Real> s_req;
    __shared__ BlockTask s_task;
    if (threadIdx.x == 0) {
        s_task = tasks[blockIdx.x];
        s_req = reqs[s_task.req];
    }
    __syncthreads();
    walk_block<Real, NS, false, kInteractEC, false>(s_req.g, s_req.t, s_req.st, s_req.ctl, s_task.block,
                                                    s_task.k0, s_task.k1);
}

template <typename Real>
cudaError_t launch_walk_batched(int ns_bucket, int32_t n_tasks, cudaStream_t stream, const ReqDesc<Real> *reqs,
                                const BlockTask *tasks)
{
    if (n_tasks <= 0) return cudaSuccess;
    const dim3 grid((unsigned)n_tasks);
    if (ns_bucket <= 1)
        walk_batched_kernel<Real, 1><<<grid, kWalkBlock, 0, stream>>>(reqs, tasks, n_tasks);
    else if (ns_bucket <= 2)
        walk_batched_kernel<Real, 2><<<grid, kWalkBlock, 0, stream>>>(reqs, tasks, n_tasks);
    else if (ns_bucket <= 4)
        walk_batched_kernel<Real, 4><<<grid, kWalkBlock, 0, stream>>>(reqs, tasks, n_tasks);
    else
        walk_batched_kernel<Real, 8><<<grid, kWalkBlock, 0, stream>>>(reqs, tasks, n_tasks);
    return cudaGetLastError();
}

// Resident blocks per SM of the batched kernel (the serving scheduler's
// count of block slots).
template <typename Real>
int batched_blocks_per_sm(int ns_bucket)
{
    int n = 0;
    cudaError_t e;
    if (ns_bucket <= 1)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_batched_kernel<Real, 1>, kWalkBlock, 0);
    else if (ns_bucket <= 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_batched_kernel<Real, 2>, kWalkBlock, 0);
    else if (ns_bucket <= 4)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_batched_kernel<Real, 4>, kWalkBlock, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, walk_batched_kernel<Real, 8>, kWalkBlock, 0);
    return e == cudaSuccess && n > 0 ? n : 1;
}

// Host-side launcher for interaction IM and absorbing membranes MT,
// instantiated in walk_fp64.cu / walk_fp32.cu (elastic collision),
// walk_reject_fp64.cu / walk_reject_fp32.cu (rejection sampling, ERL) and
// walk_mt_fp64.cu / walk_mt_fp32.cu (the three with absorbing membranes).
template <typename Real, int IM, bool MT>
cudaError_t launch_walk(int n_shapes, bool hash, dim3 grid, cudaStream_t stream, const Geometry &g,
                        const Tables<Real> &t, const WalkerState<Real> &st, const RunCtl &ctl,
                        int64_t k_begin, int64_t k_end)
{
#define RMS_LAUNCH(NSV)                                                                              \
    do {                                                                                             \
        if (hash)                                                                                    \
            walk_kernel<Real, NSV, true, IM, MT><<<grid, kWalkBlock, 0, stream>>>(g, t, st, ctl,     \
                                                                                 k_begin, k_end);    \
        else                                                                                         \
            walk_kernel<Real, NSV, false, IM, MT><<<grid, kWalkBlock, 0, stream>>>(g, t, st, ctl,    \
                                                                                  k_begin, k_end);   \
    } while (0)
    if (n_shapes <= 1)
        RMS_LAUNCH(1);
    else if (n_shapes <= 2)
        RMS_LAUNCH(2);
    else if (n_shapes <= 4)
        RMS_LAUNCH(4);
    else
        RMS_LAUNCH(8);
#undef RMS_LAUNCH
    return cudaGetLastError();
}

}  // namespace rms
