// soft_fp64.cuh -- correctly rounded FP64 division, square root and
// multiplication built on the integer ALU, bit-identical to IEEE 754
// round-to-nearest-even.
//
// Why: GB300's FP64 pipe issues about two operations per clock per SM, a
// sixty-fourth of its FP32 rate, and an FP64 division or square root is a
// sequence of several of them.  The plain FP64 form of the walker step keeps
// that pipe busy; computing its quotients and its square root with 64-bit
// integer arithmetic (multiplies on the integer pipe, a single-precision
// seed) gives the same bits at a fraction of the pipe time.
//
// Method: a reciprocal (or reciprocal square root) seed from single
// precision, refined by Newton-Raphson iterations in fixed point (for the
// reciprocal x' = x + x(1 - b x); for the square root q' = q + (X - q^2)/(2q)
// with 1/(2q) from the seed), then an exact integer remainder that fixes the
// last unit and decides the rounding -- the classical scheme of, e.g.,
// Muller et al., Handbook of Floating-Point Arithmetic (2nd ed., 2018),
// ch. 4 (Newton-Raphson based division and square root) with the final
// correction by the remainder.  Division and square root have no exact
// half-way cases, but the rounding rule is written out in full anyway.
//
// Each function handles the operands the walker step produces -- finite,
// normal, with a normal result -- and returns false for anything else, so
// the caller falls back to the hardware operation for zeros, subnormals,
// infinities, NaNs and out-of-range results.  Host and device share the
// code: the host build (for the host-side checks) replaces the two device
// intrinsics by their exact definitions.
#pragma once

#include <cstdint>
#include <cstring>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace rms {
namespace sfp {

constexpr uint64_t kMant = 0x000FFFFFFFFFFFFFULL;  // the 52 stored mantissa bits
constexpr uint64_t kHidden = 0x0010000000000000ULL;  // 2^52

__host__ __device__ __forceinline__ uint64_t bits_of(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}

__host__ __device__ __forceinline__ double double_of(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}

__host__ __device__ __forceinline__ uint32_t float_bits(float x)
{
#ifdef __CUDA_ARCH__
    return (uint32_t)__float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}

// high 64 bits of the 128-bit product a*b
__host__ __device__ __forceinline__ uint64_t mulhi(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// single-precision reciprocal and square root, correctly rounded on both sides
__host__ __device__ __forceinline__ float rcp_rn(float x)
{
#ifdef __CUDA_ARCH__
    return __frcp_rn(x);
#else
    return 1.0f / x;
#endif
}
__host__ __device__ __forceinline__ float sqrt_rn(float x)
{
#ifdef __CUDA_ARCH__
    return __fsqrt_rn(x);
#else
    return __builtin_sqrtf(x);
#endif
}

// floor(x * e / 2^64) rounded toward zero, x < 2^64 unsigned, e signed
__host__ __device__ __forceinline__ int64_t smulhi(uint64_t x, int64_t e)
{
    const uint64_t m = mulhi(x, e < 0 ? (uint64_t)(-e) : (uint64_t)e);
    return e < 0 ? -(int64_t)m : (int64_t)m;
}

// a / b for a >= +0 and b > +0 (sign bits clear).  Returns false when a or b
// is subnormal, infinite or NaN, or the quotient leaves the normal range
// (except an overflow to infinity by rounding, which is the IEEE result).
__host__ __device__ __forceinline__ bool div_pos(double a, double b, double &q)
{
    const uint64_t ua = bits_of(a), ub = bits_of(b);
    if (ua == 0) {  // 0 / b = +0
        q = 0.0;
        return true;
    }
    const int32_t ea = (int32_t)(ua >> 52), eb = (int32_t)(ub >> 52);
    if ((uint32_t)(ea - 1) >= 0x7FEu || (uint32_t)(eb - 1) >= 0x7FEu) return false;
    const uint64_t A = (ua & kMant) | kHidden, B = (ub & kMant) | kHidden;  // [2^52, 2^53)
    const bool ge = A >= B;
    const int32_t e = ea - eb + 1022 + (ge ? 1 : 0);  // biased exponent of the quotient
    if ((uint32_t)(e - 1) >= 0x7FEu) return false;
    // x ~ 2^115 / B in (2^62, 2^63]: seed from the single-precision reciprocal
    // of B's top 24 bits (relative error below 2^-22), exact as a shifted
    // integer; then two Newton steps x += x e / 2^115, e = 2^115 - B x
    const float fr = rcp_rn((float)(uint32_t)(B >> 29));  // in (2^-24, 2^-23]
    const uint32_t fb = float_bits(fr);
    uint64_t x = (uint64_t)((fb & 0x7FFFFFu) | 0x800000u) << ((fb >> 23) - 64u);  // fr 2^86
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t plo = B * x, phi = mulhi(B, x);  // B x < 2^116
        // e = 2^115 - B x as a 128-bit two's-complement (ehi, elo); |e| < 2^94
        const uint64_t elo = 0ULL - plo;
        const int64_t ehi = (int64_t)(0x0008000000000000ULL - phi - (plo != 0ULL ? 1ULL : 0ULL));
        const int64_t e51 = (int64_t)(((uint64_t)ehi << 13) | (elo >> 51));  // e / 2^51, |e51| < 2^43
        x += (uint64_t)smulhi(x, e51);
    }
    // Q = floor(A 2^s / B), s = 52 (A >= B) or 53: from (A 2^11) x / 2^(126 - s),
    // within one unit; the exact remainder fixes it
    const int s = ge ? 52 : 53;
    uint64_t Q = mulhi(A << 11, x) >> (ge ? 10 : 9);
    int64_t R = (int64_t)((A << s) - Q * B);  // exact: the true value lies in (-B, 2B)
    if (R < 0) {
        --Q;
        R += (int64_t)B;
    } else if (R >= (int64_t)B) {
        ++Q;
        R -= (int64_t)B;
    }
    // round to nearest, ties to even (no ties occur for a quotient): up iff
    // 2R > B, or 2R == B and Q odd
    const uint64_t up = ((uint64_t)R << 1) + (Q & 1ULL) > B ? 1ULL : 0ULL;
    q = double_of((((uint64_t)(e - 1)) << 52) + Q + up);  // Q carries the hidden bit; a carry moves into the exponent
    return true;
}

// The product of the significands of a and b rounded to 53 bits, given the
// biased exponent e of the result: the 106-bit product is exact in two words,
// brought to [2^105, 2^106) (doubled when below), so that the 53 kept bits
// and the 53 below them sit at fixed places; rounding is to nearest with ties
// to even (products do have ties).
__host__ __device__ __forceinline__ double mul_core(uint64_t ua, uint64_t ub, uint64_t lo, uint64_t hi, bool top,
                                                    int32_t e)
{
    const uint64_t hn = top ? hi : (hi << 1) | (lo >> 63);
    const uint64_t ln = top ? lo : lo << 1;
    const uint64_t M = (hn << 11) | (ln >> 53);  // in [2^52, 2^53)
    const uint64_t rem = ln & 0x001FFFFFFFFFFFFFULL;
    // up iff rem > 2^52, or rem == 2^52 and M odd
    const uint64_t up = rem + (M & 1ULL) > 0x0010000000000000ULL ? 1ULL : 0ULL;
    return double_of(((ua ^ ub) & 0x8000000000000000ULL) | ((((uint64_t)(e - 1)) << 52) + M + up));
}

// a * b, both finite, normal and of any sign, with a normal product
// (including an overflow to infinity by rounding).  Returns false for a zero,
// subnormal, infinite or NaN operand, or a product out of the normal range.
__host__ __device__ __forceinline__ bool mul_rn(double a, double b, double &p)
{
    const uint64_t ua = bits_of(a), ub = bits_of(b);
    const int32_t ea = (int32_t)((ua >> 52) & 0x7FFu), eb = (int32_t)((ub >> 52) & 0x7FFu);
    if ((uint32_t)(ea - 1) >= 0x7FEu || (uint32_t)(eb - 1) >= 0x7FEu) return false;
    const uint64_t A = (ua & kMant) | kHidden, B = (ub & kMant) | kHidden;
    const uint64_t lo = A * B, hi = mulhi(A, B);  // A B in [2^104, 2^106)
    const bool top = (hi >> 41) != 0ULL;          // A B >= 2^105
    const int32_t e = ea + eb - 1023 + (top ? 1 : 0);
    if ((uint32_t)(e - 1) >= 0x7FEu) return false;
    p = mul_core(ua, ub, lo, hi, top, e);
    return true;
}

// a * b for operands that are known to be normal, with a product known to be
// normal (the caller's ranges guarantee it): mul_rn without its checks.
__host__ __device__ __forceinline__ double mul_normal(double a, double b)
{
    const uint64_t ua = bits_of(a), ub = bits_of(b);
    const int32_t ea = (int32_t)((ua >> 52) & 0x7FFu), eb = (int32_t)((ub >> 52) & 0x7FFu);
    const uint64_t A = (ua & kMant) | kHidden, B = (ub & kMant) | kHidden;
    const uint64_t lo = A * B, hi = mulhi(A, B);
    const bool top = (hi >> 41) != 0ULL;
    return mul_core(ua, ub, lo, hi, top, ea + eb - 1023 + (top ? 1 : 0));
}

// sqrt(x) for an x known to be normal and positive (no checks).
__host__ __device__ __forceinline__ double sqrt_normal(double x)
{
    const uint64_t ux = bits_of(x);
    const int32_t ex = (int32_t)(ux >> 52);
    const uint64_t M = (ux & kMant) | kHidden;
    const int32_t E = ex - 1023;                        // x = M 2^(E - 52)
    const bool odd = (E & 1) != 0;
    // X = M 2^52 (E even) or M 2^53 (E odd): sqrt(x) = sqrt(X) 2^((E - odd)/2 - 52),
    // sqrt(X) in [2^52, 2^53).  X as 128 bits:
    const int sh = odd ? 53 : 52;
    const uint64_t Xlo = M << sh, Xhi = M >> (64 - sh);
    // seed: X 2^-80 = M 2^(sh - 80) in [2^24, 2^26); q ~ sqrt(X) = sqrtf(.) 2^40,
    // rq ~ 2^103 / sqrt(X) ~ 2^103 / q (for corrections D / (2 q))
    const float xf = (float)(uint32_t)(M >> (80 - sh));  // truncated: relative error < 2^-24
    const float sf = sqrt_rn(xf);                         // in [2^12, 2^13)
    const uint32_t sb = float_bits(sf);
    uint64_t q = (uint64_t)((sb & 0x7FFFFFu) | 0x800000u) << ((sb >> 23) - 110u);  // sf 2^40
    const float rf = rcp_rn(sf);                          // in (2^-13, 2^-12]
    const uint32_t rb = float_bits(rf);
    const uint64_t rq = (uint64_t)((rb & 0x7FFFFFu) | 0x800000u) << ((rb >> 23) - 87u);  // rf 2^63
    // two steps q += (X - q^2) / (2 q), the difference in 128 bits
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t slo = q * q, shi = mulhi(q, q);
        const uint64_t dlo = Xlo - slo;
        const int64_t dhi = (int64_t)(Xhi - shi - (Xlo < slo ? 1ULL : 0ULL));  // |X - q^2| < 2^87
        const int64_t d40 = (int64_t)(((uint64_t)dhi << 24) | (dlo >> 40));   // (X - q^2) / 2^40
        // (X - q^2)/(2q) = d40 2^40 / (2 q) ~ d40 rq 2^40 / 2^104 = d40 rq / 2^64
        q += (uint64_t)smulhi(rq, d40);
    }
    // exact remainder R = X - q^2 (mod 2^64; the true value is far inside);
    // bring q to floor(sqrt(X)): 0 <= R <= 2q
    int64_t R = (int64_t)(Xlo - q * q);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (R < 0) {
            R += (int64_t)(2 * q - 1);
            --q;
        } else if (R > (int64_t)(2 * q)) {
            R -= (int64_t)(2 * q + 1);
            ++q;
        }
    }
    // round to nearest: sqrt(X) >= q + 1/2 iff X - q^2 > q (no ties)
    const uint64_t up = (uint64_t)R > q ? 1ULL : 0ULL;
    const int32_t er = ((E - (odd ? 1 : 0)) >> 1) + 1023;
    return double_of((((uint64_t)(er - 1)) << 52) + q + up);
}

// sqrt(x) for a normal x > 0.  Returns false otherwise (zero, subnormal,
// negative, infinite or NaN x).
__host__ __device__ __forceinline__ bool sqrt_pos(double x, double &r)
{
    const int32_t ex = (int32_t)(bits_of(x) >> 52);
    if ((uint32_t)(ex - 1) >= 0x7FEu) return false;
    r = sqrt_normal(x);
    return true;
}

}  // namespace sfp
}  // namespace rms
