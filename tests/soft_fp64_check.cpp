// Host check of the integer-ALU FP64 division, square root and product
// (paper_2012_06478_gb300/csrc/soft_fp64.cuh) against the host's IEEE
// operations, built with -ffp-contract=off.  Classes: random operands over
// the whole normal range and over the ranges of the walker step, quotients
// and roots within one unit of the rounding midpoint, products with exact
// ties, powers of two and extreme mantissas, perfect squares and their
// neighbours; the unchecked product and root agree with the checked ones
// wherever the checks pass.  Prints the number of cases compared and of
// mismatches; exit status 1 on a mismatch.
#include "../paper_2012_06478_gb300/csrc/soft_fp64.cuh"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

using namespace rms::sfp;
typedef unsigned __int128 u128;

static long g_tested = 0, g_bad = 0, g_fallback = 0;

static void check_div(double a, double b)
{
    double q;
    if (!div_pos(a, b, q)) {
        ++g_fallback;
        return;
    }
    ++g_tested;
    const double r = a / b;
    if (bits_of(q) != bits_of(r)) {
        if (g_bad < 10) std::printf("div %a / %a = %a, IEEE %a\n", a, b, q, r);
        ++g_bad;
    }
}

static void check_sqrt(double x)
{
    double s;
    if (!sqrt_pos(x, s)) {
        ++g_fallback;
        return;
    }
    ++g_tested;
    if (bits_of(sqrt_normal(x)) != bits_of(s)) {
        if (g_bad < 10) std::printf("sqrt_normal %a differs from sqrt_pos\n", x);
        ++g_bad;
    }
    const double r = std::sqrt(x);
    if (bits_of(s) != bits_of(r)) {
        if (g_bad < 10) std::printf("sqrt %a = %a, IEEE %a\n", x, s, r);
        ++g_bad;
    }
}

static void check_mul(double a, double b)
{
    double p;
    if (!mul_rn(a, b, p)) {
        ++g_fallback;
        return;
    }
    ++g_tested;
    if (bits_of(mul_normal(a, b)) != bits_of(p)) {  // the unchecked form, where the checks pass
        if (g_bad < 10) std::printf("mul_normal %a * %a differs from mul_rn\n", a, b);
        ++g_bad;
    }
    const double r = a * b;
    if (bits_of(p) != bits_of(r)) {
        if (g_bad < 10) std::printf("mul %a * %a = %a, IEEE %a\n", a, b, p, r);
        ++g_bad;
    }
}

static double make(uint64_t mant, int e) { return double_of(((uint64_t)e << 52) | (mant & kMant)); }
static double make_s(uint64_t mant, int e, uint64_t sign) { return double_of((sign << 63) | ((uint64_t)e << 52) | (mant & kMant)); }

int main(int argc, char **argv)
{
    const long n = argc > 1 ? std::atol(argv[1]) : 1000000;
    std::mt19937_64 g(argc > 2 ? std::strtoull(argv[2], nullptr, 10) : 12345);
    const uint64_t H = kHidden;
    for (long i = 0; i < n; ++i) {
        // random operands: any normal exponent; the walk's ranges (numerators in
        // [0, 1], step components of 1e-10 .. 1 voxel)
        check_div(make(g(), 1 + (int)(g() % 2046)), make(g(), 1 + (int)(g() % 2046)));
        check_div(make(g(), 990 + (int)(g() % 34)), make(g(), 990 + (int)(g() % 33)));
        check_sqrt(make(g(), 1 + (int)(g() % 2046)));
        check_sqrt(make(g(), 991 + (int)(g() % 33)));
        // quotients one unit around a rounding midpoint: A ~ (Q + 1/2) B / 2^52
        const uint64_t B = H | (g() & kMant), Q = H | (g() & kMant);
        const uint64_t A = (uint64_t)(((u128)(2 * Q + 1) * B) >> 53);
        for (int k = -1; k <= 1; ++k)
            if (A + k >= H && A + k < 2 * H) check_div(make(A + k, 1000 + (int)(g() % 40)), make(B, 1000 + (int)(g() % 40)));
        // powers of two, all-ones and seed-boundary mantissas
        const uint64_t sp[] = {H, H + 1, 2 * H - 1, H | (1ULL << 29), H | ((1ULL << 29) - 1), 2 * H - (1ULL << 29)};
        const uint64_t r = H | (g() & kMant);
        for (uint64_t s : sp) {
            check_div(make(r, 1023), make(s, 1022));
            check_div(make(s, 1022), make(r, 1023));
            check_div(make(s, 1023), make(s, 1023));
            check_sqrt(make(s, 1023));
            check_sqrt(make(s, 1022));
        }
        // square roots one unit around a rounding midpoint: X ~ (q + 1/2)^2
        const uint64_t q = H | (g() & kMant);
        const u128 X4 = (u128)(2 * q + 1) * (2 * q + 1);
        for (int odd = 0; odd < 2; ++odd) {
            const uint64_t M = (uint64_t)(X4 >> ((odd ? 53 : 52) + 2));
            for (int k = -1; k <= 1; ++k)
                if (M + k >= H && M + k < 2 * H) check_sqrt(make(M + k, odd ? 1022 : 1023));
        }
        // products: random signs and exponents; the walk's ranges; exact ties
        // (significands with few bits, so that the discarded part is exactly one half)
        check_mul(make_s(g(), 1 + (int)(g() % 2046), g() & 1), make_s(g(), 1 + (int)(g() % 2046), g() & 1));
        check_mul(make_s(g(), 980 + (int)(g() % 60), g() & 1), make_s(g(), 990 + (int)(g() % 40), g() & 1));
        {
            const uint64_t ma = H | ((g() & ((1ULL << 27) - 1)) << 25), mb = H | ((g() & ((1ULL << 27) - 1)) << 25);
            check_mul(make_s(ma, 1023, g() & 1), make_s(mb, 1023, g() & 1));
            check_mul(make_s(ma | 1, 1023, 0), make_s(mb | (1ULL << 25), 1022, 1));
        }
        check_mul(make(2 * H - 1, 1023), make(2 * H - 1, 1023));
        check_mul(make(H, 1023), make(r, 1000));
        check_mul(make(2 * H - 1, 2046), make(H, 1024));   // overflow by rounding or beyond: hardware
        check_mul(make(2 * H - 1, 1), make(H, 1022));      // underflow: hardware
        // perfect squares and their neighbours
        const uint64_t qq = (H >> 26) | (g() & ((1ULL << 26) - 1));
        const u128 sq = (u128)qq * qq;
        if (sq >= H && sq < 2 * H)
            for (int k = -1; k <= 1; ++k) check_sqrt(make((uint64_t)sq + k, 1023));
    }
    // the cases the functions hand back to the hardware
    double t;
    const bool zero_ok = div_pos(0.0, 0.5, t) && bits_of(t) == 0 && !mul_rn(0.0, 1.0, t) && !mul_rn(-1.0, -0.0, t) &&
                         !mul_rn(INFINITY, 1.0, t) && !mul_rn(0x1p-1040, 2.0, t) && !mul_rn(0x1p-600, 0x1p-500, t);
    const bool rejects = !div_pos(-0.0, 0.5, t) && !div_pos(0x1p-1040, 0.5, t) && !div_pos(1.0, 0x1p-1040, t) &&
                         !div_pos(INFINITY, 1.0, t) && !div_pos(1.0, NAN, t) && !div_pos(0x1p-1000, 0x1p+100, t) &&
                         !sqrt_pos(0.0, t) && !sqrt_pos(-1.0, t) && !sqrt_pos(0x1p-1050, t) && !sqrt_pos(INFINITY, t);
    std::printf("tested %ld mismatches %ld fallbacks %ld special %d\n", g_tested, g_bad, g_fallback,
                (int)(zero_ok && rejects));
    return (g_bad || !zero_ok || !rejects) ? 1 : 0;
}
