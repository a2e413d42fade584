// rms_device.cuh -- device-side building blocks shared by the library's own
// translation units: the counter-based generator, the checksum mixer and the
// parameter blocks handed to the kernels.
#pragma once

#include <cstdint>

namespace rms {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; in each,
// the even words are multiplied by the two round multipliers, the high
// halves are XOR-ed with the odd words and the key, and the key advances by
// the two Weyl increments between rounds.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same generator with the ten rounds' keys given: rk[2r], rk[2r + 1] =
// the key after r Weyl increments (round_keys below).  The step kernel reads
// them from its launch parameters, where they cost no instruction per draw.
constexpr int kRoundKeys = 20;

__device__ __forceinline__ U4 philox4x32_10_rk(U4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0};
    }
    return c;
}

__host__ __device__ inline void round_keys(uint64_t seed, uint32_t *rk)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Counter layout: key (seed_lo, seed_hi); counter (walker_lo, walker_hi,
// step, tag << 16 | call).
enum : uint32_t { kTagInit = 1u, kTagDir = 2u, kTagPerm = 3u, kTagMT = 4u };

__device__ __forceinline__ U4 draw(uint64_t seed, uint64_t w, uint32_t step, uint32_t tag,
                                   uint32_t call)
{
    return philox4x32_10(U4{(uint32_t)w, (uint32_t)(w >> 32), step, (tag << 16) | call},
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

// (x + 1/2) 2^-32: uniform in (0,1), exact in FP64.
__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

// sin and cos on [0, pi/4] by Taylor polynomials (degree 17 / 16, truncation
// below 1e-18), separate multiplies and adds.  Used to fill the azimuth table.
__device__ __forceinline__ void poly_sincos(double th, double &sn, double &cs)
{
    const double t = th * th;
    double ps = 1.0 / 355687428096000.0;
    ps = -1.0 / 1307674368000.0 + t * ps;
    ps = 1.0 / 6227020800.0 + t * ps;
    ps = -1.0 / 39916800.0 + t * ps;
    ps = 1.0 / 362880.0 + t * ps;
    ps = -1.0 / 5040.0 + t * ps;
    ps = 1.0 / 120.0 + t * ps;
    ps = -1.0 / 6.0 + t * ps;
    sn = th + (th * t) * ps;
    double pc = 1.0 / 20922789888000.0;
    pc = -1.0 / 87178291200.0 + t * pc;
    pc = 1.0 / 479001600.0 + t * pc;
    pc = -1.0 / 3628800.0 + t * pc;
    pc = 1.0 / 40320.0 + t * pc;
    pc = -1.0 / 720.0 + t * pc;
    pc = 1.0 / 24.0 + t * pc;
    pc = -1.0 / 2.0 + t * pc;
    cs = 1.0 + t * pc;
}

constexpr int kTrigParts = 1024;  // parts of the octant [0, pi/4] in the azimuth table

// SplitMix64 finaliser (Steele, Lea & Flood 2014), the trajectory checksum.
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

constexpr int kMoments = 22;  // alpha, 6 second-order, 15 fourth-order terms
constexpr int kMaxShapes = 8;

// Device status bits: errors, and one warning (an ERL step that found no
// admissible direction in kMaxLeaps draws; the walker stayed for that step).
enum : int { kErrTimeout = 4, kWarnLeaps = 8, kErrInit = 16, kErrInvariant = 32, kErrOrder = 64 };
constexpr uint32_t kMaxInit = 4096;  // start draws per walker (spin concentrations)

// A saturated walker (Sec. 2.1.3, magnetization transfer) has weight 0 for
// good.  The FP64 form keeps A = +inf, as the CPU reference does; the FP32
// form keeps A = kSaturatedF (its Kahan sum would turn +inf into NaN), which
// the walker export turns into +inf.
constexpr float kSaturatedF = 1e30f;

// Particle-membrane interaction (Sec. 2.1.2, App. A and B).
enum : int { kInteractEC = 0, kInteractRS = 1, kInteractERL = 2 };
constexpr uint32_t kMaxLeaps = 64;  // ERL draws per step

// Walker state, structure of arrays, one entry per walker.
template <typename Real>
struct WalkerState {
    Real *o[3];        // offset inside the voxel, [0,1]
    Real *o0[3];       // initial offset
    int32_t *i0[3];    // initial voxel (wrapped coordinates)
    int32_t *di[3];    // unwrapped voxel displacement i - i0
    int32_t *c;        // current label
    Real *A;           // relaxation exponent (FP32 form: Kahan sum with A_c)
    Real *A_c;         // Kahan compensation (FP32 form only)
    Real *phase;       // [shape][axis][W]
    Real *phase_c;     // Kahan compensation (FP32 form only), same layout
    uint64_t *hash;
    int32_t *counts;   // [3][W]: face events, crossings, reflections (RMS_COUNTS) or nullptr
    int32_t *wid;      // walker (relative to the run's first) in each slot, or nullptr: the slot's index
};

struct Geometry {
    const uint16_t *labels;
    int32_t nx, ny, nz;
    int32_t per_x, per_y, per_z;
    double voxel_um;
    float voxel_f;  // voxel_um rounded to single precision (the FP32 form's phase)
};

template <typename Real>
struct Tables {
    const Real *s;          // step length per label, voxel units
    const Real *dtR;        // [mode][label]: dt / T (0 = none)
    const uint32_t *T;      // [from][to] Bernoulli thresholds
    const uint32_t *Tmt;    // [from][to] saturation thresholds (MT), or nullptr
    int32_t n_labels;
    const Real *wG;         // [shape][step]: dt * G
    const uint8_t *flags;   // [step]: bit0 any G != 0, bit1 recording step
    const int32_t *rec_of;  // [step]: recording index or -1
    const uint8_t *mode;    // [step] relaxation mode (or nullptr = 0)
    int32_t any_relax;
    const double *trig;     // [part][cos, sin] of the azimuth table (FP64 form)
};

struct RunCtl {
    uint64_t seed;
    int64_t w_begin;
    int64_t n_walkers;
    int64_t n_steps;
    int32_t n_shapes;
    int32_t n_rec;
    int32_t *status;                // device error bits
    int32_t checked;                // verify the walker invariants every step (verification kernel)
    const volatile int32_t *cancel; // host-mapped cancel flag (nullptr = none)
    double *mom_partial;            // [rec][block][22]
    int32_t n_blocks;
    uint32_t rk[kRoundKeys];        // Philox round keys of seed (round_keys)
};

// One request of a batched launch: everything the walk needs.
template <typename Real>
struct ReqDesc {
    Geometry g;
    Tables<Real> t;
    WalkerState<Real> st;
    RunCtl ctl;
};

// One block of a batched launch: block `block` of request `req`, steps (k0, k1].
struct BlockTask {
    int32_t req;
    int32_t pad;
    int64_t block;
    int64_t k0, k1;
};

}  // namespace rms
