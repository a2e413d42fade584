/*
 * rms_oracle.c -- plain, slow, obviously-correct CPU FP64 reference walker.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle against which the CUDA
 * path is checked.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product path never calls it.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * What it computes (Lee, Fieremans & Novikov, "Realistic Microstructure
 * Simulator (RMS)", arXiv 2012.06478):
 *   - Sec. 2.2 item 1: walkers start uniformly over all non-dead voxels.
 *   - Sec. 2.2 items 2-4, Sec. 2.1.1 (corner reflector, Fig. 2): each step is a
 *     vector of length ds = sqrt(2 d D dt), d = 3 (Eq. 1), in a random
 *     direction; the walker moves through voxel faces, at most three face
 *     events per step.  A face between voxels of the same label is
 *     transparent; a face between different labels is crossed with the
 *     probability of Eq. 3 (finite-step corrected P_{1->2}) and otherwise
 *     reflected specularly (Sec. 2.1.3: elastic collision).
 *   - Sec. 2.1.4, Eq. 5: the weight alpha = exp(-sum_i t_i / T^(i)).
 *   - Sec. 2.3, Eq. 7: phase phi = int g(t).x(t) dt, S = <alpha e^{-i phi}>/<alpha>.
 *   - Sec. 2.3 (narrow-pulse D and K): alpha-weighted displacement moments.
 *   - Sec. 2.1.3 (magnetization transfer): a walker meeting a membrane of
 *     surface relaxivity rho is saturated with probability
 *     P_MT = rho ds C_3 / D0 and contributes nothing afterwards (alpha_rho = 0).
 *   - Sec. 2.1.2, App. A and B: two alternative particle-membrane interactions
 *     the paper analyses for their bias.  Rejection sampling cancels a step
 *     that a membrane refuses (the walker stays, the step's dt still counts
 *     for relaxation); the equal-step-length random leap (ERL) cancels it and
 *     draws a new direction until a step is admitted (at most 64 draws, then
 *     the walker stays and an error bit is set).
 *   - App. C.2-C.3: spin concentrations c per label -- the generalised Eq. 3
 *     with (c2/c1)^lambda factors and its finite-step correction, walkers
 *     starting with density proportional to c -- and Baxter's rule
 *     P_{1->2} = c2 sqrt(D2) / (c1 sqrt(D1)) (at most 1).
 *
 * The paper does not print its kernel; the step is taken here in the order
 * and notation of Sec. 2.2, with every point where the text is silent fixed
 * by an explicit reading (direction sampler, event tie-break, counter layout,
 * phase discretisation).  Each reading is stated at the place it is used.
 *
 * Arithmetic rules (so that a GPU path with the same readings can reproduce
 * every trajectory bit for bit): FP64 only, +,-,*,/,sqrt correctly rounded,
 * no FMA contraction (built with -ffp-contract=off), no transcendental
 * function on the trajectory (exp, cos, sin appear only in the readout).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11,
 * "Parallel random numbers: as easy as 1, 2, 3"), written here from that
 * definition.  Counter layout: key = (seed_lo, seed_hi);
 * ctr = (walker_lo, walker_hi, step, tag << 16 | call), tag INIT=1, DIR=2,
 * PERM=3, MT=4.  Trajectory checksum: SplitMix64 finaliser (Steele, Lea & Flood,
 * OOPSLA'14).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TAG_INIT 1u
#define TAG_DIR 2u
#define TAG_PERM 3u
#define TAG_MT 4u

/* error bits reported through rmso_run's return value */
#define RMSO_ERR_BAD_ARG 4
#define RMSO_ERR_OOM 8

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011, Sec. 4): ten rounds of the       */
/* S-box  (L0,R0,L1,R1) -> (hi(B*R1)^L1^k1, lo(B*R1), hi(A*R0)^L0^k0,   */
/* lo(A*R0)) with multipliers A=0xD2511F53, B=0xCD9E8D57 and the key    */
/* bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.*/
/* ------------------------------------------------------------------ */
void rmso_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Vector form for tests: out[4r..4r+3] = Philox(ctr[4r..], key[2r..]). */
void rmso_philox_many(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    for (int64_t r = 0; r < n; r++) rmso_philox4x32_10(ctr + 4 * r, key + 2 * r, out + 4 * r);
}

static void draw(uint64_t seed, uint64_t w, uint32_t step, uint32_t tag, uint32_t call, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)w, (uint32_t)(w >> 32), step, (tag << 16) | call};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    rmso_philox4x32_10(ctr, key, out);
}

/* uniform in (0,1): (x + 1/2) 2^-32, exact in FP64, never 0 or 1 */
static double u01(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

/* SplitMix64 finaliser */
uint64_t rmso_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ */
/* Inputs                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    /* substrate: Sec. 2.1.1, one uint16 label per isotropic voxel, x fastest */
    int32_t nx, ny, nz;
    double voxel_um;          /* l_p */
    int32_t periodic[3];
    const uint16_t *labels;
    int32_t n_labels;
    const double *D;          /* per label, um^2/ms */
    const double *T2;         /* per label, ms (INFINITY: no decay) */
    const double *T1;         /* per label, ms (INFINITY: no decay) */
    const double *kappa;      /* n_labels x n_labels, um/ms */
    const uint8_t *dead;      /* per label: 1 = no walker may start in or enter */
    /* sequence */
    double dt;                /* ms */
    int64_t n_steps;
    int32_t n_shapes;
    const double *G;          /* n_shapes x n_steps: unit-amplitude effective gradient */
    const uint8_t *mode;      /* n_steps (or NULL = all 0): 0 T2 weighting, 1 T1, 2 none */
    int32_t n_rec;
    const int64_t *rec_steps; /* increasing, in [1, n_steps] */
    /* run */
    uint64_t seed;
    int64_t w_begin, w_end;   /* global walker ids [w_begin, w_end) */
    int32_t n_threads;
    int32_t hash;             /* 1: keep the trajectory checksum */
    int32_t interaction;      /* 0 elastic collision (Sec. 2.1.2-2.1.3), 1 rejection sampling
                                 (App. B), 2 equal-step-length random leap (App. A) */
    const double *rho;        /* n_labels x n_labels surface relaxivity (um/ms) of the membrane met
                                 from label r (row) towards label c (column), or NULL: none */
    /* App. C.2-C.3: spin concentration and the permeation model */
    const double *conc;       /* per label spin concentration (> 0 where walkers live), or NULL: all 1 */
    double lambda;            /* exponent of (c2/c1) in the generalised Eq. 3, in [0,1] (the label of
                                 lower index is side 1); < 0: the lambda minimising alpha_lambda */
    int32_t perm_model;       /* 0 nominal kappa (Eq. 3 generalised), 1 Baxter (kappa > 0 only marks
                                 a permeable pair) */
} rmso_config;

#define RMSO_EC 0
#define RMSO_RS 1
#define RMSO_ERL 2
#define RMSO_MAX_LEAPS 64
#define RMSO_ERR_LEAPS 16 /* an ERL step found no admissible direction in RMSO_MAX_LEAPS draws */
#define RMSO_PERM_KAPPA 0
#define RMSO_PERM_BAXTER 1
#define RMSO_MAX_INIT 4096
#define RMSO_ERR_INIT 32  /* a walker found no accepted start in RMSO_MAX_INIT draws */

typedef struct {
    /* per walker, index = w - w_begin */
    int32_t *i;        /* 3 per walker, unwrapped voxel index */
    double *o;         /* 3 per walker, offset inside the voxel in [0,1] */
    int32_t *i0;       /* 3 per walker */
    double *o0;        /* 3 per walker */
    int32_t *c;        /* current label */
    double *A;         /* sum_i t_i / T^(i) (Eq. 5 exponent) */
    double *phase;     /* n_shapes x 3 per walker: sum_k dt G_k Delta x_k (um ms) */
    uint64_t *hash;
    int64_t *counts;   /* 3 per walker: face events, membrane crossings, reflections */
    /* reductions over walkers */
    double *moments;   /* n_rec x 22 (Neumaier sums) */
} rmso_output;

/* ------------------------------------------------------------------ */
/* Per-label and per-pair tables (set-up, FP64)                        */
/* ------------------------------------------------------------------ */
typedef struct {
    const rmso_config *cfg;
    double *s;        /* ds_c / l_p : step length of label c in voxel units */
    double *dtR[3];   /* dt / T2_c, dt / T1_c, 0 : relaxation per unit time fraction */
    uint32_t *T;      /* per ordered pair: floor(P_{c->c'} 2^32), clamped */
    uint32_t *Tmt;    /* per ordered pair: floor(P_MT 2^32), clamped (NULL: no absorbing membrane) */
    uint64_t *acc;    /* per label: start accepted iff word < acc (density ~ conc); NULL: always */
    int64_t n_ok;
    int64_t *ok_list; /* raster list of non-dead voxels (NULL if none dead) */
    int any_relax;
    int err;
} ctx;

/* Eq. 1 with d = 3: ds = sqrt((6 D) dt) */
double rmso_step_length(double D, double dt) { return sqrt((6.0 * D) * dt); }

/* Eq. 3, the finite-step corrected permeation probability from label 1
 * (D1, ds1) into label 2 (D2, ds2), with C_3 = 2/3 (Eq. 2b):
 *   P = (kappa ds1 C / D1) / (1 + (kappa/2)(ds1/D1 + ds2/D2) C).
 * Evaluation order fixed: num = ((kappa*ds1)/D1)*C;
 * den = 1 + ((kappa/2)*((ds1/D1)+(ds2/D2)))*C.                          */
double rmso_perm_prob(double kappa, double D1, double ds1, double D2, double ds2)
{
    const double C = 2.0 / 3.0;
    double num = ((kappa * ds1) / D1) * C;
    double den = 1.0 + ((kappa / 2.0) * ((ds1 / D1) + (ds2 / D2))) * C;
    return num / den;
}

/* App. C.2, the generalised Eq. 3 for spin concentrations c1 (side of the
 * walker, D1, ds1) and c2: with f12 = (c2/c1)^lambda12 and
 * f21 = (c1/c2)^lambda21, lambda21 = 1 - lambda12,
 *   P = (kappa ds1 C f12 / D1) / (1 + (kappa/2)(ds1 f12/D1 + ds2 f21/D2) C),
 * which keeps P12/P21 = c2 sqrt(D2) / (c1 sqrt(D1)) (equilibrium density ratio
 * c1/c2) and applies the finite-step correction kappa = kappa0/(1 - alpha_lambda).
 * Evaluation order fixed as written; f = 1 gives rmso_perm_prob's bits. */
double rmso_perm_prob_conc(double kappa, double D1, double ds1, double f12, double D2, double ds2, double f21)
{
    const double C = 2.0 / 3.0;
    double num = (((kappa * ds1) / D1) * f12) * C;
    double den = 1.0 + ((kappa / 2.0) * (((ds1 / D1) * f12) + ((ds2 / D2) * f21))) * C;
    return num / den;
}

/* (c_to / c_from)^lambda for the walker's side `from`: lambda fixed (the
 * label of lower index is side 1, so the other side uses 1 - lambda) or,
 * for lambda < 0, the minimiser of alpha_lambda,
 * 1 / (1 + c_to sqrt(D_to) / (c_from sqrt(D_from))). */
double rmso_conc_factor(double c_from, double c_to, double D_from, double D_to, double lambda, int from_is_side1)
{
    double lam;
    if (lambda < 0.0)
        lam = 1.0 / (1.0 + (c_to * sqrt(D_to)) / (c_from * sqrt(D_from)));
    else
        lam = from_is_side1 ? lambda : 1.0 - lambda;
    return pow(c_to / c_from, lam);
}

/* App. C.3 (Baxter): P_{1->2} = c2 sqrt(D2) / (c1 sqrt(D1)) from the
 * high-flux side, 1 from the other: min(1, that ratio) either way. */
double rmso_perm_prob_baxter(double c1, double D1, double c2, double D2)
{
    return (c2 * sqrt(D2)) / (c1 * sqrt(D1));
}

/* Sec. 2.1.3 (magnetization transfer): the probability that a walker of
 * label 1 (D1, ds1) meeting a membrane of surface relaxivity rho is
 * saturated, P_MT = (rho ds1 / D1) C with C_3 = 2/3.  Evaluation order fixed:
 * ((rho*ds1)/D1)*C. */
double rmso_mt_prob(double rho, double D1, double ds1)
{
    const double C = 2.0 / 3.0;
    return ((rho * ds1) / D1) * C;
}

/* Bernoulli threshold: cross iff a uniform 32-bit word e < T, with
 * T = min(floor(P 2^32), 2^32 - 1); P clamped to [0,1] first. */
uint32_t rmso_threshold(double P)
{
    if (!(P > 0.0)) return 0u;
    if (P >= 1.0) return 0xFFFFFFFFu;
    double x = floor(P * 4294967296.0);
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)x;
}

static int64_t pmod(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

static int build_ctx(const rmso_config *cfg, ctx *X)
{
    int L = cfg->n_labels;
    memset(X, 0, sizeof(*X));
    X->cfg = cfg;
    if (cfg->lambda > 1.0) return RMSO_ERR_BAD_ARG;
    if (cfg->conc)
        for (int c = 0; c < L; c++)
            if (!cfg->dead[c] && !(cfg->conc[c] > 0.0)) return RMSO_ERR_BAD_ARG;
    X->s = (double *)malloc(sizeof(double) * L);
    for (int m = 0; m < 3; m++) X->dtR[m] = (double *)calloc(L, sizeof(double));
    X->T = (uint32_t *)calloc((size_t)L * L, sizeof(uint32_t));
    if (!X->s || !X->dtR[0] || !X->dtR[1] || !X->dtR[2] || !X->T) return RMSO_ERR_OOM;
    double *ds = (double *)malloc(sizeof(double) * L);
    if (!ds) return RMSO_ERR_OOM;
    for (int c = 0; c < L; c++) {
        ds[c] = rmso_step_length(cfg->D[c], cfg->dt);
        X->s[c] = ds[c] / cfg->voxel_um;
        /* Eq. 5: t_i / T^(i) accumulated per segment as (segment fraction) * (dt / T) */
        X->dtR[0][c] = isinf(cfg->T2[c]) ? 0.0 : cfg->dt / cfg->T2[c];
        X->dtR[1][c] = isinf(cfg->T1[c]) ? 0.0 : cfg->dt / cfg->T1[c];
        X->dtR[2][c] = 0.0;
        if (X->dtR[0][c] != 0.0 || X->dtR[1][c] != 0.0) X->any_relax = 1;
    }
    for (int a = 0; a < L; a++)
        for (int b = 0; b < L; b++) {
            double k = cfg->kappa[(size_t)a * L + b];
            if (a == b || cfg->dead[a] || cfg->dead[b] || !(k > 0.0)) {
                X->T[(size_t)a * L + b] = 0u;
                continue;
            }
            double P;
            const double ca = cfg->conc ? cfg->conc[a] : 1.0, cb = cfg->conc ? cfg->conc[b] : 1.0;
            if (cfg->perm_model == RMSO_PERM_BAXTER) {
                P = rmso_perm_prob_baxter(ca, cfg->D[a], cb, cfg->D[b]);
            } else if (cfg->conc) {
                double fab = rmso_conc_factor(ca, cb, cfg->D[a], cfg->D[b], cfg->lambda, a < b);
                double fba = rmso_conc_factor(cb, ca, cfg->D[b], cfg->D[a], cfg->lambda, b < a);
                P = rmso_perm_prob_conc(k, cfg->D[a], ds[a], fab, cfg->D[b], ds[b], fba);
            } else {
                P = rmso_perm_prob(k, cfg->D[a], ds[a], cfg->D[b], ds[b]);
            }
            X->T[(size_t)a * L + b] = rmso_threshold(P);
        }
    if (cfg->conc) {
        /* initial density proportional to the spin concentration (the
         * equilibrium rho1/rho2 = c1/c2 of App. C.2): a uniform start in
         * label l is kept with probability c_l / c_max */
        double cmax = 0.0;
        for (int c = 0; c < L; c++)
            if (!cfg->dead[c] && cfg->conc[c] > cmax) cmax = cfg->conc[c];
        X->acc = (uint64_t *)calloc(L, sizeof(uint64_t));
        if (!X->acc) {
            free(ds);
            return RMSO_ERR_OOM;
        }
        for (int c = 0; c < L; c++)
            X->acc[c] = cfg->dead[c] ? 0u : (uint64_t)floor((cfg->conc[c] / cmax) * 4294967296.0);
    }
    if (cfg->rho) {
        X->Tmt = (uint32_t *)calloc((size_t)L * L, sizeof(uint32_t));
        if (!X->Tmt) {
            free(ds);
            return RMSO_ERR_OOM;
        }
        for (int a = 0; a < L; a++)
            for (int b = 0; b < L; b++) {
                double r = cfg->rho[(size_t)a * L + b];
                if (a == b || cfg->dead[a] || !(r > 0.0)) continue; /* a membrane into a dead label counts */
                X->Tmt[(size_t)a * L + b] = rmso_threshold(rmso_mt_prob(r, cfg->D[a], ds[a]));
            }
    }
    free(ds);
    /* Sec. 2.2 item 1: uniform over non-dead voxels, raster order (x fastest) */
    int64_t nvox = (int64_t)cfg->nx * cfg->ny * cfg->nz;
    int any_dead = 0;
    for (int c = 0; c < L; c++) any_dead |= cfg->dead[c] != 0;
    if (!any_dead) {
        X->n_ok = nvox;
        X->ok_list = NULL;
    } else {
        X->ok_list = (int64_t *)malloc(sizeof(int64_t) * (size_t)nvox);
        if (!X->ok_list) return RMSO_ERR_OOM;
        int64_t n = 0;
        for (int64_t v = 0; v < nvox; v++)
            if (!cfg->dead[cfg->labels[v]]) X->ok_list[n++] = v;
        X->n_ok = n;
    }
    return 0;
}

static void free_ctx(ctx *X)
{
    free(X->s);
    for (int m = 0; m < 3; m++) free(X->dtR[m]);
    free(X->T);
    free(X->Tmt);
    free(X->acc);
    free(X->ok_list);
}

/* ------------------------------------------------------------------ */
/* Walker                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t i[3];
    double o[3];
    int64_t i0[3];
    double o0[3];
    int c;
    double A;
    double *phase; /* n_shapes x 3 */
    uint64_t h;
    int64_t n_events, n_cross, n_refl;
} walker;

static int label_at(const rmso_config *cfg, int64_t x, int64_t y, int64_t z)
{
    int64_t v = pmod(x, cfg->nx) + (int64_t)cfg->nx * (pmod(y, cfg->ny) + (int64_t)cfg->ny * pmod(z, cfg->nz));
    return cfg->labels[v];
}

static int64_t flat_index(const rmso_config *cfg, const int64_t i[3])
{
    return pmod(i[0], cfg->nx) + (int64_t)cfg->nx * (pmod(i[1], cfg->ny) + (int64_t)cfg->ny * pmod(i[2], cfg->nz));
}

/* Sec. 2.2 item 1.  r = x0 << 32 | x1 from INIT call 0 picks the voxel
 * floor(r n_ok / 2^64) of the raster list; the offset inside it is
 * (u(x2), u(x3), u(y0)) with y from INIT call 1. */
/* Sec. 2.2 item 1.  Attempt j uses INIT calls 2j and 2j + 1; with spin
 * concentrations a start in label l is kept iff word 1 of call 2j + 1 is
 * below acc[l] (at most RMSO_MAX_INIT attempts; returns 1 if none was
 * kept, the last one then stands). */
static int init_walker(const ctx *X, uint64_t w, walker *s)
{
    const rmso_config *cfg = X->cfg;
    uint32_t x[4], y[4];
    int64_t v = 0;
    int ok = 0;
    for (uint32_t j = 0; j < RMSO_MAX_INIT && !ok; j++) {
        draw(cfg->seed, w, 0u, TAG_INIT, 2u * j, x);
        draw(cfg->seed, w, 0u, TAG_INIT, 2u * j + 1u, y);
        uint64_t r = ((uint64_t)x[0] << 32) | (uint64_t)x[1];
        int64_t idx = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)X->n_ok) >> 64);
        v = X->ok_list ? X->ok_list[idx] : idx;
        ok = !X->acc || (uint64_t)y[1] < X->acc[cfg->labels[v]];
    }
    s->i[0] = v % cfg->nx;
    s->i[1] = (v / cfg->nx) % cfg->ny;
    s->i[2] = v / ((int64_t)cfg->nx * cfg->ny);
    s->o[0] = u01(x[2]);
    s->o[1] = u01(x[3]);
    s->o[2] = u01(y[0]);
    for (int a = 0; a < 3; a++) {
        s->i0[a] = s->i[a];
        s->o0[a] = s->o[a];
    }
    s->c = cfg->labels[v];
    s->A = 0.0;
    for (int k = 0; k < 3 * cfg->n_shapes; k++) s->phase[k] = 0.0;
    s->h = 0;
    s->n_events = s->n_cross = s->n_refl = 0;
    return !ok;
}

/* Sec. 2.2 item 2, direction sampler (the paper does not name one):
 * Archimedes' hat-box theorem -- z = 1 - 2u is uniform on [-1,1] for a
 * uniform point of the sphere -- with the azimuth phi = 2 pi (x1 + 1/2) 2^-32
 * from the second word.  sin and cos of the azimuth: an octant reduction in
 * integers, then a table of 1024 angles of [0, pi/4] (itself from Taylor
 * polynomials of degree 17 / 16), a 5th-order polynomial for the small
 * offset from the nearest table angle and the angle-addition formula.  Only
 * +, *, sqrt are used, so the result is the same bits on every IEEE machine.  One DIR call (k, call 0)
 * per step: words 0 and 1 give the direction, words 2 and 3 are the PERM
 * words of the step's first two membrane events. */
static const double kPi4 = 0.78539816339744830962; /* pi/4 */

/* sin and cos on [0, pi/4] by Taylor polynomials (degree 17 / 16). */
static void poly_sincos(double th, double *sn, double *cs)
{
    const double t = th * th;
    double ps = 1.0 / 355687428096000.0;       /*  1/17! */
    ps = -1.0 / 1307674368000.0 + t * ps;       /* -1/15! */
    ps = 1.0 / 6227020800.0 + t * ps;           /*  1/13! */
    ps = -1.0 / 39916800.0 + t * ps;            /* -1/11! */
    ps = 1.0 / 362880.0 + t * ps;               /*  1/9!  */
    ps = -1.0 / 5040.0 + t * ps;                /* -1/7!  */
    ps = 1.0 / 120.0 + t * ps;                  /*  1/5!  */
    ps = -1.0 / 6.0 + t * ps;                   /* -1/3!  */
    *sn = th + (th * t) * ps;
    double pc = 1.0 / 20922789888000.0;         /*  1/16! */
    pc = -1.0 / 87178291200.0 + t * pc;         /* -1/14! */
    pc = 1.0 / 479001600.0 + t * pc;            /*  1/12! */
    pc = -1.0 / 3628800.0 + t * pc;             /* -1/10! */
    pc = 1.0 / 40320.0 + t * pc;                /*  1/8!  */
    pc = -1.0 / 720.0 + t * pc;                 /* -1/6!  */
    pc = 1.0 / 24.0 + t * pc;                   /*  1/4!  */
    pc = -1.0 / 2.0 + t * pc;                   /* -1/2!  */
    *cs = 1.0 + t * pc;
}

/* The octant [0, pi/4] is cut into 1024 equal parts; TRIG[j] = (cos, sin) of
 * the centre of part j, theta_j = (2j + 1) 2^-11 pi/4. */
static double g_trig[1024][2];
static pthread_once_t g_trig_once = PTHREAD_ONCE_INIT;

static void build_trig(void)
{
    for (int j = 0; j < 1024; j++) {
        const double th = ((double)(2 * j + 1) * 0x1p-11) * kPi4;
        poly_sincos(th, &g_trig[j][1], &g_trig[j][0]);
    }
}

static void direction_from(uint32_t x0, uint32_t x1, double n[3])
{
    pthread_once(&g_trig_once, build_trig);
    const double z = 1.0 - 2.0 * u01(x0);
    const double r = sqrt((1.0 - z) * (1.0 + z));
    const uint32_t oct = x1 >> 29;
    uint32_t m = x1 & 0x1FFFFFFFu;
    if (oct & 1u) m = 0x1FFFFFFFu - m; /* odd octant: angle measured back from the octant's end */
    /* angle (m + 1/2) 2^-29 pi/4 = theta_j + e: j = the top 10 bits of m, e the
     * offset of the low 19 bits from the part's centre, |e| <= 2^-11 pi/4 */
    const uint32_t j = m >> 19;
    const int32_t lo = (int32_t)(m & 0x7FFFFu);
    const double e = ((double)(2 * lo + 1 - (1 << 19)) * 0x1p-30) * kPi4;
    const double t = e * e;
    const double se = e + (e * t) * (-1.0 / 6.0 + t * (1.0 / 120.0)); /* truncation < 1e-25 */
    const double ce = 1.0 + t * (-1.0 / 2.0 + t * (1.0 / 24.0));      /* truncation < 1e-22 */
    const double cj = g_trig[j][0], sj = g_trig[j][1];
    const double cs = cj * ce - sj * se; /* cos(theta_j + e) */
    const double sn = sj * ce + cj * se; /* sin(theta_j + e) */
    double cx, sy; /* cos and sin of oct pi/4 + angle (even) or (oct+1) pi/4 - angle (odd) */
    switch (oct) {
    case 0: cx = cs; sy = sn; break;
    case 1: cx = sn; sy = cs; break;
    case 2: cx = -sn; sy = cs; break;
    case 3: cx = -cs; sy = sn; break;
    case 4: cx = -cs; sy = -sn; break;
    case 5: cx = -sn; sy = -cs; break;
    case 6: cx = sn; sy = -cs; break;
    default: cx = cs; sy = -sn; break;
    }
    n[0] = r * cx;
    n[1] = r * sy;
    n[2] = z;
}

/* The step's DIR call (call = the attempt: 0, or the redraw of an ERL leap):
 * direction from words 0, 1; PERM words 0, 1 from words 2, 3. */
static void direction_call(uint64_t seed, uint64_t w, uint32_t k, uint32_t call, double n[3], uint32_t perm01[2])
{
    uint32_t x[4];
    draw(seed, w, k, TAG_DIR, call, x);
    direction_from(x[0], x[1], n);
    perm01[0] = x[2];
    perm01[1] = x[3];
}

static void direction(uint64_t seed, uint64_t w, uint32_t k, double n[3], uint32_t perm01[2])
{
    direction_call(seed, w, k, 0u, n, perm01);
}

static double clamp01(double x)
{
    if (x < 0.0) return 0.0;
    if (x > 1.0) return 1.0;
    return x;
}

/* One step's face walk (Sec. 2.2 items 3-4, Sec. 2.1.3, Fig. 2).
 *
 * Time within the step runs over [0, 1]; in the walker's current label c the
 * displacement per unit time is d = n s_c (voxel units).  For each axis a
 * with d_a != 0 the face ahead is dist_a = 1 - o_a (d_a > 0) or o_a (d_a < 0)
 * away and is met at time T_a = dist_a / |d_a| (from the step start; it may
 * lie beyond the step).  Events are taken in time order (smallest T first,
 * ties to the lowest axis, x < y < z) while T < 1:
 *   the other axes move to that time (o += (T - tau) d, clamped to [0,1]),
 *   the event axis is put exactly on its face, and the voxel across the face
 *   has label c' (periodic lookups i mod N; beyond a non-periodic edge there
 *   is an impermeable wall):
 *     c' == c                       -> cross (transparent face, Sec. 2.2 item 3)
 *     word[e] < T[c][c'] (Eq. 3)    -> cross into c' (the remaining time of the
 *                                      step is kept; the step length becomes s_c')
 *     otherwise                     -> reflect: n_a = -n_a (elastic collision)
 *   where e is the index of this event in the step and word[0], word[1] are
 *   words 2, 3 of the step's DIR call, word[2] word 0 of its PERM call.
 * An axis meets at most one face per step (with s_c < 1 a crossed or
 * reflected axis would need a whole voxel to meet another: the corner
 * reflector), so its time is then set to infinity.  A crossing into a label
 * with another step length changes the speed: the remaining axes' times are
 * then recomputed from their current positions, T_a = tau + dist_a / |d_a|.
 * Finally every axis moves by (1 - tau) d and is clamped to [0,1].  The
 * relaxation exponent accumulates (segment duration) x (dt / T of the
 * segment's label). */
#define WALK_REJECTED 1 /* walk_step: a membrane refused the step (rejection sampling or ERL) */

static int walk_step(const ctx *X, uint64_t w, uint32_t k, walker *s, double n[3],
                     const uint32_t perm01[2], const uint32_t *perm2_given, int mode, int interaction,
                     uint32_t attempt)
{
    const rmso_config *cfg = X->cfg;
    const int L = cfg->n_labels;
    const int32_t N[3] = {cfg->nx, cfg->ny, cfg->nz};
    double sc = X->s[s->c];
    double rate = X->dtR[mode][s->c];
    double d[3] = {n[0] * sc, n[1] * sc, n[2] * sc};
    double T[3];
    for (int a = 0; a < 3; a++) {
        if (d[a] > 0.0)
            T[a] = (1.0 - s->o[a]) / d[a];
        else if (d[a] < 0.0)
            T[a] = s->o[a] / (-d[a]);
        else
            T[a] = INFINITY;
    }
    double tau = 0.0;
    for (int ev = 0; ev < 3; ev++) {
        int best = 0;
        double tmin = T[0];
        if (T[1] < tmin) {
            best = 1;
            tmin = T[1];
        }
        if (T[2] < tmin) {
            best = 2;
            tmin = T[2];
        }
        if (!(tmin < 1.0)) break;
        const double dt_seg = tmin - tau;
        for (int a = 0; a < 3; a++)
            if (a != best) s->o[a] = clamp01(s->o[a] + dt_seg * d[a]);
        const int up = d[best] > 0.0;
        s->o[best] = up ? 1.0 : 0.0;
        s->A = s->A + dt_seg * rate;
        tau = tmin;
        T[best] = INFINITY;
        s->n_events++;

        int64_t j = s->i[best] + (up ? 1 : -1);
        int c2;
        if (!cfg->periodic[best] && (j < 0 || j >= N[best])) {
            c2 = -1; /* outer wall */
        } else {
            int64_t q[3] = {s->i[0], s->i[1], s->i[2]};
            q[best] = j;
            c2 = label_at(cfg, q[0], q[1], q[2]);
        }
        /* Sec. 2.1.3, magnetization transfer: meeting an absorbing membrane
         * saturates the walker with probability P_MT (word e of the step's
         * MT call, call = the attempt); a saturated walker's weight is 0 for
         * good (Eq. wt-mt), kept as an infinite exponent A. */
        if (X->Tmt && c2 >= 0 && c2 != s->c) {
            uint32_t Tm = X->Tmt[(size_t)s->c * L + c2];
            if (Tm != 0u && !isinf(s->A)) {
                uint32_t m4[4];
                draw(cfg->seed, w, k, TAG_MT, attempt, m4);
                if (m4[ev] < Tm) s->A = INFINITY;
            }
        }
        int cross;
        if (c2 == s->c) {
            cross = 1;
        } else if (c2 < 0) {
            cross = 0;
        } else {
            uint32_t Th = X->T[(size_t)s->c * L + c2];
            if (Th == 0u) {
                cross = 0;
            } else {
                uint32_t word;
                if (ev < 2) {
                    word = perm01[ev];
                } else if (perm2_given) {
                    word = *perm2_given;
                } else {
                    uint32_t p4[4];
                    draw(cfg->seed, w, k, TAG_PERM, attempt, p4);
                    word = p4[0];
                }
                cross = word < Th;
            }
        }
        if (cross) {
            s->i[best] = j;
            s->o[best] = up ? 0.0 : 1.0;
            if (c2 != s->c) {
                s->c = c2;
                s->n_cross++;
                rate = X->dtR[mode][c2];
                if (X->s[c2] != sc) {
                    sc = X->s[c2];
                    for (int a = 0; a < 3; a++) {
                        d[a] = n[a] * sc;
                        if (T[a] == INFINITY) continue;
                        if (d[a] > 0.0)
                            T[a] = tau + (1.0 - s->o[a]) / d[a];
                        else
                            T[a] = tau + s->o[a] / (-d[a]);
                    }
                }
            }
        } else if (interaction != RMSO_EC) {
            return WALK_REJECTED; /* the caller undoes the partial move */
        } else {
            n[best] = -n[best];
            d[best] = -d[best];
            s->n_refl++;
        }
    }
    const double rem = 1.0 - tau;
    for (int a = 0; a < 3; a++) s->o[a] = clamp01(s->o[a] + rem * d[a]);
    s->A = s->A + rem * rate;
    return 0;
}

/* Sec. 2.3, Eq. 7 discretised: phi = sum_k (dt G_k) . x_k with x_k the
 * position at the end of step k.  Positions enter relative to the start,
 * Delta x = l_p ((i - i0) + (o - o0)); for a waveform with sum_k G_k = 0
 * this is the same phase (the constant x_0 term vanishes). */
static void displacement(const rmso_config *cfg, const walker *s, double dx[3])
{
    for (int a = 0; a < 3; a++)
        dx[a] = cfg->voxel_um * ((double)(s->i[a] - s->i0[a]) + (s->o[a] - s->o0[a]));
}

static void neumaier_add(double *sum, double *comp, double x)
{
    double t = *sum + x;
    if (fabs(*sum) >= fabs(x))
        *comp += (*sum - t) + x;
    else
        *comp += (x - t) + *sum;
    *sum = t;
}

/* Sec. 2.3 narrow-pulse D and K need <alpha>, <alpha dx_i dx_j> and
 * <alpha dx_i dx_j dx_k dx_l>: 1 + 6 + 15 = 22 sums, symmetric tensor
 * components in lexicographic index order (i<=j, i<=j<=k<=l). */
static void moment_terms(double alpha, const double dx[3], double m[22])
{
    int p = 0;
    m[p++] = alpha;
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++) m[p++] = alpha * dx[a] * dx[b];
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++)
            for (int c = b; c < 3; c++)
                for (int d = c; d < 3; d++) m[p++] = alpha * dx[a] * dx[b] * dx[c] * dx[d];
}

typedef struct {
    const ctx *X;
    rmso_output *out;
    int64_t wb, we;  /* global ids */
    double *msum, *mcomp;
    int err;
} job;

static void *run_range(void *arg)
{
    job *J = (job *)arg;
    const ctx *X = J->X;
    const rmso_config *cfg = X->cfg;
    rmso_output *out = J->out;
    const int S = cfg->n_shapes;
    walker s;
    s.phase = (double *)malloc(sizeof(double) * 3 * (S > 0 ? S : 1));
    if (!s.phase) {
        J->err |= RMSO_ERR_OOM;
        return NULL;
    }
    for (int64_t w = J->wb; w < J->we; w++) {
        if (init_walker(X, (uint64_t)w, &s)) J->err |= RMSO_ERR_INIT;
        int r = 0;
        for (int64_t k = 1; k <= cfg->n_steps; k++) {
            double n[3];
            uint32_t perm01[2];
            direction(cfg->seed, (uint64_t)w, (uint32_t)k, n, perm01);
            int mode = cfg->mode ? cfg->mode[k - 1] : 0;
            if (cfg->interaction == RMSO_EC) {
                walk_step(X, (uint64_t)w, (uint32_t)k, &s, n, perm01, NULL, mode, RMSO_EC, 0u);
            } else {
                /* App. B (rejection sampling): a step that a membrane refuses is
                 * cancelled and the walker stays where it was for the step.
                 * App. A (ERL): a refused step is cancelled and redrawn in a new
                 * direction (DIR call = attempt) until one is admitted. */
                const walker s0 = s;
                const double rate0 = X->dtR[mode][s.c];
                int accepted = 0, saturated = 0;
                const uint32_t attempts = cfg->interaction == RMSO_ERL ? RMSO_MAX_LEAPS : 1u;
                for (uint32_t att = 0; att < attempts && !accepted; att++) {
                    if (att > 0) {
                        s = s0; /* a saturation met on a cancelled draw stays */
                        if (saturated) s.A = INFINITY;
                        direction_call(cfg->seed, (uint64_t)w, (uint32_t)k, att, n, perm01);
                    }
                    accepted = walk_step(X, (uint64_t)w, (uint32_t)k, &s, n, perm01, NULL, mode,
                                         cfg->interaction, att) == 0;
                    saturated |= isinf(s.A);
                }
                if (!accepted) {
                    s = s0; /* stays for the step, in its label */
                    if (saturated) s.A = INFINITY;
                    s.A = s.A + 1.0 * rate0;
                    s.n_refl++;
                    if (cfg->interaction == RMSO_ERL) J->err |= RMSO_ERR_LEAPS;
                }
            }
            if (cfg->hash) {
                uint64_t v = (((uint64_t)k & 0xFFFFu) << 48) ^ ((uint64_t)(uint32_t)s.c << 32) ^
                             (uint64_t)flat_index(cfg, s.i);
                s.h = rmso_mix64(s.h ^ v);
            }
            double dx[3];
            int have_dx = 0;
            for (int sh = 0; sh < S; sh++) {
                double wG = cfg->dt * cfg->G[(size_t)sh * cfg->n_steps + (k - 1)];
                if (!have_dx) {
                    displacement(cfg, &s, dx);
                    have_dx = 1;
                }
                for (int a = 0; a < 3; a++) s.phase[3 * sh + a] = s.phase[3 * sh + a] + wG * dx[a];
            }
            if (r < cfg->n_rec && cfg->rec_steps[r] == k) {
                if (!have_dx) displacement(cfg, &s, dx);
                double m[22];
                moment_terms(exp(-s.A), dx, m);
                for (int q = 0; q < 22; q++)
                    neumaier_add(&J->msum[(size_t)r * 22 + q], &J->mcomp[(size_t)r * 22 + q], m[q]);
                r++;
            }
        }
        int64_t o = w - cfg->w_begin;
        for (int a = 0; a < 3; a++) {
            if (out->i) out->i[3 * o + a] = (int32_t)s.i[a];
            if (out->o) out->o[3 * o + a] = s.o[a];
            if (out->i0) out->i0[3 * o + a] = (int32_t)s.i0[a];
            if (out->o0) out->o0[3 * o + a] = s.o0[a];
        }
        if (out->c) out->c[o] = s.c;
        if (out->A) out->A[o] = s.A;
        if (out->phase)
            for (int k = 0; k < 3 * S; k++) out->phase[(size_t)o * 3 * S + k] = s.phase[k];
        if (out->hash) out->hash[o] = s.h;
        if (out->counts) {
            out->counts[3 * o + 0] = s.n_events;
            out->counts[3 * o + 1] = s.n_cross;
            out->counts[3 * o + 2] = s.n_refl;
        }
    }
    free(s.phase);
    return NULL;
}

/* Run walkers [w_begin, w_end) through all n_steps steps.  Returns 0 or an
 * OR of RMSO_ERR_* bits. */
int rmso_run(const rmso_config *cfg, rmso_output *out)
{
    if (!cfg || !out || cfg->nx <= 0 || cfg->ny <= 0 || cfg->nz <= 0 || cfg->n_labels <= 0 ||
        cfg->w_end < cfg->w_begin || cfg->n_steps < 0 || cfg->n_shapes < 0 || !(cfg->dt > 0.0))
        return RMSO_ERR_BAD_ARG;
    ctx X;
    int err = build_ctx(cfg, &X);
    if (err) {
        free_ctx(&X);
        return err;
    }
    int nt = cfg->n_threads > 0 ? cfg->n_threads : 1;
    int64_t nw = cfg->w_end - cfg->w_begin;
    if (nt > nw) nt = nw > 0 ? (int)nw : 1;
    job *jobs = (job *)calloc(nt, sizeof(job));
    pthread_t *th = (pthread_t *)calloc(nt, sizeof(pthread_t));
    size_t nm = (size_t)(cfg->n_rec > 0 ? cfg->n_rec : 1) * 22;
    for (int t = 0; t < nt; t++) {
        jobs[t].X = &X;
        jobs[t].out = out;
        jobs[t].wb = cfg->w_begin + nw * t / nt;
        jobs[t].we = cfg->w_begin + nw * (t + 1) / nt;
        jobs[t].msum = (double *)calloc(nm, sizeof(double));
        jobs[t].mcomp = (double *)calloc(nm, sizeof(double));
    }
    for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, run_range, &jobs[t]);
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
    /* combine the per-thread compensated sums in thread order */
    if (out->moments) {
        for (size_t q = 0; q < (size_t)cfg->n_rec * 22; q++) {
            double s = 0.0, c = 0.0;
            for (int t = 0; t < nt; t++) {
                neumaier_add(&s, &c, jobs[t].msum[q]);
                neumaier_add(&s, &c, jobs[t].mcomp[q]);
            }
            out->moments[q] = s + c;
        }
    }
    for (int t = 0; t < nt; t++) {
        err |= jobs[t].err;
        free(jobs[t].msum);
        free(jobs[t].mcomp);
    }
    free(jobs);
    free(th);
    free_ctx(&X);
    return err;
}

/* ------------------------------------------------------------------ */
/* Readout (Sec. 2.3, Eq. 7)                                           */
/* ------------------------------------------------------------------ */
/* b of a unit-amplitude waveform: with F_j = sum_{k<=j} dt G_k,
 * b_s = dt sum_{j=1..N} F_{j-1}^2 (compensated sum).  For a rectangular
 * pulse pair this tends to delta^2 (Delta - delta/3) as dt -> 0. */
double rmso_bvalue(const double *G, int64_t n_steps, double dt)
{
    double F = 0.0, s = 0.0, c = 0.0;
    for (int64_t j = 1; j <= n_steps; j++) {
        neumaier_add(&s, &c, F * F);
        F = F + dt * G[j - 1];
    }
    return dt * (s + c);
}

/* S(b, g) = sum alpha e^{-i phi} / sum alpha with alpha = exp(-A) and
 * phi = q g.Phi_s, q = sqrt(b / b_s) the gradient amplitude that gives
 * b-value b for shape s (phi is linear in the amplitude, so one phase
 * vector per shape serves every direction and b-value).
 * Output S_re/S_im: n_shapes x n_dirs x n_b. */
void rmso_readout(int64_t n_walkers, int32_t n_shapes, const double *phase, const double *A,
                  const double *G, int64_t n_steps, double dt, int32_t n_dirs, const double *dirs,
                  int32_t n_b, const double *b, double *S_re, double *S_im, double *alpha_sum)
{
    double as = 0.0, ac = 0.0;
    for (int64_t w = 0; w < n_walkers; w++) neumaier_add(&as, &ac, exp(-A[w]));
    double asum = as + ac;
    if (alpha_sum) *alpha_sum = asum;
    for (int s = 0; s < n_shapes; s++) {
        double bs = rmso_bvalue(G + (size_t)s * n_steps, n_steps, dt);
        for (int g = 0; g < n_dirs; g++) {
            for (int ib = 0; ib < n_b; ib++) {
                double q = (bs > 0.0) ? sqrt(b[ib] / bs) : 0.0;
                double rs = 0.0, rc = 0.0, is = 0.0, ic = 0.0;
                for (int64_t w = 0; w < n_walkers; w++) {
                    const double *P = phase + (size_t)w * 3 * n_shapes + 3 * s;
                    double phi = q * (dirs[3 * g] * P[0] + dirs[3 * g + 1] * P[1] + dirs[3 * g + 2] * P[2]);
                    double al = exp(-A[w]);
                    neumaier_add(&rs, &rc, al * cos(phi));
                    neumaier_add(&is, &ic, -al * sin(phi));
                }
                size_t o = ((size_t)s * n_dirs + g) * n_b + ib;
                S_re[o] = (rs + rc) / asum;
                S_im[o] = (is + ic) / asum;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Test hooks (tests only)                                             */
/* ------------------------------------------------------------------ */
/* One face walk from a given state with a given direction and given PERM
 * words perm[0..2] for the step's events 0..2 (bypasses the random draws).  state_i/state_o/c/A are in-out;
 * n is in-out (reflections flip it).  Returns error bits; events out. */
int rmso_walk_once(const rmso_config *cfg, int64_t state_i[3], double state_o[3], int32_t *c,
                   double *A, double n[3], const uint32_t perm[4], int32_t mode, int64_t counts[3])
{
    ctx X;
    int err = build_ctx(cfg, &X);
    if (err) {
        free_ctx(&X);
        return err;
    }
    walker s;
    memset(&s, 0, sizeof(s));
    for (int a = 0; a < 3; a++) {
        s.i[a] = state_i[a];
        s.o[a] = state_o[a];
    }
    s.c = *c;
    s.A = *A;
    err = walk_step(&X, 0u, 1u, &s, n, perm, perm + 2, mode, RMSO_EC, 0u);
    for (int a = 0; a < 3; a++) {
        state_i[a] = s.i[a];
        state_o[a] = s.o[a];
    }
    *c = s.c;
    *A = s.A;
    if (counts) {
        counts[0] = s.n_events;
        counts[1] = s.n_cross;
        counts[2] = s.n_refl;
    }
    free_ctx(&X);
    return err;
}

/* The per-pair thresholds the walker uses (n_labels^2, row = from-label). */
int rmso_thresholds(const rmso_config *cfg, uint32_t *T_out, double *s_out)
{
    ctx X;
    int err = build_ctx(cfg, &X);
    if (!err) {
        memcpy(T_out, X.T, sizeof(uint32_t) * (size_t)cfg->n_labels * cfg->n_labels);
        if (s_out) memcpy(s_out, X.s, sizeof(double) * cfg->n_labels);
    }
    free_ctx(&X);
    return err;
}

/* The unit direction of step k of walker w (DIR stream). */
int rmso_direction(uint64_t seed, uint64_t w, uint32_t k, double n[3])
{
    uint32_t p[2];
    direction(seed, w, k, n, p);
    return 0;
}

/* The unit direction made from two given words. */
void rmso_direction_from_words(uint32_t x0, uint32_t x1, double n[3]) { direction_from(x0, x1, n); }
