/*
 * rms.h -- C ABI of the GB300 random-walker engine for diffusion MRI Monte
 * Carlo in voxelised cell segmentations, after Lee, Fieremans & Novikov,
 * "Realistic Microstructure Simulator (RMS)", arXiv 2012.06478.
 *
 * The engine runs the method's data-parallel hot path on one GPU: walkers
 * start uniformly over non-dead voxels (Sec. 2.2 item 1), take steps of
 * length ds = sqrt(6 D dt) (Eq. 1) in Philox4x32-10 random directions, walk
 * through voxel faces with at most three face events per step (Sec. 2.1.1,
 * Fig. 2), cross a face between two labels with the finite-step corrected
 * probability of Eq. 3 or are reflected specularly (Sec. 2.1.3), accumulate
 * the phase of Eq. 7 and the relaxation weight of Eq. 5, and are reduced to
 * the signal S(b, g) (Eq. 7) and the displacement moments behind the
 * narrow-pulse D(t) and K(t) (Sec. 2.3).  It also runs the alternatives the
 * paper analyses: rejection sampling and the equal-step-length random leap
 * (App. A-B), absorbing membranes for magnetization transfer (Sec. 2.1.3),
 * spin concentrations and Baxter's permeation rule (App. C.2-C.3).
 *
 * Conventions for every call:
 *   - Plain C types and pointers only.  "host pointer" = ordinary process
 *     memory; "device pointer" = memory on the current CUDA device.
 *   - The library copies every input array; the caller keeps ownership and
 *     may free its buffers as soon as the call returns.
 *   - Handles own their device memory and free it on destroy.
 *   - A `void *stream` is a cudaStream_t (NULL = the legacy default stream).
 *     Work is enqueued on it asynchronously; calls that return results to
 *     host memory synchronise with it.
 *   - Every call returns an rms_status; on an error rms_last_error() gives a
 *     message (per calling thread).  No C++ exception crosses this boundary.
 *   - All handles belong to the device that was current when they were made;
 *     use them with that device current.
 */
#ifndef RMS_H
#define RMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int rms_status;

#define RMS_OK 0
#define RMS_W_PROB_RANGE 1        /* warning: some P_{1->2} of Eq. 3 exceeded 1 and was clamped */
#define RMS_W_LEAP_LIMIT 2        /* warning (RMS_ERL runs): some step found no admissible direction in
                                     RMS_MAX_LEAPS draws; that walker stayed for the step (results valid) */
#define RMS_E_INVALID_ARG (-1)    /* a null pointer, a size out of range, an inconsistent array */
#define RMS_E_OOM (-2)            /* a device or host allocation failed */
#define RMS_E_CUDA (-3)           /* a CUDA runtime call failed (message has the CUDA error) */
#define RMS_E_STEP_TOO_LARGE (-4) /* ds_c >= l_p for some label: a step could meet more than three faces */
#define RMS_E_TIMEOUT (-6)        /* a bounded wait gave up */
#define RMS_E_CANCELLED (-7)      /* the run was cancelled before it finished */
#define RMS_E_BUSY (-8)           /* the handle is still referenced by a live sequence or run */
#define RMS_E_DEVICE (-9)         /* a kernel reported a broken invariant (see message) */
#define RMS_E_NOT_READY (-10)     /* the run is still in flight */

/* precision forms of rms_run */
#define RMS_FP64 0 /* plain form: FP64 positions and phases, no FMA; bit-exact trajectories */
#define RMS_FP32 1 /* precision form: voxel index + FP32 offset, FP32 Kahan phase, FP64 reductions; the
                      read-out's terms alpha e^{-i phi} in FP32 (within ~1e-5 of their FP64 sum, Eq. 7) */

/* rms_run flags */
#define RMS_TRAJ_HASH 1u /* keep a per-walker 64-bit checksum of the (step, voxel, label) sequence */
#define RMS_CHECKED 2u   /* verify the walker invariants after every step -- voxel coordinates in range,
                            flat index consistent with them, the walker's label equal to its voxel's,
                            offsets in [0,1] -- in the verification kernel (the one that also keeps
                            the checksum); a violation makes the read calls return RMS_E_DEVICE.
                            Slower; for testing and debugging. */
#define RMS_COUNTS 4u    /* count, per walker, face events, crossings into another label and
                            reflections (or steps a refused walker stayed, RS/ERL) -- in the
                            verification kernel; read with rms_read_counts */
#define RMS_MORTON 8u    /* before every step launch, put the walkers in Morton order of their voxel
                            (x, y, z bits interleaved; for edges above 256 voxels the coordinates are
                            first shifted right to 8 bits), so that walkers next to each other in
                            memory look up neighbouring parts of the label volume (Sec. 2.1.1: the
                            volume is the lookup table).  For volumes about the size of the L2
                            cache or larger (measured: +23 % at 128 MB, +10 % at 256 MiB, no
                            change at 32 MB).
                            Changes no trajectory (the random streams follow the walker id, not its
                            place in memory) and nothing rms_read_walkers / rms_read_counts return;
                            only the order of the sums over walkers (signal and moment sums agree to
                            rounding).  Costs a second copy of the walker state and about 17 bytes
                            per walker of sort buffers.  With this flag the default launch covers
                            about 8e9 walker-steps (steps_per_launch 0), and one re-ordering of 1e7
                            walkers takes about 1.3 % of it. */

/* Particle-membrane interaction of rms_run (Sec. 2.1.2).  A face is "refused"
 * when it is impermeable (a label pair with kappa = 0, a dead label, the wall
 * beyond a non-periodic edge) or when the Bernoulli trial of Eq. 3 fails.
 *   RMS_EC  elastic collision: a refused face reflects the step specularly
 *           and the rest of the step goes on (the paper's method).
 *   RMS_RS  rejection sampling (App. B): a refused face cancels the whole
 *           step; the walker stays where it was for that step (its dt still
 *           counts in the relaxation exponent of Eq. 5).
 *   RMS_ERL equal-step-length random leap (App. A): a refused face cancels
 *           the step and a new direction is drawn, until a step meets no
 *           refused face; draw m (m = 0, 1, ...) takes Philox DIR call m and
 *           PERM call m.  After RMS_MAX_LEAPS refused draws the walker stays
 *           for the step, as in RMS_RS, and the run reports RMS_W_LEAP_LIMIT.
 * App. A and B show that RS biases D parallel to membranes and that ERL also
 * makes the density near membranes inhomogeneous; they are here to reproduce
 * those biases and to compare against other simulators. */
#define RMS_EC 0
#define RMS_RS 1
#define RMS_ERL 2
#define RMS_MAX_LEAPS 64

/* Permeation models of rms_substrate_desc.perm_model (Sec. 2.1.3, App. C) */
#define RMS_PERM_KAPPA 0
#define RMS_PERM_BAXTER 1
#define RMS_MAX_INIT 4096 /* start draws per walker with spin concentrations */

typedef struct rms_substrate rms_substrate;
typedef struct rms_sequence rms_sequence;
typedef struct rms_run_handle rms_run_handle;

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int rms_version(void);

/* Message of the last error on the calling thread ("" if none). */
const char *rms_last_error(void);

/* ------------------------------------------------------------------ */
/* Substrate: the voxelised label volume and per-label tissue tables.  */
/* Sec. 2.1.1 (the label volume is its own lookup table), Sec. 2.1.3   */
/* (D, kappa), Sec. 2.1.4 (T1, T2), Table 1.                           */
/* ------------------------------------------------------------------ */
typedef struct {
    const uint16_t *labels;   /* nx*ny*nz labels, x fastest (index x + nx*(y + ny*z)) */
    int32_t labels_on_device; /* 1: `labels` is a device pointer, 0: host pointer */
    int32_t nx, ny, nz;       /* grid size, each >= 1, nx*ny*nz < 2^31 */
    double voxel_um;          /* isotropic voxel edge l_p (um), > 0 */
    int32_t periodic[3];      /* per axis: 1 periodic (lookups i mod N), 0 impermeable outer wall */
    int32_t n_labels;         /* L: every label value is < L; 1 <= L <= 65536 */
    const double *D;          /* host, L: intrinsic diffusivity (um^2/ms), > 0 */
    const double *T2;         /* host, L or NULL: T2 (ms), INFINITY = none */
    const double *T1;         /* host, L or NULL: T1 (ms), INFINITY = none */
    const double *kappa;      /* host, L*L or NULL: permeability (um/ms) of the membrane from
                                 label r (row) into label c (column); diagonal ignored */
    double kappa_scalar;      /* used for every pair when kappa == NULL */
    const double *rho;        /* host, L*L or NULL: surface relaxivity (um/ms) of the membrane met
                                 from label r (row) towards label c (column), for magnetization
                                 transfer (Sec. 2.1.3): each such face event saturates the walker
                                 with probability P_MT = (rho ds_r / D_r) C_3 (C_3 = 2/3; clamped to
                                 1 with RMS_W_PROB_RANGE), after which its weight is 0.  A membrane
                                 into a dead label counts; diagonal ignored; NULL: none */
    const double *conc;       /* host, L or NULL (all equal): spin concentration per label, > 0 for
                                 every live label (App. C.2).  Walkers start with density ~ c (a
                                 uniform start in label l is kept with probability c_l / c_max, at
                                 most RMS_MAX_INIT draws; RMS_E_INVALID_ARG when the volume mean of
                                 c / c_max is below 1/200), and permeation keeps the equilibrium
                                 density ratio c1/c2 */
    double lambda;            /* RMS_PERM_KAPPA with conc: P_{1->2} carries (c2/c1)^lambda and
                                 P_{2->1} (c2/c1)^(lambda-1), with the finite-step correction
                                 kappa = kappa0 / (1 - alpha_lambda); lambda in [0,1] with the label
                                 of lower index as side 1, or < 0 for the alpha-minimising lambda =
                                 1 / (1 + c2 sqrt(D2) / (c1 sqrt(D1))) */
    int32_t perm_model;       /* RMS_PERM_KAPPA (0): nominal permeability kappa, Eq. 3 (generalised
                                 when conc is given); RMS_PERM_BAXTER: P_{1->2} = c2 sqrt(D2) /
                                 (c1 sqrt(D1)) from the high-flux side, 1 from the other (App. C.3;
                                 its effective permeability grows as 1/sqrt(dt)); kappa > 0 then
                                 only marks which pairs are permeable */
    const uint8_t *dead;      /* host, L or NULL: 1 = no walker starts in or enters the label */
    void *stream;             /* cudaStream_t for the upload */
} rms_substrate_desc;

/* Upload the volume and build the per-label tables.  Errors:
 * RMS_E_INVALID_ARG, RMS_E_OOM, RMS_E_CUDA.  The permeation and saturation
 * thresholds are built when a sequence fixes dt (rms_set_sequence). */
rms_status rms_create_substrate(const rms_substrate_desc *desc, rms_substrate **out);

/* Free the substrate.  RMS_E_BUSY (and nothing freed) while a sequence made
 * from it is alive. */
rms_status rms_destroy_substrate(rms_substrate *sub);

/* ------------------------------------------------------------------ */
/* Sequence: time step, gradient waveforms, read-out directions and    */
/* b-values, recording steps.  Table 1 (dt, N_step), Eq. 7 (g(t)),     */
/* Sec. 2.3 (b, directions).                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    double dt_ms;             /* time step (ms), > 0 */
    int64_t n_steps;          /* N_step >= 0 */
    int32_t n_shapes;         /* number of waveform shapes, 1..8 */
    const double *G;          /* host, n_shapes*n_steps: effective gradient of unit amplitude,
                                 the average of g(t)/|g| over step k (row = shape) */
    const uint8_t *mode;      /* host, n_steps or NULL: relaxation during step k: 0 = T2, 1 = T1
                                 (stimulated-echo mixing time), 2 = none */
    int32_t n_dirs;           /* >= 1; n_shapes * n_dirs * n_b <= 8e6 */
    const double *dirs;       /* host, n_dirs*3 unit gradient directions */
    int32_t n_b;              /* >= 1 */
    const double *b;          /* host, n_b b-values (ms/um^2), >= 0 */
    int32_t n_rec;            /* >= 0 */
    const int64_t *rec_steps; /* host, n_rec strictly increasing steps in [1, n_steps] at which
                                 the displacement moments are recorded */
} rms_sequence_desc;

/* Validate and upload.  Builds ds_c = sqrt(6 D_c dt) (Eq. 1), the relaxation
 * rates, the per-pair Bernoulli thresholds floor(P 2^32) from Eq. 3, and
 * b_s = dt sum_j F_{j-1}^2 per shape.  Errors: RMS_E_INVALID_ARG,
 * RMS_E_STEP_TOO_LARGE (ds_c >= l_p for a non-dead label, Sec. 2.1.1 and
 * Table 1), RMS_E_OOM, RMS_E_CUDA.  Returns RMS_W_PROB_RANGE (with *out set)
 * when some P_{1->2} > 1 had to be clamped (Eq. 3 assumes P << 1). */
rms_status rms_set_sequence(rms_substrate *sub, const rms_sequence_desc *desc, rms_sequence **out);

/* b_s of each shape (host pointer, n_shapes doubles); synchronises. */
rms_status rms_sequence_bvalues(const rms_sequence *seq, double *b_s);

/* RMS_E_BUSY while a run made from it is alive. */
rms_status rms_destroy_sequence(rms_sequence *seq);

/* ------------------------------------------------------------------ */
/* Run                                                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t n_walkers;        /* W >= 1 */
    int64_t walker_begin;     /* global id of the first walker (walkers are w_begin .. w_begin+W-1);
                                 the random streams depend only on (seed, global id, step) */
    uint64_t seed;            /* Philox key */
    int32_t precision;        /* RMS_FP64 or RMS_FP32 */
    uint32_t flags;           /* RMS_TRAJ_HASH or 0 */
    int32_t steps_per_launch; /* steps per kernel launch (0 = default) */
    int32_t interaction;      /* RMS_EC (0), RMS_RS or RMS_ERL */
    void *stream;             /* cudaStream_t the whole run is enqueued on */
} rms_run_desc;

/* Allocate walker state and enqueue the whole simulation: initialisation
 * (Sec. 2.2 item 1), every step (Sec. 2.2 items 2-5, with the interaction
 * desc->interaction), the moment reductions and the signal read-out (Eq. 7).
 * Returns without waiting.  Errors: RMS_E_INVALID_ARG (also an unknown
 * interaction), RMS_E_OOM, RMS_E_CUDA. */
rms_status rms_run(rms_sequence *seq, const rms_run_desc *desc, rms_run_handle **out);

/* A run's state after `step` steps, for resuming it (checkpoint/restart).
 * Host arrays in the layouts rms_read_walkers writes; the caller keeps
 * ownership (they are read before rms_run_range returns). */
typedef struct {
    int64_t step;            /* steps already taken, 0 <= step <= n_steps */
    const int32_t *i;        /* W*3 unwrapped voxel index */
    const double *o;         /* W*3 offset in [0,1] */
    const int32_t *i0;       /* W*3 start voxel (wrapped) */
    const double *o0;        /* W*3 start offset */
    const int32_t *c;        /* W label */
    const double *A;         /* W relaxation exponent of Eq. 5 (+INFINITY: saturated) */
    const double *phase;     /* W*n_shapes*3 (may be NULL when n_shapes = 0) */
    const uint64_t *hash;    /* W checksums, or NULL (0) */
    const double *moments;   /* n_rec*22 moment sums (rms_read_signal layout) of the recording steps
                                <= step, or NULL (zeros) */
} rms_run_state;

/* rms_run over part of the sequence: start from the initialisation (from ==
 * NULL) or from a stored state (from->step steps taken, same W, walker_begin,
 * seed, precision and interaction as the run that wrote it), and stop after
 * step_end (0: n_steps).  The signal read afterwards is that of the phases
 * at step_end; moment sums of recording steps beyond step_end are 0.  The
 * random streams depend only on (seed, walker, step), so in the plain FP64
 * form a run split at any step and resumed gives the uninterrupted run's
 * walkers, checksums, moments and signal bit for bit; the FP32 form resumes
 * from the widened state (its Kahan terms restart from the float rounding of
 * each value) and agrees to rounding.  rms_run(seq, desc, out) is
 * rms_run_range(seq, desc, NULL, 0, out).  Errors as rms_run, and
 * RMS_E_INVALID_ARG for a step range outside 0 <= from->step <= step_end <=
 * n_steps or a missing array. */
rms_status rms_run_range(rms_sequence *seq, const rms_run_desc *desc, const rms_run_state *from, int64_t step_end,
                         rms_run_handle **out);

/* RMS_OK when the run has finished, RMS_E_NOT_READY while in flight. */
rms_status rms_run_query(rms_run_handle *run);

/* Ask a run to stop: launches not yet started do no work.  Reading it then
 * returns RMS_E_CANCELLED. */
rms_status rms_cancel(rms_run_handle *run);

/* Wait for the run and copy results to host memory (any pointer may be NULL).
 * Returns RMS_OK, or RMS_W_LEAP_LIMIT (results valid) for an RMS_ERL run in
 * which some step used up its draws:
 *   S_re, S_im : n_shapes*n_dirs*n_b, S = sum alpha e^{-i phi} / sum alpha
 *                (index (shape*n_dirs + dir)*n_b + b)
 *   moments    : n_rec*22 unnormalised sums over walkers at each recording step
 *                of alpha, alpha dx_i dx_j (i<=j: xx xy xz yy yz zz) and
 *                alpha dx_i dx_j dx_k dx_l (i<=j<=k<=l, lexicographic), dx in um
 *   alpha_sum  : 1 double, sum over walkers of alpha = exp(-sum t_i / T^(i)) at the end
 * Errors: RMS_E_CANCELLED, RMS_E_DEVICE, RMS_E_CUDA. */
rms_status rms_read_signal(rms_run_handle *run, double *S_re, double *S_im, double *moments,
                           double *alpha_sum);

/* Wait for the run and copy its UNNORMALISED reductions to host memory, for
 * combining runs over disjoint walker ranges of one simulation (walker
 * shards on several ranks, Sec. 2.1.5 runs walkers independently): sums over
 * walkers before the division by sum alpha of Eq. 7.  Any pointer may be
 * NULL; layouts as rms_read_signal:
 *   num_re, num_im : n_shapes*n_dirs*n_b, sum over walkers of alpha e^{-i phi}
 *   alpha_sum      : 1 double, sum over walkers of alpha at the end
 *   moments        : n_rec*22 sums (as rms_read_signal)
 * Shards combine by adding these element by element; rms_normalise_partials
 * then gives S.  Return codes as rms_read_signal. */
rms_status rms_read_partials(rms_run_handle *run, double *num_re, double *num_im, double *alpha_sum,
                             double *moments);

/* S = num / alpha_sum element by element (Eq. 7's normalisation), on host
 * arrays of n_combo doubles; the division rms_read_signal applies.
 * RMS_E_INVALID_ARG for n_combo < 0 or a null array. */
rms_status rms_normalise_partials(int64_t n_combo, const double *num_re, const double *num_im, double alpha_sum,
                                  double *S_re, double *S_im);

/* Wait for the run and copy the final per-walker state to host memory (any
 * pointer may be NULL; return codes as rms_read_signal; a saturated walker's
 * A is +INFINITY): i (W*3 int32 unwrapped voxel index), o (W*3 double
 * offset in [0,1]; the FP32 form's offsets widened), i0 (W*3), o0 (W*3),
 * c (W int32 label), A (W double exponent of Eq. 5), phase (W*n_shapes*3
 * double, sum_k dt G_k dx_k in um ms), hash (W uint64, RMS_TRAJ_HASH runs). */
rms_status rms_read_walkers(rms_run_handle *run, int32_t *i, double *o, int32_t *i0, double *o0, int32_t *c,
                            double *A, double *phase, uint64_t *hash);

/* Wait for the run and copy its per-walker counts to host memory: W*3 int64
 * (face events, crossings into another label, reflections -- under RS/ERL
 * the steps a refused walker stayed), over the run's steps.  The events of
 * a draw that a membrane refused are not counted.  RMS_E_INVALID_ARG when
 * the run was made without RMS_COUNTS. */
rms_status rms_read_counts(rms_run_handle *run, int64_t *counts);

/* Wait for the run and copy, for each slot of its walker state in device
 * memory, the walker in that slot (relative to walker_begin): W int32 on the
 * host.  0, 1, ..., W-1 unless the run has RMS_MORTON, whose walkers are in
 * Morton order of their voxels at the start of the last step launch.  A
 * diagnostic of the memory layout; no result depends on it.  Return codes as
 * rms_read_signal. */
rms_status rms_read_slots(rms_run_handle *run, int32_t *walker_of_slot);

/* Free the run (waits for it first). */
rms_status rms_destroy_run(rms_run_handle *run);

/* Device time (ms) between the start of the first and the end of the last
 * step launch of a finished run (with RMS_MORTON, the re-orderings before
 * each launch included); synchronises. */
rms_status rms_run_step_time_ms(rms_run_handle *run, float *ms);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of simulation requests.                */
/* Not in the paper (which runs one simulation per GPU, Sec. 2.1.5):   */
/* requests on resident substrates arrive at any time, are admitted as */
/* request slots and device memory free up, and every active request   */
/* advances in the same batched kernel launches, tick by tick.         */
/* ------------------------------------------------------------------ */
typedef struct rms_server rms_server;

/* Tick policies of rms_server_config.policy */
#define RMS_SERVE_STEPS 0 /* every active request advances steps_per_tick steps per tick (processor sharing by
                             steps: a request's latency grows with its step count, whatever its size) */
#define RMS_SERVE_FILL 1  /* size-aware: the batched launch of a precision takes as long as its largest
                             requests need for steps_per_tick steps (their blocks span several waves of the
                             GPU's block slots); a request whose blocks fit in one wave advances that many
                             waves' worth of steps instead (up to 64 x steps_per_tick), so small requests run
                             for the whole tick rather than waiting on the large ones */

typedef struct {
    int64_t memory_budget_bytes; /* device memory for the walker state of admitted requests (0: 8 GiB);
                                    a request is admitted when it fits (or when nothing else runs) */
    int32_t max_active;          /* requests admitted at once, 1..1024 (0: 64) */
    int32_t steps_per_tick;      /* steps every active request advances per tick (0: 256) */
    int32_t policy;              /* RMS_SERVE_STEPS (0) or RMS_SERVE_FILL */
} rms_server_config;

/* Start the scheduler thread on the current device. */
rms_status rms_server_create(const rms_server_config *cfg, rms_server **out);

/* Queue a request: n_walkers walkers of `seq` (its substrate stays resident;
 * both must outlive the request -- destroying them returns RMS_E_BUSY
 * meanwhile), Philox key `seed`, RMS_FP64 or RMS_FP32, elastic collision
 * (RMS_EC), on a substrate without absorbing membranes (rho == NULL, else
 * RMS_E_INVALID_ARG).  Returns at once with a ticket.  The result equals
 * rms_run's for the same arguments. */
rms_status rms_server_submit(rms_server *srv, rms_sequence *seq, int64_t n_walkers, uint64_t seed,
                             int32_t precision, int64_t *ticket);

/* RMS_OK when the ticket's request has finished (or failed, or was
 * cancelled), RMS_E_NOT_READY otherwise. */
rms_status rms_server_poll(rms_server *srv, int64_t ticket);

/* Wait up to timeout_ms (< 0: no limit) and copy the result to host memory
 * (layouts as rms_read_signal; any pointer may be NULL); the ticket is then
 * released.  RMS_E_TIMEOUT (ticket kept), RMS_E_CANCELLED, RMS_E_DEVICE. */
rms_status rms_server_wait(rms_server *srv, int64_t ticket, int64_t timeout_ms, double *S_re, double *S_im,
                           double *moments, double *alpha_sum);

/* Timing of a finished request, before rms_server_wait releases its ticket:
 * out[0] queueing (ms, submit to admission), out[1] latency (ms, submit to
 * result), out[2] its walker-steps (walkers x steps), out[3] the ticks it
 * took part in.  RMS_E_NOT_READY while it runs, RMS_E_INVALID_ARG for an
 * unknown ticket or a null pointer. */
rms_status rms_server_request_info(rms_server *srv, int64_t ticket, double *out);

/* Withdraw a queued or running request (a finishing one still completes). */
rms_status rms_server_cancel(rms_server *srv, int64_t ticket);

/* 11 doubles: p50, p99 and mean request latency (ms, submit to result),
 * walker-steps/s (all requests, first submit to last completion), completed,
 * in flight, queued, peak in flight, ticks, graph updates, graph
 * instantiations. */
rms_status rms_server_stats(rms_server *srv, double *out);

/* Cancel what is queued or running, stop the thread, free everything. */
rms_status rms_server_destroy(rms_server *srv);

/* ------------------------------------------------------------------ */
/* The counter-based generator behind every random draw (Sec. 2.2:     */
/* directions, Bernoulli trials of Eq. 3, start points), exposed so    */
/* that its words can be checked against other implementations.       */
/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11) on n (counter, key) pairs: DEVICE
 * pointers ctr (n*4 uint32 words c0..c3), key (n*2 words k0, k1) and out (n*4
 * words), the same function the walk kernels call with counter (walker_lo,
 * walker_hi, step, tag << 16 | call) and key (seed_lo, seed_hi).  Enqueued on
 * `stream` (cudaStream_t); returns without waiting.  RMS_E_INVALID_ARG for
 * n < 0 or a null pointer with n > 0, RMS_E_CUDA. */
rms_status rms_philox4x32_10(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out, void *stream);

/* ------------------------------------------------------------------ */
/* Signal read-out that allocates nothing.  The paper has no           */
/* counterpart: this is a service for callers that may not allocate    */
/* device memory at the point of the call -- for example a serving     */
/* loop sharing the GPU with other streams (cudaMalloc and cudaFree    */
/* can synchronise the whole device and stall them), or an application */
/* whose device memory all belongs to its own fixed pool or arena.     */
/* ------------------------------------------------------------------ */
#define RMS_NOALLOC_SCRATCH_BYTES (8 * 1024 * 1024)

/* The same read-out as rms_run's in the plain FP64 form (S = sum alpha
 * e^{-i phi} / sum alpha, phi = q g.Phi_s, q = sqrt(b / b_s), alpha =
 * exp(-A), every term in FP64) over walker data the caller holds.  Every pointer is a DEVICE pointer of the current device:
 *   phase     : n_walkers*n_shapes*3 doubles, row-major (walker, shape, axis),
 *               the layout rms_read_walkers returns
 *   A         : n_walkers doubles, exponent of Eq. 5
 *   b_s       : n_shapes doubles (rms_sequence_bvalues), dirs: n_dirs*3, b: n_b
 *   S_re, S_im: outputs, n_shapes*n_dirs*n_b doubles, index (shape*n_dirs + dir)*n_b + b
 *   alpha_sum : output, 1 double (may be NULL)
 * The work is enqueued on `stream` (cudaStream_t) and the call returns
 * without waiting.  It calls no cudaMalloc, cudaFree or other allocating
 * routine: its scratch is a fixed RMS_NOALLOC_SCRATCH_BYTES array inside the
 * library.  The CUDA runtime takes the array's memory on a device when it
 * loads the library's device code there -- lazily, at the library's first
 * use on that device, which may be this call -- and holds it until the
 * process exits.  The first call on each device also looks up the array's
 * address: make it (a warm-up call) before any stream capture on that
 * device.  After the device's context is replaced (cudaDeviceReset) the next
 * call loads the code and looks the address up again.  All calls share the array:
 * calls that may overlap on the GPU (other streams, other host threads) must
 * be serialised by the caller.  Errors: RMS_E_INVALID_ARG (null pointer,
 * n_walkers < 1, n_shapes outside 1..8, or 2*(n_shapes*n_dirs*n_b + 1) doubles
 * not fitting the scratch), RMS_E_CUDA. */
rms_status rms_readout_noalloc(const double *phase, const double *A, int64_t n_walkers, int32_t n_shapes,
                               const double *b_s, int32_t n_dirs, const double *dirs, int32_t n_b,
                               const double *b, double *S_re, double *S_im, double *alpha_sum, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RMS_H */
