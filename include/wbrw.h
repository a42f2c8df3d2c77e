/*
 * wbrw.h -- C ABI of the GB300 (sm_103a) signed-particle Wigner branching
 * random walk.
 *
 * The method is that of Xiong & Shao, "The Wigner branching random walk:
 * efficient implementation and performance evaluation" (arXiv:1709.02121):
 * signed particles of the Wigner equation (Eq. 1) with the kernel V_W of Eq. 2
 * are propagated interval by interval (Alg. 1) and resampled every T_A steps,
 * either by annihilation in the signed histogram (sp1, Eq. signed_histogram)
 * or by the signed residual bootstrap (sp2, Alg. 2 with Eq. lambda,
 * double_bootstrap and boostrap_histogram), followed by importance sampling
 * from the histogram (Alg. 3).
 *
 * Conventions
 *  - Every call returns a wbrw_status.  Plain C types only; no exception ever
 *    crosses this boundary.
 *  - The caller owns all device memory (particle arrays, histogram, scratch,
 *    optional event log) and the CUDA stream.  The library owns only the
 *    opaque context.  It never allocates, reallocates or frees device memory.
 *  - All GPU work is enqueued on the caller's stream.  wbrw_init, wbrw_step,
 *    wbrw_annihilate and wbrw_run do not wait for the GPU.  wbrw_density,
 *    wbrw_particles, wbrw_counters and wbrw_sync_status synchronise the stream.
 *  - Device-side faults are latched in a device error word: particle or queue
 *    capacity exceeded, offspring nesting too deep (WBRW_ERR_CAPACITY), or a
 *    non-finite coordinate at binning (WBRW_ERR_NUMERIC).  The next
 *    synchronising call reports them.  After any error the context refuses
 *    further work with WBRW_ERR_STATE; only wbrw_last_error and wbrw_destroy
 *    remain valid.
 *  - Random numbers are Philox4x32-10 keyed by config.seed and indexed by
 *    (particle id, step, draw).  Results therefore do not depend on the order
 *    in which the GPU processes particles.
 */
#ifndef WBRW_H
#define WBRW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wbrw_ctx wbrw_ctx; /* opaque, owned by the library */

typedef enum {
  WBRW_OK = 0,
  WBRW_ERR_ARG = -1,      /* invalid argument or configuration             */
  WBRW_ERR_CAPACITY = -2, /* particle, queue, record or nesting capacity   */
  WBRW_ERR_CUDA = -3,     /* a CUDA runtime call failed                    */
  WBRW_ERR_STATE = -4,    /* context already failed, or call out of order  */
  WBRW_ERR_TIMEOUT = -5,  /* reserved, never returned: no kernel waits on  */
                          /* another block or launch (every queue segment  */
                          /* has one producer and one consumer warp)       */
  WBRW_ERR_NUMERIC = -6   /* a non-finite position or wavevector reached   */
                          /* binning (latched by the device, reported by   */
                          /* the next synchronising call)                  */
} wbrw_status;

/* WBRW_WP: weighted particles (pairs always made with weights
 * +/- w cacc |sin|, as sp2 between its filters), resampled by the weighted
 * histogram of Eq. piecewise_constant_function (weights summed in fixed
 * point 2^-31) and Alg. 3 with its rounding step (sp2's rounding stream). */
typedef enum { WBRW_SP1_PAIR = 1, WBRW_SP2_BOOTSTRAP = 2, WBRW_WP = 3 } wbrw_strategy;
typedef enum { WBRW_FP64 = 0, WBRW_FP32 = 1 } wbrw_precision;
typedef enum { WBRW_POT_GAUSSIAN = 0, WBRW_POT_SOFT_COULOMB_2E = 1 } wbrw_potential_kind;

/* Potential.
 * WBRW_POT_GAUSSIAN (dim 2; Sec. 4.2, symmetric about xc):
 *   V(x) = H exp(-(x-xc)^2/(2 w^2)).  Its Wigner kernel (Eq. 2) is
 *   V_W(x,k) = (2/(pi hbar)) Vhat(2k) sin(2 (x-xc) k) with
 *   Vhat(q) = H w sqrt(2 pi) exp(-q^2 w^2/2).
 * WBRW_POT_SOFT_COULOMB_2E (dim 4; the Helium-like system of Example 1 with
 *   soft-Coulomb terms): two electrons at x1, x2 and a nucleus at xc,
 *   V = -H/sqrt((x1-xc)^2 + w^2) - H/sqrt((x2-xc)^2 + w^2)
 *       + ee/sqrt((x1-x2)^2 + w^2),
 *   i.e. H = Z the nuclear charge, w = a the softening length, ee the
 *   interaction strength.  Each term's kernel is
 *   (2/(pi hbar)) q Uhat(2 kappa) sin(2 y kappa), Uhat(q) = 2 K0(w |q|), with
 *   y = x1 - xc, x2 - xc or x1 - x2 and q = -H, -H or ee (Eq. M); the first
 *   two kick k1 or k2, the interaction kicks k1 by +kappa and k2 by -kappa. */
typedef struct {
  int kind;        /* wbrw_potential_kind                                   */
  double H, w, xc; /* Gaussian: height (any sign), width (> 0), centre;    */
                   /* soft-Coulomb: Z, softening a (> 0), nucleus          */
  double ee;       /* soft-Coulomb: interaction strength (Gaussian: unused) */
} wbrw_potential;

/* Problem statement (Sec. 2 and Sec. 4): hbar, mass, interval dt of the
 * time partition (Eq. def.time_partition), constant auxiliary rate gamma0
 * (Sec. 3.2; <= 0 selects the majorant rate C/2 = |H|/hbar, and values below
 * C/2 are rejected), the histogram = truncation domain K (Sec. 4.3, uniform
 * cells, x-major with k contiguous), the resampling period T_A in steps, and
 * the sample size N_alpha of the estimator (Eq. estimator). */
typedef struct {
  int dim;                  /* 2: (x, k); 4: (x1, x2, k1, k2), two electrons */
  int precision;            /* wbrw_precision: particle state and arithmetic */
  int strategy;             /* wbrw_strategy                                 */
  double hbar, mass, dt, gamma0;
  int nx, nk;               /* cells per coordinate: nx * nk (dim 2) or      */
                            /* nx^2 nk^2 (dim 4) cells, < 2^30               */
  double xmin, xmax, kmin, kmax;
  int resample_every;       /* steps per T_A for wbrw_run; 0 = never          */
  long long n_alpha;        /* N_alpha (> 0)                                 */
  unsigned long long seed;  /* Philox key                                    */
  int table_ny, table_nkappa; /* dim 4: kernel tables of table_ny y nodes x  */
                            /* table_nkappa kappa cells (0: 4096 x 2048)     */
  int tangent;              /* 1: carry likelihood-ratio tangents d/dH, d/dw */
                            /* (dim 2, sp1, Gaussian kind; see               */
                            /* wbrw_transmission_gradients)                  */
  double tangent_quantum;   /* largest |tau| of a tangent particle (<= 0: 1) */
} wbrw_config;

/* Caller-owned device buffers, structure of arrays, `capacity` elements each
 * (1 <= capacity <= WBRW_MAX_CAPACITY, else WBRW_ERR_ARG at init):
 *   x, k : positions and wavevectors, double (WBRW_FP64) or float (WBRW_FP32);
 *          dim 4: 2*capacity elements each (see wbrw_init4d)
 *   s    : signs +1 / -1 (int8)
 *   w    : signed weights (sp2 and wp; same type as x; NULL for sp1)
 *   grid : nx*nk int32 signed counts c_nu (grid_cells >= nx*nk), valid after
 *          a resampling
 *   scratch : >= wbrw_scratch_bytes(config, capacity) bytes, 256-byte aligned
 *   event_log : optional (NULL disables): event_log_capacity wbrw_event
 *          records of accepted events, for parity checks.
 * The arrays stay owned by the caller.  Between calls they hold the current
 * particles only after wbrw_step or wbrw_particles; wbrw_run keeps the
 * particle state implicit in the histogram. */
#define WBRW_MAX_CAPACITY 4293918720LL /* 2^32 - 2^20: slots index in 32 bits */
typedef struct {
  void* x;
  void* k;
  signed char* s;
  void* w;
  long long capacity;
  int* grid;
  long long grid_cells;
  void* scratch;
  size_t scratch_bytes;
  void* event_log;
  long long event_log_capacity;
  void* tangent;   /* tangent mode: 2*capacity doubles, tau_H of slot i at  */
                   /* [i] and tau_w at [capacity + i] (else NULL)           */
} wbrw_buffers;

/* One accepted branching event (Alg. 1 item 3), as logged for parity tests.
 * kappa is the oriented kick: the + child is at k + kappa, the - child at
 * k - kappa (dim 4: k +/- kappa e_comp with e_0 = (1,0), e_1 = (0,1),
 * e_2 = (1,-1)).  factor: dim 2, cacc |sin(2 (xe - xc) kappa)|; dim 4, the
 * probability xi_h(y)/gamma_comp that the death made a pair.  xe2 is the
 * second electron's position (dim 4; dim 2 repeats xe). */
typedef struct {
  unsigned long long pid, pid_plus, pid_minus;
  unsigned int step, j;
  double t, xe, kappa, factor;
  int kill_plus, kill_minus;
  double xe2;
  int comp, pad;
} wbrw_event;

/* Counter slots returned by wbrw_counters. */
enum {
  WBRW_C_LIVE = 0,        /* materialised particles (or implied by the grid) */
  WBRW_C_EVENTS = 1,      /* accepted events (pairs emitted), cumulative     */
  WBRW_C_KILL_PLUS = 2,   /* + offspring killed outside K, cumulative        */
  WBRW_C_KILL_MINUS = 3,
  WBRW_C_OUT_PLUS = 4,    /* + particles outside the grid at resampling      */
  WBRW_C_OUT_MINUS = 5,
  WBRW_C_PARTICLE_STEPS = 6, /* sum over steps of particles alive at start   */
  WBRW_C_LOG_LEN = 7,     /* events written to event_log                     */
  WBRW_C_STEP = 8,        /* index of the next interval                      */
  WBRW_C_EPOCH = 9,       /* resamplings so far                              */
  WBRW_C_LAUNCHES = 10,   /* kernels launched by this context                */
  WBRW_C_BOOT_NPLUS = 11, /* last sp2 filter: N^+, N^-, N_r^+, N_r^-          */
  WBRW_C_BOOT_NMINUS = 12,
  WBRW_C_BOOT_NRPLUS = 13,
  WBRW_C_BOOT_NRMINUS = 14,
  WBRW_C_BOOT_WPLUS = 15, /* last sp2 filter: W^+ and W^- in Q1.31           */
  WBRW_C_BOOT_WMINUS = 16,
  WBRW_C_NONZERO_CELLS = 17,
  WBRW_C_ERROR = 18,      /* device error word                               */
  WBRW_C_PARTICLE_STEPS_FIRST = 19, /* the part carried by the first wave of  */
                                    /* each chunk (particles present at its start) */
  WBRW_C_CANDIDATES = 20, /* candidate intervals, cumulative: a particle alive */
                          /* at the start of an interval has its first event   */
                          /* inside it (probability 1 - exp(-gamma0 dt), Sec. 3.2) */
  WBRW_C_FIRST_PAIRS = 21, /* of those, the first events that emitted a pair  */
  WBRW_C_COUNT = 24
};

/* Scratch bytes the library needs for `capacity` particles of `config`.
 * Returns 0 for an invalid configuration. */
size_t wbrw_scratch_bytes(const wbrw_config* config, long long capacity);

/* Create a context and draw n_init initial particles from the Wigner
 * function of a Gaussian wavepacket,
 *   f0(x,k) = (1/pi) exp(-(x-x0)^2/(2 sigma_x^2) - 2 sigma_x^2 (k-k0)^2),
 * which is positive: x ~ N(x0, sigma_x^2), k ~ N(k0, 1/(4 sigma_x^2)),
 * sign +1 (Sec. 4.1: f0 is its own instrumental density).
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).  On success
 * *out receives the context; on failure *out is NULL and the status says
 * why. */
wbrw_status wbrw_init(const wbrw_config* config, const wbrw_potential* pot,
                      const wbrw_buffers* buffers, long long n_init,
                      double x0, double sigma_x, double k0, void* cuda_stream,
                      wbrw_ctx** out);

/* The 4D Helium-like system (config->dim = 4, pot->kind =
 * WBRW_POT_SOFT_COULOMB_2E, sp1): draw n_init particles from the product of
 * two Gaussian-wavepacket Wigner functions (electron e: x0[e], sigma_x,
 * k0[e]), sign +1.  The kernel tables are built on the device from the
 * definition above: rows at y_i = -Y + i 2Y/(table_ny - 1) with Y = xmax - xmin
 * (one-body) or 2 (xmax - xmin) (interaction), cells
 * kappa_j = -K + (j + 1/2) 2K/table_nkappa with K = kmax - kmin, values
 * max(V_W(y_i, kappa_j), 0) and their running sums along each row,
 * xi_i = (row sum) dkappa.  Each component's rate is the smallest multiple
 * of 2^-10 at or above its largest xi_i; deaths come at the total rate
 * Gamma = 2 gamma_onebody + gamma_interaction (Sec. 3.2), pick a component
 * in proportion to its rate, and make a pair with probability
 * xi_h(y)/gamma (xi_h linear between rows, clamped outside them), the kick
 * drawn by inverse CDF of the interpolated row (Eq. def.xi_m and Sec. 4.2).
 * Buffers: x and k hold 2*capacity elements each (electron 1 in
 * [0, capacity), electron 2 in [capacity, 2 capacity)); grid holds
 * nx^2 nk^2 cells, cell ((ix1 nx + ix2) nk + ik1) nk + ik2.  Synchronises
 * the stream once (the tables' maxima).  Otherwise as wbrw_init. */
wbrw_status wbrw_init4d(const wbrw_config* config, const wbrw_potential* pot,
                        const wbrw_buffers* buffers, long long n_init, const double x0[2],
                        double sigma_x, const double k0[2], void* cuda_stream,
                        wbrw_ctx** out);

/* A time-dependent potential (Remark 1; dim 2): the sum of ncomp
 * (1..WBRW_MAX_COMPONENTS) Gaussian components
 *   V_m(x, t) = (a + b cos(omega t + phase)) exp(-(x - xc)^2 / (2 w^2)),
 * t the absolute time t_l + tau of an event.  Each component's kernel is that
 * of the Gaussian barrier with height H_m(t) (Eq. 2).  Its majorant rate is
 * gamma_m = (|a| + |b|)/hbar >= C_m(t)/2 for every t; the life-length clock
 * runs at Gamma = sum gamma_m (config->gamma0 is ignored).  A death picks
 * component m with probability gamma_m/Gamma and makes a pair with
 * probability |H_m(t)|/(hbar gamma_m) |sin(2 (x - xc) kappa)|, the kick
 * kappa ~ N(0, (1/(2w))^2) oriented by the sign of H_m(t) sin (sp2/wp: the
 * pair's weights carry that factor instead).  Otherwise as wbrw_init. */
#define WBRW_MAX_COMPONENTS 4
typedef struct {
  double a, b, omega, phase, w, xc;
} wbrw_component;

wbrw_status wbrw_init_td(const wbrw_config* config, int ncomp, const wbrw_component* comps,
                         const wbrw_buffers* buffers, long long n_init, double x0,
                         double sigma_x, double k0, void* cuda_stream, wbrw_ctx** out);

/* Advance nsteps intervals [t_l, t_{l+1}] (Alg. 1) without resampling and
 * leave the particles in the caller's arrays (offspring appended).  Async. */
wbrw_status wbrw_step(wbrw_ctx* ctx, int nsteps);

/* Resample now: sp1 signed histogram, or sp2 signed bootstrap + histogram +
 * Alg. 3 rounding, into buffers.grid.  The particle set becomes the one
 * Alg. 3 regenerates from the grid.  A second call with no step in between
 * does nothing.  Async. */
wbrw_status wbrw_annihilate(wbrw_ctx* ctx);

/* Advance nsteps intervals and resample whenever the interval index reaches
 * a multiple of config.resample_every (the schedule of Sec. 4.3 with period
 * T_A).  Each period fuses regeneration, flight and histogram in one pass, so
 * particles only reach the arrays if nsteps ends between two resamplings.
 * FP64: equivalent, bit for bit, to the same sequence of wbrw_step and
 * wbrw_annihilate.  FP32: equivalent in law; a regenerated particle takes
 * its first candidate interval from the bits of its regeneration draw in a
 * fused period and from a draw of its own once it is materialised in the
 * arrays, so the two sequences draw different (equally distributed)
 * numbers.  Async. */
wbrw_status wbrw_run(wbrw_ctx* ctx, int nsteps);

/* Observables (Eq. estimator) of the current state:
 *   density_host [nx*nk]: c_nu / (N_alpha dx dk)   (or NULL)
 *   marginal_x_host [nx]: sum_k c_nu / (N_alpha dx) (or NULL)
 *   transmission: sum over cells with centre x > 0 of c_nu / N_alpha
 *   live_particles: particles now (or NULL)
 * For dim 4 these are electron 1's: the counts summed over (x2, k2) give
 * the reduced Wigner function f1(x1, k1), its x1-marginal, and the
 * probability of x1 > 0.
 * After a resampling c_nu is the grid.  Otherwise the current particles are
 * histogrammed on the fly (sp2: signed weights in Q1.31) without changing
 * the state.  The outputs are host memory; pinned (page-locked) buffers
 * take the copies at full speed, pageable ones through a staging copy.
 * Synchronises the stream. */
wbrw_status wbrw_density(wbrw_ctx* ctx, double* density_host,
                         double* marginal_x_host, double* transmission,
                         long long* live_particles);

/* Materialise the particles into the caller's arrays (regenerating them from
 * the grid if needed), write their count to *n_host and, if pid_dev is not
 * NULL, their 64-bit stream ids to pid_dev[0..n) (device memory).
 * Synchronises the stream. */
wbrw_status wbrw_particles(wbrw_ctx* ctx, long long* n_host,
                           unsigned long long* pid_dev);

/* Checkpoint.  The histogram is the whole state of the method between two
 * periods (the pipeline of Sec. 4).  Right after a
 * resampling, copy the signed counts c_nu (nx*nk int32, x-major) to grid_out,
 * which may be host or device memory, and return the interval index and the
 * number of resamplings so far.  Returns WBRW_ERR_STATE if the particles have
 * moved since the last resampling.  Synchronises the stream. */
wbrw_status wbrw_checkpoint(wbrw_ctx* ctx, int* grid_out, long long* step,
                            long long* epoch);

/* Resume from a checkpoint: load the counts c_nu (host or device memory,
 * nx*nk int32), the interval index and the resampling count.  The particle
 * set becomes the regeneration of that histogram by Alg. 3, so a resumed run
 * is bit-identical to the uninterrupted one.  Ledger counters are kept.
 * Async. */
wbrw_status wbrw_restore(wbrw_ctx* ctx, const int* grid, long long step,
                         long long epoch);

/* Timing of the flight kernel that carries the particles present at the
 * start of each chunk of intervals.  This is the first wave of every chunk,
 * and in wbrw_run it is the fused regeneration + flight + histogram pass.
 * While enabled, each such launch is bracketed by CUDA events recorded on a
 * side stream of the context that waits for the context stream's work so far
 * (a record in the stream's own order would delay the next kernel by several
 * microseconds); at most 4096 launches are kept.  wbrw_profile_read
 * synchronises both streams and returns the summed milliseconds and the launch
 * count since the last read or enable.  Errors: WBRW_ERR_ARG for a null
 * context, WBRW_ERR_CUDA if an event or the side stream cannot be created. */
wbrw_status wbrw_profile(wbrw_ctx* ctx, int enable);
wbrw_status wbrw_profile_read(wbrw_ctx* ctx, double* total_ms,
                              long long* launches);

/* The same for the event kernel, which performs the first event of every
 * candidate interval (WBRW_C_CANDIDATES counts them): while wbrw_profile is
 * enabled each of its launches is bracketed by CUDA events on the context's
 * stream (at most 4096 launches are kept; in a CUDA-graph replay, those of
 * the period's first 64 rounds).  wbrw_profile_read_events synchronises and
 * returns the summed milliseconds and the launch count since the last read
 * or enable. */
wbrw_status wbrw_profile_read_events(wbrw_ctx* ctx, double* total_ms,
                                     long long* launches);

/* CUDA graphs for wbrw_run.  With enable = 1, each resampling period that
 * regenerates its particles from the histogram (every period but one that
 * starts from the initial particles or from wbrw_step) is captured into a
 * CUDA graph the first time a period of its length runs, and replayed after
 * that: one launch per period instead of one per kernel.  This holds for
 * every strategy (sp1, sp2, wp).  Results are bit for bit those of
 * enable = 0 (the kernels read the period's first interval and id base from
 * device memory, the resampling kernels the epoch of the histogram they make,
 * and the graph advances them).  The context stream must be a created stream
 * (not the legacy or per-thread default stream) and must not be capturing;
 * otherwise WBRW_ERR_ARG.  enable = 0 synchronises the stream and releases
 * the graphs.  The CUDA events of wbrw_profile are part of a
 * graph only if profiling was on when it was captured (each event costs a
 * few microseconds per replay), so the first replay after wbrw_profile
 * switches profiling on or off captures its period again. */
wbrw_status wbrw_graph(wbrw_ctx* ctx, int enable);

/* Schedule of the periods that regenerate from the histogram under sp1 or
 * wp (sp2 periods always run launch per round), in contexts whose kernels
 * can run a period as one launch: the 2D FP32 contexts with the static
 * potential and no event log (tangent mode included) and the FP32 4D
 * contexts.  enable = 1 (the default): the first
 * wave (or waves) and every event round of a period run in one kernel
 * launch, each warp on its own candidate segments (Alg. 1 over the period,
 * the resampling of Sec. 4.3 after it).  enable = 0: the launch-per-round
 * schedule, a first-wave launch and one event launch per round.  The
 * results are the same bit for bit (random numbers are keyed by particle
 * and interval); only the launches and the time differ.  Other contexts
 * accept the call and always run launch per round.  Takes effect from the
 * next period; releases captured graphs (synchronises the stream).
 * WBRW_ERR_ARG for a NULL context, WBRW_ERR_STATE after a failure. */
wbrw_status wbrw_one_launch_periods(wbrw_ctx* ctx, int enable);

/* Launch shape.  Neither knob changes any result (random numbers are keyed
 * by particle and interval, and every count is an integer sum), only speed:
 *   blocks_per_sm : resident 256-thread blocks per SM of the particle
 *                   kernels, from 1 to the context's maximum (default that
 *                   maximum): 4 for 2D FP32 contexts (plain or batched)
 *                   with the static potential, no event log and no
 *                   tangents, and for the FP32 4D model, whose kernels are
 *                   built for 64 registers; 3 for the others
 *                   (WBRW_TUNE_BLOCKS_PER_SM_MAX is the largest).
 *                   Each warp owns one segment of every queue, so this also
 *                   sets the queue segmentation.
 *   event_passes  : offspring with further events in their interval are
 *                   processed one event per lockstep pass for this many
 *                   passes (0..WBRW_TUNE_PASSES_MAX, default 3); what remains
 *                   is finished by one recursive pass.  The 2D FP32
 *                   contexts with the static potential and no event log
 *                   (those with four blocks per SM above, and the same in
 *                   tangent mode) and the FP32 4D contexts finish every such
 *                   segment in lockstep passes inside the event kernel
 *                   itself, so there event_passes changes nothing; their
 *                   regenerating sp1 and wp periods run in one launch (first
 *                   waves and event rounds together), at most three blocks
 *                   per SM.
 * wbrw_set_tuning takes effect from the next call and releases captured
 * graphs; out-of-range values (including blocks_per_sm above the context's
 * maximum) give WBRW_ERR_ARG. */
#define WBRW_TUNE_BLOCKS_PER_SM_MAX 4
#define WBRW_TUNE_PASSES_MAX 6
typedef struct {
  int blocks_per_sm;
  int event_passes;
} wbrw_tuning;

wbrw_status wbrw_get_tuning(wbrw_ctx* ctx, wbrw_tuning* out);
wbrw_status wbrw_set_tuning(wbrw_ctx* ctx, const wbrw_tuning* tuning);

/* Autotuner: time one resampling period of wbrw_run (the period that starts
 * now) under every setting, `trials` times each (>= 1), keep the fastest
 * setting and report it in *best (may be NULL).  ms_table (may be NULL)
 * receives WBRW_TUNE_BLOCKS_PER_SM_MAX x (WBRW_TUNE_PASSES_MAX + 1) times in
 * milliseconds, entry (b - 1) * (WBRW_TUNE_PASSES_MAX + 1) + p for
 * blocks_per_sm = b and event_passes = p, each the fastest of its trials
 * (negative if that setting hit a capacity limit, lies above the
 * context's maximum blocks_per_sm, or has event_passes > 0 in a context
 * where event_passes changes nothing, which is timed only at 0).  Every trial starts from
 * the same histogram, and the context is put back afterwards: state, counters
 * and interval index are as before the call.  Needs the state right after a
 * resampling (as wbrw_checkpoint) and resample_every > 0; the event log is
 * not written while tuning.  Synchronises the stream. */
wbrw_status wbrw_autotune(wbrw_ctx* ctx, int trials, wbrw_tuning* best, double* ms_table);

/* Observables of a signed histogram without any allocation and without a
 * context.  The paper has no counterpart: this is an interface for callers
 * that cannot call cudaMalloc, such as code running inside a fixed device
 * memory pool owned by someone else, or a host process that is not allowed to
 * grow the device footprint after start-up.  Such callers cannot hand the
 * library a scratch buffer on every call.  It computes what wbrw_density
 * computes from a histogram (density c_nu/(N_alpha dx dk), x-marginal, and
 * the transmission over cells with centre x > 0) for the counts `grid`
 * (nx*nk int32, x-major, device memory).  Outputs are device memory owned by
 * the caller: density (nx*nk doubles, or NULL), marginal_x (nx doubles) and
 * transmission (1 double).  Work is enqueued on cuda_stream; nothing waits.
 *
 * Its only scratch, the per-column sums, lives in a static device array of
 * WBRW_STATIC_MAX_NX int64 entries (512 KiB) that every GPU loading the
 * library keeps until the process exits.  nx above that maximum is refused
 * with WBRW_ERR_CAPACITY.  Invalid arguments give WBRW_ERR_ARG, and so does
 * any non-NULL buffer that is not device (or managed) memory of the current
 * device: host memory or another GPU's buffer is refused before any launch.
 * The first call on each device looks up the array's device address on that
 * device and keeps it (make that first call before any stream capture).
 * The address is not looked up again, so calls after a cudaDeviceReset in
 * the same process are not supported.  All calls share the array: calls
 * whose GPU work overlaps (other streams, other threads) race and must be
 * serialised by the caller.  Each call overwrites every entry it reads, so
 * nothing needs clearing between calls.  A launch failure gives
 * WBRW_ERR_CUDA; the check also consumes, and reports, an error that an
 * earlier runtime call of the caller left pending. */
#define WBRW_STATIC_MAX_NX 65536
wbrw_status wbrw_observables_static(const int* grid, int nx, int nk,
                                    double xmin, double xmax, double kmin,
                                    double kmax, long long n_alpha,
                                    double* density, double* marginal_x,
                                    double* transmission, void* cuda_stream);

/* Measurement aid: the Philox4x32-10 call of the flight and event kernels
 * (Salmon et al., SC'11; keyed by `seed`), run in a dependent chain of
 * `iters` calls by each of `nthreads` threads (each call's output is the
 * next call's counter), with nothing else around it.  Its call rate,
 * nthreads * iters / (the kernel's time on cuda_stream), is the integer-pipe
 * ceiling of the hot path's random numbers: the peak that the integer-bound
 * kernels are compared against.  out: nthreads uint32 in device memory of
 * the current device (the XOR of each thread's last output), else
 * WBRW_ERR_ARG.  Async; no context.  The paper has no counterpart. */
wbrw_status wbrw_philox_chain(unsigned long long seed, int iters, long long nthreads,
                              unsigned int* out, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batches: many independent problems in the same launches.
 *
 * The paper treats one problem at a time; running many of them side by side
 * is an extension for throughput.  Each instance of a batch is the run that
 * wbrw_init would make for its own potential, initial wavepacket, rate and
 * N_alpha, with the shared config (hbar, mass, dt, grid, resample_every,
 * seed, precision) -- except that its particles are labelled
 * (instance << 32) | index at start and (epoch << 40) | (instance << 32) | j
 * after a resampling, so instances draw from disjoint random streams.
 * Instance 0 of a batch is therefore bit-identical to the plain run.
 *
 * The histogram buffer holds the instances one after the other:
 * instance i owns grid[i*nx*nk .. (i+1)*nx*nk), x-major with k contiguous;
 * buffers.grid_cells >= ninst*nx*nk, and ninst*nx*nk < 2^30.  The particle
 * arrays are shared: initial particles of instance i occupy the slots after
 * those of instances 0..i-1.  Every strategy runs in a batch: sp2
 * bootstraps each instance on its own (Alg. 2 per instance and side, with
 * the shares of that instance's N^s and W^s), and the residual draws and
 * the roundings of sp2 and wp are counted (instance << 32) | d and
 * (instance << 32) | (cell within the instance), salt 0 being the plain
 * run's.  The sp2 counters of wbrw_counters are then sums over instances.
 * wbrw_step, wbrw_annihilate, wbrw_run, wbrw_particles, wbrw_checkpoint
 * (all instances' counts), wbrw_restore, wbrw_counters (sums over
 * instances), wbrw_profile and wbrw_destroy work on a batch unchanged;
 * wbrw_density reports instance 0.
 * ------------------------------------------------------------------------ */
#define WBRW_MAX_INSTANCES 256

typedef struct {
  wbrw_potential pot;       /* the instance's potential                      */
  double x0, sigma_x, k0;   /* initial Gaussian wavepacket (see wbrw_init)   */
  long long n_init;         /* initial particles, 0 .. 2^32 - 1              */
  long long n_alpha;        /* N_alpha of its estimator (> 0)                */
  double gamma0;            /* <= 0: the majorant rate C/2 of its potential  */
} wbrw_instance;

/* Scratch bytes for a batch of ninst instances sharing `capacity` particle
 * slots (config->gamma0 and config->n_alpha are ignored).  0 if invalid. */
size_t wbrw_batch_scratch_bytes(const wbrw_config* config, int ninst, long long capacity);

/* Create a batch context: ninst (1..WBRW_MAX_INSTANCES) instances described
 * by inst[0..ninst) (host memory, copied), initial particles drawn as in
 * wbrw_init.  Sum of n_init <= buffers.capacity.  Async; *out as in
 * wbrw_init. */
wbrw_status wbrw_batch_init(const wbrw_config* config, int ninst, const wbrw_instance* inst,
                            const wbrw_buffers* buffers, void* cuda_stream, wbrw_ctx** out);

/* wbrw_density for instance `instance` of a batch (0 for a plain context):
 * density and marginal from its own cells and N_alpha, its transmission and
 * its live particle count.  Synchronises the stream. */
wbrw_status wbrw_instance_density(wbrw_ctx* ctx, int instance, double* density_host,
                                  double* marginal_x_host, double* transmission,
                                  long long* live_particles);

/* Transmission (Eq. estimator with A = 1{x > 0}) of every instance, read
 * from the histogram right after a resampling: out_host[0..ninst).
 * WBRW_ERR_STATE if the particles moved since.  Synchronises the stream. */
wbrw_status wbrw_transmissions(wbrw_ctx* ctx, double* out_host);

/* After wbrw_particles: the instance of every materialised particle,
 * inst_dev[0..n) (device memory).  Synchronises the stream. */
wbrw_status wbrw_particle_instances(wbrw_ctx* ctx, unsigned int* inst_dev);

/* ------------------------------------------------------------------------
 * Likelihood-ratio derivatives (config->tangent = 1).  The paper has no
 * differentiation; this is an extension.  The expected particle measure of
 * the branching walk is a sum over lineages of products of the birth
 * intensities V_W^+(x_b, kappa_b; theta) (a parent outlives its births, so no
 * survival factor enters).  Each particle therefore carries a tangent weight
 * tau = s S: its sign times the sum, over the births of its lineage, of
 * g = d/dtheta log V_W^+ = (1/H, 1/w - 4 w kappa^2), theta = (H, w).  A birth
 * from (s, tau) gives the + child (s, tau + s g) and the - child
 * (-s, -(tau + s g)).  Then d/dtheta E[sum_i s_i A(x_i, k_i)] =
 * E[sum_i tau_i A(x_i, k_i)].  Annihilation also sums the tangent histogram
 * D_nu (tau rounded to multiples of 2^-32, exact and order-free) and
 * regeneration carries it on particles of sign 0: ceil(max(|D_H|, |D_w|) /
 * tangent_quantum) per cell with tau = D_nu / count, ids
 * (epoch << 40) | (instance << 32) | 2^31 | j.  The signed particles, their
 * ids and every count are exactly those of the run without tangents.
 * Batches differentiate each instance in its own (H, w).  wbrw_restore loads
 * no tangent (the restored run has D = 0).
 * ------------------------------------------------------------------------ */

/* (dT/dH, dT/dw) of every instance's transmission estimate
 * (sum over cells with centre x > 0 of D_nu / N_alpha), right after a
 * resampling: out_host[2 i], out_host[2 i + 1].  Synchronises the stream. */
wbrw_status wbrw_transmission_gradients(wbrw_ctx* ctx, double* out_host);

/* Copy the counters (WBRW_C_*) to out[0..WBRW_C_COUNT).  Synchronises. */
wbrw_status wbrw_counters(wbrw_ctx* ctx, long long* out);

/* Synchronise the stream and report the device error word. */
wbrw_status wbrw_sync_status(wbrw_ctx* ctx);

/* Human-readable description of the last error of ctx (never NULL). */
const char* wbrw_last_error(const wbrw_ctx* ctx);

/* Release the context (not the caller's buffers).  NULL is allowed. */
void wbrw_destroy(wbrw_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* WBRW_H */
