/*
 * lbm_mix.h — C ABI of the GB300 (sm_103a) two-species lattice Boltzmann hot
 * path for a rarefied binary gas mixture in a pressure-driven microchannel.
 *
 * Method: Wang, Xu & Guo, "Lattice Boltzmann simulation of separation
 * phenomenon in a binary gaseous flow through a microchannel"
 * (arXiv:1603.08221), Sec. 3: D2Q9 multiple-relaxation-time LBE for each
 * species (Eqs. MRT, MR, m, S, feq, rhou), Knudsen-dependent effective
 * relaxation times (Eqs. EQFrb, EQFrsp, psi, taos), diffuse-bounce-back walls
 * (Eqs. bot, bot2, R, taoq, A12) and extrapolation-correction pressure ends
 * (Eqs. rho1, rho2); separation diagnostics of Sec. 2 (Eqs. C, CL, Clline).
 *
 * Conventions for every call:
 *  - Lattice units: dx = dt = 1, c_s^2 = k_B T / m_min = 1/3, masses
 *    normalised by m_min, outlet number density 1, channel height H = N.
 *  - The lattice has N rows (j = 0 .. N-1; the bottom wall sits half a cell
 *    below row 0, the top wall half a cell above row N-1) and N_x columns
 *    (x = 0 .. N_x-1).  With pressure ends, columns 0 and N_x-1 are the
 *    inlet and outlet boundary columns and columns 1 .. N_x-2 are updated.
 *  - Host arrays laid out [row][column] hold N*N_x doubles; population arrays
 *    are [species][i][row][column] (2*9*N*N_x floats), species a first,
 *    velocities c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
 *    (-1,-1),(1,-1).
 *  - Every function returns LBM_OK (0) or a negative LBM_E* code and, on
 *    error, sets a thread-local message readable with lbm_mix_last_error().
 *  - A handle is used by one host thread at a time.  Work is enqueued on the
 *    handle's CUDA stream; getters synchronise that stream, lbm_mix_step
 *    does not.
 */
#ifndef LBM_MIX_H
#define LBM_MIX_H

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)         /* bad argument or parameter */
#define LBM_ENOMEM (-2)         /* device or host allocation failed */
#define LBM_ECUDA (-3)          /* CUDA runtime error (message has details) */
#define LBM_ENONFINITE (-4)     /* a non-finite density or mass appeared */
#define LBM_ENOTCONVERGED (-5)  /* run_to_steady hit max_steps */
#define LBM_ETIMEOUT (-6)       /* reserved: a bounded device wait expired */

/* Population storage.  Every form stores deviations from the rest
 * equilibrium of a per-column reference density and computes in FP32. */
#define LBM_FP32 0 /* FP32 deviations (144 B per node per step) */
#define LBM_BF16 1 /* BF16 deviations (72 B per node per step) */
#define LBM_FP16 2 /* FP16 deviations (72 B per node per step) */

/* Rounding of the BF16/FP16 stores of the step.  Round to nearest repeats
 * the same rounding error every step once the flow is steady, and the
 * collision conserves the momentum that error carries, so it accumulates
 * into a bias of the velocity field; stochastic rounding makes each
 * rounding error zero-mean and independent of the previous step's. */
#define LBM_ROUND_STOCHASTIC 0 /* default: stochastic rounding (hardware cvt.rs) */
#define LBM_ROUND_NEAREST 1    /* round to nearest even */

/* Wall rule.  The paper's diffuse bounce-back (Eqs. bot, bot2) with r of
 * Eq. R, or the bounce-back and specular-reflection scheme it validates
 * against (Method validation section): an unknown population is the
 * fraction r_b = 1/(1 + X) of its bounced-back partner at the node plus
 * 1 - r_b of its specularly reflected partner from the upstream neighbour
 * column, X the slip factor of Eq. R (r = 2 - 2/(1 + X)); both give the
 * first-order slip c_m lambda du/dn, and with tau_q of Eq. taoq the BSR
 * scheme also gives the second-order term of Eq. A12 exactly. */
#define LBM_WALL_DBB 0 /* default */
#define LBM_WALL_BSR 1

/* Readings of Eq. R, whose two printed forms disagree for unequal masses
 * (masses in units of m_min; all three agree when m_a = m_b):
 * r_s = 2 - 2/(1 + X_s) with X_s = c_m sqrt(pi m_x / 6) for both species
 * (the first form, the default), c_m sqrt(pi m_x / (6 m_s)) (m_min of the
 * first form replaced by the species mass) or c_m sqrt(pi m_x^2 / (6 m_s))
 * (the second form, with m_r = m_s / m_x). */
#define LBM_R_FIRST 0
#define LBM_R_SPECIES 1
#define LBM_R_SECOND 2

typedef struct lbm_mix lbm_mix; /* opaque, owned by the library */

/* Physical problem (Sec. 2, Table 1) and model knobs (Sec. 3). */
typedef struct {
  double m_a, m_b;      /* molecular masses, any common unit, > 0 */
  double C_l;           /* light-species mole fraction at the inlet, (0,1) */
  double C_l_out;       /* at the outlet; < 0 means equal to C_l */
  double theta;         /* P_in / P_out >= 1 */
  double Kn_out;        /* lambda_out / H > 0 */
  int N;                /* lattice cells across H, >= 2 */
  int N_x;              /* lattice columns; <= 0 means round(N * L_over_H) */
  double L_over_H;      /* channel aspect ratio, used when N_x <= 0 */
  double accommodation; /* uniform wall accommodation alpha in (0,1] (Eq. A12) */
  double c_m0;          /* velocity slip coefficient at alpha = 1 (Eq. R);
                           scaled by (2 - alpha)/alpha per wall node */
  double tau_rho, tau_e, tau_eps; /* fixed relaxation times (Sec. 3.3) */
  double mu_ratio_a, mu_ratio_b;  /* mu_sigma / mu of the mixture */
  int storage;          /* LBM_FP32, LBM_BF16 or LBM_FP16 */
  int x_periodic;       /* 1: periodic in x instead of pressure ends */
  int diag_every;       /* >= 1: steps between separation-diagnostic reductions */
  int reref_every;      /* steps between re-referencings of the stored deviations
                           (lbm_mix_rereference); 0 = never; -1 = 256 for BF16/FP16
                           storage and never for FP32 */
  int rounding;         /* BF16/FP16 stores: LBM_ROUND_STOCHASTIC or LBM_ROUND_NEAREST
                           (FP32 storage ignores it) */
  int wall;             /* LBM_WALL_DBB or LBM_WALL_BSR */
  int r_form;           /* LBM_R_FIRST, LBM_R_SPECIES or LBM_R_SECOND (Eq. R) */
  int lambda_pressure;  /* species mean free path lambda_s = (mu_s / p') sqrt(pi
                           k_B T / (2 m_s)) with p' the partial pressure x_s p
                           (0, default) or the mixture pressure p (1) */
} lbm_mix_params;

/* Fills the defaults: He-Ar (4.003, 39.948), C_l = 0.5, C_l_out = -1,
 * theta = 2, Kn_out = 0.1, N = 16, N_x = 0, L_over_H = 20, alpha = 1,
 * c_m0 = 1.016, tau_rho = 1, tau_e = 1.1, tau_eps = 1.2, mu ratios 1,
 * LBM_FP32, x_periodic = 0, diag_every = 1, reref_every = -1,
 * rounding = LBM_ROUND_STOCHASTIC, wall = LBM_WALL_DBB, r_form = LBM_R_FIRST,
 * lambda_pressure = 0.  NULL-safe. */
void lbm_mix_default_params(lbm_mix_params* p);

/* Validates p, derives the lattice constants (Eqs. P, EQFrb, rho2 with the
 * outlet mean free path Kn_out * N), allocates the two population buffers
 * and the reduction buffers on the current CUDA device and returns a handle
 * in *out.  stream: a cudaStream_t to enqueue on, or NULL for a stream owned
 * by the handle.  No device work is done besides allocation.  Parameters are
 * checked before any CUDA call, so LBM_EINVAL needs no GPU.  Errors:
 * LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA; *out is NULL on error. */
int lbm_mix_create(const lbm_mix_params* p, void* stream, lbm_mix** out);

/* Releases every resource of h. NULL-safe. */
void lbm_mix_destroy(lbm_mix* h);

/* Initial state: pressure linear from theta * p_out (column 0) to p_out
 * (column N_x-1), zero velocity, light mole fraction linear from C_l to
 * C_l_out, populations at equilibrium (Eq. feq).  Resets the step count. */
int lbm_mix_init(lbm_mix* h);

/* Advances nsteps >= 0 time steps (Eq. MRT), one fused collide-stream pass
 * per step on the handle's stream, asynchronously.  With 16-bit storage, and
 * with FP32 storage when the step's grid holds two or more waves of CTAs on
 * the device, a small kernel computes r (Eq. R) and tau_q (Eq. taoq) of
 * every column ahead of each pass; both are launched with programmatic
 * dependent launch.  The pass of every
 * diag_every-th step (counted from init) and of the last step of the call
 * also reduces the separation diagnostics of the new state in FP64 (one
 * history record each), so lbm_mix_separation after lbm_mix_step always
 * describes the current state.  After every reref_every-th step (counted
 * from init) the stored deviations are re-referenced (lbm_mix_rereference). */
int lbm_mix_step(lbm_mix* h, long nsteps);

/* Re-references the stored state: the populations are kept as deviations
 * d_i = f_i - w_i alpha_si rhobar_s(x) from the rest equilibrium (Eq. feq,
 * u = 0) of a per-column reference density, initially the profile of
 * lbm_mix_init.  This sets rhobar_s(x) to the current column mean
 * (1/N) sum_j rho_s(x, j) of every updated column and rewrites the
 * deviations to match, so that they stay small as the flow departs from its
 * initial state: f itself changes only by one rounding of the storage type.
 * With BF16/FP16 storage the deviations' precision is relative to their
 * size, which is why lbm_mix_step does this periodically there.  One pass
 * over both population buffers plus a column reduction, asynchronous on the
 * handle's stream.  No counterpart in the paper (a storage device, not physics).
 * Errors: LBM_EINVAL for a bad handle, LBM_ECUDA. */
int lbm_mix_rereference(lbm_mix* h);

/* Steps in blocks of `check_every` (>= 1) until the steady-state residual
 * R = |c(t) - c(t-K)|_2 / (K |c(t)|_2) of the column-integrated species
 * densities and x mass flows c drops to tol, or max_steps are taken
 * (LBM_ENOTCONVERGED), or a non-finite value appears (LBM_ENONFINITE).
 * steps_out / residual_out (nullable) receive the steps taken and final R. */
int lbm_mix_run_to_steady(lbm_mix* h, double tol, long max_steps, long check_every,
                          long* steps_out, double* residual_out);

/* Macroscopic fields of the current state, FP64 host arrays [N][N_x], each
 * nullable: species densities and the species velocities of Eq. rhou,
 * rho_s u_s = (2 tau_d - 1)/(2 tau_d) sum_i c_i f_si + rho_s u / (2 tau_d).
 * Columns 0 and N_x-1 (pressure ends) hold rho_s = kappa_s (2 rho_s(1) -
 * rho_s(2)) with the density-correction factor of Eq. rho2, and
 * u_s = 2 u_s(1) - u_s(2).  Synchronises. */
int lbm_mix_moments(lbm_mix* h, double* rho_a, double* rho_b, double* ua_x, double* ua_y,
                    double* ub_x, double* ub_y);

/* Same fields written to caller-owned DEVICE memory d_out[6][N][N_x]
 * (rho_a, rho_b, ua_x, ua_y, ub_x, ub_y); enqueued, not synchronised. */
int lbm_mix_moments_device(lbm_mix* h, double* d_out);

/* Separation diagnostics of the current state (Eqs. C, CL, Clline), each
 * nullable: CL = (C_l,in - min_x C_l(x)) / C_l,in over the updated columns,
 * with C_l(x) = sum_j n_l / sum_j (n_a + n_b); C~_l over all N_x columns
 * (boundary columns at their imposed values); mdot_s = mean over updated
 * columns of sum_j rho_s u_s,x; Cl_profile receives N_x values; x_min the
 * column of the minimum.  Synchronises; LBM_ENONFINITE if the state holds a
 * non-finite value. */
int lbm_mix_separation(lbm_mix* h, double* CL, double* Cl_tilde, double* mdot_a,
                       double* mdot_b, double* Cl_profile, int* x_min);

/* Device pointers of the handle's current state, for zero-copy views (e.g.
 * torch tensors through __cuda_array_interface__); each output nullable:
 *   populations    the latest post-collision populations as stored: deviations
 *                  d = f - w_i alpha_si rhobar_s(x) from the rest equilibrium
 *                  (Eq. feq, u = 0), element type of the storage (float, or
 *                  2-byte BF16/FP16), strip layout
 *                  index = (x/32) * 576 N + j * 576 + i * 64 + 2 * (x%32) + sigma,
 *                  *n_populations elements (18 * N * 32 * ceil(N_x/32));
 *   refrho         rhobar_s(x), float [2][N_x];
 *   alpha          accommodation coefficients, float [2][N_x] (bottom, top);
 *   colsum         FP64 [4][N_x] column sums of the latest diagnostic step
 *                  (sum_j rho_a, sum_j rho_b, and the species x momenta).
 * The pointers stay owned by the handle and are valid until the next call
 * that steps, re-references, initialises or uploads a state (the two
 * population buffers alternate).  Reading them must be ordered after the
 * handle's stream.  No counterpart in the paper. */
int lbm_mix_device_ptrs(lbm_mix* h, void** populations, long* n_populations, void** refrho,
                        void** alpha, void** colsum);

/* Volume flow Q_v of the mixture through column x (Sec. 4.2, Fig. 7; the
 * paper gives no formula: read as the sum over the rows of the mixture
 * velocity u_x = (rho_a u_a,x + rho_b u_b,x)/(rho_a + rho_b) of Eq. rhou,
 * in lattice units).  x < 0 selects the last updated column N_x - 2 (the
 * outlet).  Synchronises.  Errors: LBM_EINVAL (x not an updated column),
 * LBM_ENONFINITE, LBM_ECUDA. */
int lbm_mix_volume_flow(lbm_mix* h, int x, double* Qv);

/* Copies up to max_records of the most recent diagnostic records, oldest
 * first, into rec[max_records][8] = {record number, CL, C~_l, mdot_a,
 * mdot_b, x_min, total mass a, total mass b}; *count gets the number copied.
 * One record per diagnostic step (see lbm_mix_step); the library keeps the
 * last 4096.  Synchronises. */
int lbm_mix_history(lbm_mix* h, double* rec, long max_records, long* count);

/* Per-wall-node accommodation coefficients alpha in (0,1] (Eq. A12):
 * n = 2*N_x values, bottom wall then top wall, host FP64. */
int lbm_mix_set_accommodation_field(lbm_mix* h, const double* alpha, long n);

/* Replaces the state by caller post-collision populations (host FP32,
 * [2][9][N][N_x], n = 18*N*N_x); the next step streams them.  Resets the
 * step count; until the next step, lbm_mix_moments reports the moments of
 * these populations themselves. */
int lbm_mix_set_post_state(lbm_mix* h, const float* f, long n);

/* Copies the current post-collision populations to host FP32 [2][9][N][N_x].
 * The library stores deviations from a per-column rest equilibrium, so a
 * set/get round trip reproduces each value to about one FP32 ulp.
 * Synchronises. */
int lbm_mix_get_post_state(lbm_mix* h, float* f, long n);

/* Same populations in FP64, [2][9][N][N_x]: the exact values the FP32
 * deviation storage represents (reference equilibrium + deviation, summed in
 * FP64).  Synchronises. */
int lbm_mix_get_post_state_f64(lbm_mix* h, double* f, long n);

/* Lattice size and steps taken since init / set_post_state. */
int lbm_mix_dims(const lbm_mix* h, int* N, int* N_x, long* steps);

/* Kernel launches of one lbm_mix_step step under h's current schedule
 * (lbm_mix_set_rows_per_block): 2 when the wall kernel runs ahead of the
 * step kernel (16-bit storage; FP32 grids of two or more waves of CTAs),
 * else 1; re-referencing adds its own.  Returns the count, or LBM_EINVAL
 * for a NULL handle. */
int lbm_mix_launches_per_step(const lbm_mix* h);

/* Waits for all work enqueued on the handle's stream. */
int lbm_mix_sync(lbm_mix* h);

/* Device evaluation (FP32) of the exponential integral E_1 = E_i of Eq. psi
 * and of psi itself at n host points x[] (> 0); writes e1[] and psi[]
 * (nullable).  Diagnostic entry point for testing the device special
 * functions; uses its own temporary device memory. */
int lbm_mix_eval_special(const double* x, double* e1, double* psi, long n);

/* One time step with no device allocation, for callers that cannot call
 * cudaMalloc (for example code that owns a fixed device-memory budget that
 * is already handed out, or runs under an allocator it does not control and
 * may not bypass).  This entry point has no
 * counterpart in the paper; it runs the fused step kernel of lbm_mix_step
 * as one launch (r and tau_q from the kernel's own wall prologue), with the
 * kernel's scratch (per-strip partial sums and the
 * arrival tickets of its two-level reduction) in a static device array of
 * 69 KB that every GPU loading the library holds until the process exits.
 * That array covers N_x <= 32768 columns; larger N_x is rejected with
 * LBM_EINVAL.  The step runs with one row block per strip.
 *
 * All buffers are caller-owned DEVICE memory, read or written on `stream`
 * (a cudaStream_t, NULL for the legacy default stream):
 *   d_in, d_out   post-collision populations before and after the step, as
 *                 FP32 deviations d = f - w_i alpha_si rhobar_s(x) from the
 *                 rest equilibrium (Eq. feq with u = 0; w_i alpha_si =
 *                 (9 - 5 s)/9, s/9, s/36 for rest, axis, diagonal
 *                 populations, s = m_min / m_sigma) of the reference density
 *                 rhobar; laid out in strips of 32 columns with the two
 *                 species of a population adjacent:
 *                 index = (x/32) * 576 N + j * 576 + i * 64 + 2 * (x%32) + sigma,
 *                 18 * N * 32 * ceil(N_x/32) floats each; must not alias;
 *   d_refrho      rhobar_s(x), [2][N_x] floats, any fixed positive profile
 *                 (the same one for every step of a run);
 *   d_alpha       accommodation coefficients, [2][N_x] floats (bottom, top);
 *   d_colsum_in   [4][N_x] doubles: column sums sum_j rho_a, sum_j rho_b of
 *                 the state in d_in (rows 2 and 3 are not read);
 *   d_colsum_out  [4][N_x] doubles written: sum_j rho_a, sum_j rho_b,
 *                 sum_j rho_a u_a,x, sum_j rho_b u_b,x of the new state;
 *   d_record      8 doubles written: {1, CL, C~_l, mdot_a, mdot_b, x_min,
 *                 total mass a, total mass b} of the new state;
 *   d_cl_profile  N_x doubles written: C_l(x) of the new state.
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is looked up again when the calling thread's current context
 * is not the one of the last lookup (after cudaDeviceReset, for example),
 * so the first call after a reset must also come before any capture.
 * Every call shares the one array and resets its counters, so calls whose
 * kernels overlap on the GPU (different streams, or different threads
 * without ordering) race and corrupt each other's results; serialise them.
 * Returns LBM_OK once the step is enqueued, LBM_EINVAL for bad parameters,
 * pointers or sizes, LBM_ECUDA for launch errors. */
int lbm_mix_step_noalloc(const lbm_mix_params* p, const float* d_in, float* d_out,
                         const float* d_refrho, const float* d_alpha, const double* d_colsum_in,
                         double* d_colsum_out, double* d_record, double* d_cl_profile,
                         void* stream);

/* Node-to-CTA schedule of h: rows of one strip handled by one CTA of the
 * step kernel, a multiple of 8 (capped at N rounded up to 8); 0 restores the
 * library default (96 rows).  Changes only the order
 * of the FP64 column reductions.  May allocate; not during stream capture.
 * Errors: LBM_EINVAL (bad handle, rows not a multiple of 8), LBM_ENOMEM,
 * LBM_ECUDA. */
int lbm_mix_set_rows_per_block(lbm_mix* h, int rows);

/* Picks the node-to-CTA schedule of h by timing real steps: for each of the
 * n candidate row counts (multiples of 8; candidates = NULL takes 64, 72,
 * 80, 88, 96, 112 and 128) it runs 2 untimed steps and `steps` steps timed
 * with CUDA events on the handle's stream, then keeps the fastest (ties to
 * the earlier candidate) and writes it to *best_rows (NULL-safe).  Which
 * count is fastest depends on how the grid's CTAs fill the device's waves,
 * so it differs between channel sizes and storage types.  The steps advance
 * the state (n * (steps + 2) of them, with their diagnostic records):
 * call lbm_mix_init or lbm_mix_set_post_state afterwards to start a run
 * from a chosen state.  Synchronises.  Not during stream capture.
 * Errors: LBM_EINVAL (bad handle, candidates or steps), LBM_ENOMEM,
 * LBM_ECUDA, and any error of lbm_mix_step. */
int lbm_mix_tune_rows(lbm_mix* h, const int* candidates, int n, long steps, int* best_rows);

/* ---------------------------------------------------------------------
 * Parametric sweeps (the study of Table 1 and Sec. 4: many independent
 * channels).  No counterpart in the paper's method: a batching device.
 *
 * A sweep owns n handles, each on its own CUDA stream.  K steps of an
 * instance are captured once as a CUDA graph and replayed, so each
 * convergence check costs the host one graph launch per instance and the
 * instances' step kernels run concurrently on the GPU.  FP32 storage only;
 * every instance's diag_every is set to the check interval.
 * ------------------------------------------------------------------- */
typedef struct lbm_sweep lbm_sweep;

/* Node-to-CTA schedules the autotuner tries: 0 library default (96 rows per
 * CTA), 1: 64, 2: 32, 3: 16 rows, 4: enough rows per CTA to give each
 * instance about two CTAs per SM. */
#define LBM_SWEEP_NPOLICY 5

/* Creates n instances from params[0..n-1] (validated like lbm_mix_create)
 * on the current device.  Errors: LBM_EINVAL (bad n, bad parameters of
 * some instance, BF16/FP16 storage), LBM_ENOMEM, LBM_ECUDA. */
int lbm_sweep_create(const lbm_mix_params* params, int n, lbm_sweep** out);

/* Releases the sweep and all its instances.  NULL-safe. */
void lbm_sweep_destroy(lbm_sweep* s);

/* lbm_mix_init on every instance. */
int lbm_sweep_init(lbm_sweep* s);

/* nsteps plain steps on every instance (each on its stream), then waits
 * for all of them. */
int lbm_sweep_step(lbm_sweep* s, long nsteps);

/* Every instance steps in blocks of check_every (even, >= 2) with the
 * convergence test of lbm_mix_run_to_steady (same residual, same block
 * boundaries, so the same step counts as a lone run) until its residual
 * drops to tol (status LBM_OK), it has taken max_steps (LBM_ENOTCONVERGED)
 * or turns non-finite (LBM_ENONFINITE); converged instances stop stepping.
 * A graph is replayed only while the instance's buffer parity, schedule,
 * reference-density table and step phase are those it was captured from;
 * calls on a borrowed handle that change them (odd step counts, state
 * uploads, lbm_mix_set_rows_per_block, lbm_mix_rereference) lead to a new
 * capture.
 * autotune != 0: the first LBM_SWEEP_NPOLICY blocks run under each
 * node-to-CTA schedule in turn (real steps, timed on the host around the
 * whole block), the rest under the fastest.  steps_out, residual_out,
 * status_out: n entries each, nullable.  Returns LBM_OK when the sweep ran
 * (per-instance outcomes are in status_out), LBM_EINVAL, LBM_ECUDA. */
int lbm_sweep_run_to_steady(lbm_sweep* s, double tol, long max_steps, long check_every,
                            int autotune, long* steps_out, double* residual_out,
                            int* status_out);

/* Borrowed handle of instance k (0 <= k < n): separation, moments and
 * post-state getters work on it; it stays owned by the sweep. */
int lbm_sweep_instance(lbm_sweep* s, int k, lbm_mix** out);

/* Schedule in use (policy: -1 before any run, else 0..LBM_SWEEP_NPOLICY-1),
 * rows per CTA of every instance (n entries) and the block times the
 * autotuner measured per policy in ms (LBM_SWEEP_NPOLICY entries, 0 where
 * not measured).  All outputs nullable. */
int lbm_sweep_schedule(lbm_sweep* s, int* policy, int* rows_per_block, double* round_ms);

/* ---------------------------------------------------------------------
 * Adjoint (gradients of a steady-channel objective).  A handle runs the
 * time step in FP64 on the full populations (the same map as lbm_mix_step:
 * Sec. 3 with the readings of this library) for nsteps steps from the
 * initial state of lbm_mix_init, keeping a checkpoint every
 * checkpoint_every steps, and computes the discrete adjoint of that run:
 * one backward sweep replays each checkpoint interval and runs the reverse
 * of each step (collision, tau_q at the walls, streaming with the DBB rule
 * of Eqs. bot, bot2, R and the ends of Eqs. rho1, rho2).  Gradients are
 * exact for the FP64 map up to rounding.  No counterpart in the paper (it
 * reports no sensitivities).
 * ------------------------------------------------------------------- */
typedef struct lbm_adj lbm_adj;

/* Objectives, both of the state after the last step:
 *   LBM_ADJ_CL    CL = (C_l,in - min_x C_l(x)) / C_l,in over the updated
 *                 columns, C_l(x) = sum_j n_l / sum_j n (Eq. CL; the
 *                 gradient flows through the minimising column);
 *   LBM_ADJ_FLUX  light-species x momentum summed over column N_x - 2 (the
 *                 outlet mass flux of the light species). */
#define LBM_ADJ_CL 0
#define LBM_ADJ_FLUX 1

/* Validates p like lbm_mix_create (storage is ignored: FP64; x_periodic
 * channels, the BSR wall and the non-default readings r_form and
 * lambda_pressure are rejected: the adjoint covers the pressure-driven
 * channel with its inlet and outlet, Eqs. rho1 and rho2, between DBB walls,
 * with the default readings) and allocates
 * the checkpoints (ceil(nsteps/checkpoint_every) + 1 states of 18 N N_x
 * doubles) and two intervals of step inputs, each step with 6 N N_x doubles
 * of wall-confinement factors and 18 N_x + 4 of column data (one interval
 * when checkpoint_every >= nsteps).  The forward run keeps its last interval
 * there; the backward sweep replays each other interval on a second,
 * internal stream while it reverses the next, and the reverse reads the
 * factors the forward run or the replay evaluated.  With
 * checkpoint_every >= nsteps the forward run keeps every step (about
 * 8 (24 N N_x + 18 N_x) bytes per step) and nothing is replayed.
 * stream: cudaStream_t or NULL for an own stream.  Errors: LBM_EINVAL,
 * LBM_ENOMEM, LBM_ECUDA. */
int lbm_adj_create(const lbm_mix_params* p, long nsteps, int checkpoint_every, void* stream,
                   lbm_adj** out);

/* Releases the handle.  NULL-safe. */
void lbm_adj_destroy(lbm_adj* a);

/* Per-wall-node accommodation coefficients alpha (Eq. A12 and c_m of
 * Eq. R), host array [2][N_x] (bottom wall then top), each in (0, 1]. */
int lbm_adj_set_accommodation_field(lbm_adj* a, const double* alpha, long n);

/* Runs the forward steps; CL and flux (nullable) receive both objectives.
 * LBM_ENONFINITE if the run diverged. */
int lbm_adj_forward(lbm_adj* a, double* CL, double* flux);

/* The FP64 state after the forward run, host [2][9][N][N_x]. */
int lbm_adj_state(lbm_adj* a, double* f, long n);

/* Backward sweep for `objective` after lbm_adj_forward: dJ/dtheta,
 * dJ/dKn_out and dJ/dalpha (host [2][N_x], n_alpha = 2 N_x); outputs
 * nullable.  theta enters the inlet densities (Eq. rho2) and the initial
 * state, Kn_out the viscosity that sets every mean free path.  May be
 * called again after one forward run (either objective): every call gives
 * what it gives after a fresh forward run, bit for bit. */
int lbm_adj_gradient(lbm_adj* a, int objective, double* dtheta, double* dkn, double* dalpha,
                     long n_alpha);

/* Static description of an error code; never NULL. */
const char* lbm_mix_strerror(int status);

/* Message of the last failed call on this host thread ("" if none). */
const char* lbm_mix_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_MIX_H */
