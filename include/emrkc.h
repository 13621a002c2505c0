/*
 * emrkc.h - C ABI of the GB300 (sm_103a) emRKC monodomain solver.
 *
 * One emRKC time step (Algorithm 3 of "Explicit stabilized multirate methods
 * for the monodomain model in cardiac electrophysiology", arXiv 2401.01745)
 * of the P1 finite-element monodomain system with lumped mass (Sec. 2.1,
 * Eq. sd_sys), split as in Eq. (mono_in_FSE):
 *   f_F(y)    = ((chi Cm M)^-1 A V, 0, 0)            A = -K (stiffness K >= 0)
 *   f_S(t, y) = (Cm^-1 (I_stim(t) - I_ion(y)), 0, g_S(y))
 *   f_E(y)    = (0, Lambda_E(y) (z_E - z_inf(y)), 0)
 * The gating variables z_E take the exponential (Rush-Larsen) step of
 * Sec. 4.1-4.2, the outer RKC iteration runs over the averaged force with
 * s stages, and the inner RKC iteration runs over the diffusion SpMV with
 * m stages (Algorithm 1).  Spectral radii rho_F and rho_S, which set s and
 * m, come from the nonlinear power iteration of Algorithm 5 (App. A).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: EMRKC_OK (0) or an EMRKC_ERR_*
 *    code.  A human-readable message is available from emrkc_last_error().
 *  - Host pointers passed in are read during the call only; the library
 *    copies what it keeps (ownership stays with the caller).  Host output
 *    buffers are allocated by the caller.  Exception: the buffers of
 *    emrkc_set_stimulus_async and emrkc_get_state_async stay in use until
 *    emrkc_sync returns.
 *  - The solver owns all device memory it allocates and frees it in
 *    emrkc_destroy().  All device work is ordered on the solver's CUDA
 *    stream (options.cuda_stream, or a stream the solver creates); the
 *    copies of the *_async calls run on two copy streams of the solver,
 *    ordered against that stream by events.
 *  - Units: cm, ms, mV, mS/cm, uF/cm^2, uA/cm^2.
 *  - The state is structure-of-arrays: variable 0 is V, variables 1..nE the
 *    gating variables z_E, the remaining ones z_S (see emrkc_num_vars()).
 *  - No CPU fallback exists: without a usable CUDA device every call that
 *    needs one fails with EMRKC_ERR_CUDA.
 */
#ifndef EMRKC_H
#define EMRKC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define EMRKC_OK 0
#define EMRKC_ERR_ARG 1       /* invalid argument (null pointer, size, range) */
#define EMRKC_ERR_CUDA 2      /* CUDA runtime error or no device              */
#define EMRKC_ERR_OOM 3       /* device or host allocation failed             */
#define EMRKC_ERR_NONFINITE 4 /* a NaN/Inf appeared in V during a step        */
#define EMRKC_ERR_TIMEOUT 5   /* a bounded device wait gave up                */
#define EMRKC_ERR_STATE 6     /* call not valid in the object's current state */

/* ---- ionic models (Sec. 2 and Sec. 5, Table 2) ------------------------- */
#define EMRKC_MODEL_NONE 0      /* pure diffusion, N = 1                      */
#define EMRKC_MODEL_PASSIVE 1   /* linear test model (V, w, c), N = 3         */
#define EMRKC_MODEL_HH 2        /* Hodgkin-Huxley 1952, N = 4 (V, m, h, n)    */
#define EMRKC_MODEL_TTP06_EPI 3 /* ten Tusscher-Panfilov 2006 epi, N = 19     */

/* ---- precision modes ---------------------------------------------------- */
#define EMRKC_PREC_FP64 0  /* every operation in FP64                          */
#define EMRKC_PREC_MIXED 1 /* z, SpMV, ionic model and gating in FP32; V, the
                              stage coefficients and rho in FP64               */

/* ---- spectral-radius policy (Sec. 5 setup; App. A) --------------------- */
#define EMRKC_RHO_ONCE 0   /* power iteration before the first step only   */
/* rho_every >= 1: power iteration every rho_every-th step (warm started)   */
#define EMRKC_RHO_FIXED -1 /* use options.rho_F / rho_S as given            */

/* ---- time integrators (Sec. 5) ---------------------------------------- */
#define EMRKC_METHOD_EMRKC 0   /* Algorithm 3 (default)                      */
#define EMRKC_METHOD_EXEX_RL 1 /* Algorithm 4 with the diffusion step taken
                                  explicitly: the paper's fine-step reference
                                  solver (Sec. 5).  FP64 only; rho options
                                  unused; s = m = 0 in the stats            */
#define EMRKC_METHOD_IMEX_RL 2 /* Algorithm 4: gates by exponential Euler,
                                  z_S by explicit Euler, then the implicit
                                  diffusion step (Cm M + dt K / chi) V_{n+1}
                                  = Cm M V_n + dt M (I_stim - I_ion), solved
                                  on the device by Jacobi-preconditioned CG
                                  in the lumped-mass inner product (stop at
                                  ||r||_M <= lin_rtol ||rhs||_M, warm start
                                  V_n).  FP64 only                          */
#define EMRKC_METHOD_MRKC 3    /* Algorithm 2 with the split of Sec. 3.3:
                                  f~_F = f_F + f_E^1 (the stiffest gate, the
                                  sodium activation m = z_E[0] of HH and
                                  TTP06, the gate of the passive model) and
                                  f~_S = f_S + f_E^2 (all other gates); no
                                  exponential step.  rho_F, rho_S are those
                                  of f~_F over (V, m) and of f~_S (Algorithm
                                  5); the rho options apply.  FP64 only     */

typedef struct emrkc_solver emrkc_solver; /* opaque; owns device memory */

/* Sparse P1 stiffness in CSR and the row-sum lumped mass (Sec. 2.1).
 * K_ij = sum_T int_T D grad(phi_j) . grad(phi_i): symmetric, row sums 0,
 * so the paper's A = -K.  Column indices must be in [0, n).  Entries whose
 * magnitude is at most 1e-14 |K_ii| are dropped when the solver is built. */
typedef struct {
  int64_t n;                  /* number of nodes                           */
  int64_t nnz;                /* stored entries                            */
  const int64_t* row_ptr;     /* n + 1 host entries                        */
  const int32_t* col;         /* nnz host entries                          */
  const double* K;            /* nnz host entries                          */
  const double* lumped_mass;  /* n host entries, all > 0                   */
} emrkc_matrix;

/* Matrix produced by emrkc_assemble_p1(); free with emrkc_free_matrix(). */
typedef struct {
  int64_t n, nnz;
  int64_t* row_ptr;
  int32_t* col;
  double* K;
  double* lumped_mass;
} emrkc_owned_matrix;

/* Tissue constants of Eq. (monodomain): chi (1/cm) and Cm (uF/cm^2). */
typedef struct {
  double chi;
  double Cm;
} emrkc_tissue;

/* Nodal stimulus (Eq. sd_sys, linear interpolation of I_stim):
 * I_stim(t, x_i) = amplitude if node_mask[i] != 0 and t_on <= t <= t_off. */
typedef struct {
  const uint8_t* node_mask; /* n host entries, or NULL for no stimulus (amplitude and
                             * window then apply to a mask set later, e.g. by
                             * emrkc_batch_set_stimulus_async) */
  double amplitude;         /* uA/cm^2 */
  double t_on, t_off;       /* ms, inclusive */
} emrkc_stimulus;

typedef struct {
  int precision;      /* EMRKC_PREC_*                                      */
  int rho_every;      /* EMRKC_RHO_ONCE, EMRKC_RHO_FIXED or k >= 1          */
  double rho_F, rho_S;/* used when rho_every == EMRKC_RHO_FIXED (1/ms)     */
  double eps;         /* RKC damping, 0.05 (Algorithm 1)                    */
  double safety;      /* factor on power-iteration rho, 1.05 (App. A)       */
  double pow_tol;     /* relative tolerance of Algorithm 5, 1e-2            */
  double pow_eps;     /* perturbation size of Algorithm 5, 1e-8             */
  int pow_max_iter;   /* iteration cap of Algorithm 5, 50                   */
  uint64_t seed;      /* start vectors: SplitMix64(seed ^ i) for rho_F and
                         SplitMix64(~seed ^ k) for rho_S (k = var*n + node) */
  double act_threshold; /* activation threshold in mV (-20); NaN disables  */
  void* cuda_stream;  /* cudaStream_t to order work on, or NULL            */
  int device;         /* CUDA device ordinal                                */
  int profile;        /* 1: time every kernel class with CUDA events        */
  int use_graphs;     /* batch API: 1 = replay each step's persistent launch
                         as a CUDA graph (re-captured when the plan
                         changes).  The single-instance solver launches its
                         step kernels directly, chained by programmatic
                         dependent launch; the option has no effect there */
  double rho_S_min;   /* known bound on rho(f_S): the step uses
                         max(safety * estimate, rho_S_min) (Sec. 3.1: rho is
                         known or estimated); 0 = estimate only            */
  int method;         /* EMRKC_METHOD_* (default EMRKC_METHOD_EMRKC)        */
  double lin_rtol;    /* IMEX-RL: relative residual of the CG solve, 1e-10  */
  int lin_max_iter;   /* IMEX-RL: CG iteration cap, 1000 (a solve that hits
                         it is not an error; see emrkc_stats.lin_iters)     */
  double pow_tol_cold;   /* Algorithm 5 with no initial guess (the first
                            estimate of rho_F or rho_S, from the arbitrary
                            start vector): relative tolerance 1e-4.  The
                            warm-started calls that follow use pow_tol.
                            From a cold start the 1e-2 test of App. A can
                            stop on an early plateau (0.80-0.97 of rho(L)
                            measured on 3-D slabs), below what the safety
                            factor covers                                 */
  int pow_max_iter_cold; /* iteration cap of a cold start, 1000            */
} emrkc_options;

/* Kernel classes reported in emrkc_stats.phase_ms / phase_launches. */
#define EMRKC_PHASE_STAGE 0   /* fused RL + ionic + first SpMV + outer update
                                 (EXEX-RL: the whole step; IMEX-RL: the ionic
                                 half and the CG set-up)                      */
#define EMRKC_PHASE_INNER 1   /* inner RKC SpMV stage (IMEX-RL: the CG solve) */
#define EMRKC_PHASE_POWER_F 2 /* power iteration on f_F                       */
#define EMRKC_PHASE_POWER_S 3 /* power iteration on f_S                       */
#define EMRKC_PHASE_OTHER 4   /* norms, start vectors, f_S(y)                 */
#define EMRKC_NUM_PHASES 5

typedef struct {
  double t;              /* current time (ms)                          */
  int64_t steps;         /* steps taken                                */
  int s, m;              /* stage counts of the last step              */
  double eta;            /* inner step of the last step                */
  double rho_F, rho_S;   /* values used by the last step (with safety) */
  int pow_iters_F, pow_iters_S; /* iterations of the last power call   */
  int64_t total_pow_iters;
  int64_t launches;      /* kernels launched since create              */
  int64_t matrix_entries;/* stored nonzeros of L after dropping zeros  */
  int64_t matrix_slots;  /* sliced-ELL slots including padding         */
  double phase_ms[EMRKC_NUM_PHASES];       /* needs options.profile    */
  int64_t phase_launches[EMRKC_NUM_PHASES];
  int lin_iters;         /* IMEX-RL: CG iterations of the last step    */
  int64_t total_lin_iters; /* IMEX-RL: CG iterations since create      */
  double lin_residual;   /* IMEX-RL: ||r||_M / ||rhs||_M after the last
                            solve                                      */
} emrkc_stats;

/* Fill *opt with the defaults listed above (FP64, rho every step, seed 0,
 * threshold -20 mV, NULL stream, device 0, no profiling, graphs on,
 * rho_S_min 0, method EMRKC_METHOD_EMRKC, lin_rtol 1e-10, lin_max_iter 1000,
 * pow_tol_cold 1e-4, pow_max_iter_cold 1000). */
int emrkc_default_options(emrkc_options* opt);

/* Number of state variables N (V included) of an ionic model, or -1. */
int emrkc_num_vars(int ionic_model);
/* Number of gating variables nE of an ionic model, or -1. */
int emrkc_num_gates(int ionic_model);

/* Algorithm 1, get_stages: the stage count s >= 1 of the damped RKC method
 * (damping eps) for a step dt and a spectral radius rho, i.e. the smallest
 * s with beta s^2 >= dt rho, beta = 2 - 4 eps / 3, so that dt times the
 * spectrum lies in the stability interval [-beta s^2, 0] (Sec. 3.1).  Every
 * path of the library takes its counts from this definition: the outer
 * stages from dt and rho_S, the inner stages from eta = 2 dt / (beta s^2)
 * and rho_F (Algorithm 3).  Writes *s and, if l_s is not NULL, the interval
 * length beta s^2.  Host routine: no device is needed.  Errors:
 * EMRKC_ERR_ARG for a NULL s; dt, rho or eps negative or not finite;
 * eps >= 1.5 (beta <= 0); or dt rho >= 1e15 (s beyond the library's limits). */
int emrkc_rkc_stages(double dt, double rho, double eps, int* s, double* l_s);

/* Algorithm 1, get_coeffs: the coefficients of the s-stage damped RKC
 * method from the Chebyshev polynomials at omega_0 = 1 + eps / s^2:
 * mu_j, nu_j, kappa_j for j = 1..s (entry 0 is 0; nu_1 = kappa_1 = 0) and the
 * internal times c_j for j = 0..s (c_0 = 0, c_s = 1).  mu, nu, kappa and c
 * are caller-owned host arrays of s + 1 doubles.  Host routine: no device
 * is needed.  Errors: EMRKC_ERR_ARG for s < 1 or s > 2^20, eps negative or
 * not finite, or a NULL array. */
int emrkc_rkc_coeffs(int s, double eps, double* mu, double* nu, double* kappa, double* c);

/* P1 stiffness K and row-sum lumped mass of a simplex mesh (Sec. 2.1).
 * dim in {1, 2, 3}; xyz: n_nodes*dim doubles (node-major); cells:
 * n_cells*(dim+1) node indices; D_per_cell: n_cells*dim*dim doubles, the
 * conductivity tensor of Eq. (def_D) per cell (row-major).  Host routine;
 * on success *out owns malloc'd arrays (free with emrkc_free_matrix).
 * Errors: EMRKC_ERR_ARG for bad sizes/indices or a zero-volume cell. */
int emrkc_assemble_p1(int dim, int64_t n_nodes, const double* xyz, int64_t n_cells,
                      const int64_t* cells, const double* D_per_cell,
                      emrkc_owned_matrix* out);
void emrkc_free_matrix(emrkc_owned_matrix* m);

/* Build a solver: validates and copies the CSR, drops near-zero entries,
 * prescales L = -(chi Cm M)^-1 K into a sliced-ELL device matrix, allocates
 * the SoA state and sets every node to the model's rest state (Sec. 5).
 * opt may be NULL (defaults).  On failure *out is NULL. */
int emrkc_create(const emrkc_matrix* mat, const emrkc_tissue* tissue, int ionic_model,
                 const emrkc_stimulus* stim, const emrkc_options* opt, emrkc_solver** out);

/* One emRKC step of size dt (ms) from the current state (Algorithm 3),
 * preceded by the power iteration when the rho policy asks for it.  The
 * step is enqueued on the solver's stream; the call synchronises only for
 * the power iteration.  Returns EMRKC_ERR_NONFINITE if a previously
 * enqueued step produced a non-finite V (checked at every synchronisation). */
int emrkc_step(emrkc_solver* s, double dt);

/* round(T/dt) steps; EMRKC_ERR_ARG if T/dt is not an integer within 1e-9.
 * Synchronises at the end and reports non-finite values. */
int emrkc_run(emrkc_solver* s, double T, double dt);

/* Wait for all enqueued work (steps and the asynchronous copies of
 * emrkc_set_stimulus_async / emrkc_get_state_async); returns
 * EMRKC_ERR_NONFINITE if any step produced a non-finite V since the last
 * check. */
int emrkc_sync(emrkc_solver* s);

/* Copy variable var (0..N-1) or the whole state (var = -1, SoA: var-major,
 * N*n doubles) to/from host memory; len must equal n or N*n.  FP32-stored
 * variables (mixed precision) are converted.  Synchronous. */
int emrkc_get_state(emrkc_solver* s, int var, double* host_out, int64_t len);
int emrkc_set_state(emrkc_solver* s, int var, const double* host_in, int64_t len);

/* Same as get/set_state with device pointers (len doubles, on this device). */
int emrkc_get_state_device(emrkc_solver* s, int var, double* dev_out, int64_t len);
int emrkc_set_state_device(emrkc_solver* s, int var, const double* dev_in, int64_t len);

/* Activation times (first upward crossing of options.act_threshold,
 * linear interpolation between step ends; NaN = never).  n doubles. */
int emrkc_get_activation_times(emrkc_solver* s, double* host_out, int64_t n);

/* Run Algorithm 5 now on the current state (warm started) and return the
 * raw estimates (without the safety factor) and iteration counts. */
int emrkc_estimate_rho(emrkc_solver* s, double* rho_F, double* rho_S, int* it_F, int* it_S);

/* Allocation-free variant of the f_F half of emrkc_estimate_rho.  The paper
 * has no counterpart: this entry point exists for callers that must not
 * allocate device memory while they run, e.g. a host whose own allocator
 * owns the whole GPU, or a time-critical loop that cannot afford
 * cudaMalloc's implicit synchronisation.  It runs the same nonlinear power
 * iteration on the diffusion term f_F at the solver's current V, with
 * caller-owned device vectors: d_v (n doubles; in: start or warm-start
 * direction, out: final iterate) and d_w (n doubles of work space);
 * rho_warm is the warm start (0 for none).  Writes the raw estimate (no
 * safety factor) and the iteration count.  emRKC solvers only (for mRKC the
 * solver's own estimate runs on (V, z_k), not on V).
 * The reduction scratch (1024 partial sums, 8 result slots and a ticket
 * counter: 8.5 KiB) is a static device array that every GPU loading the
 * library holds until exit.  The reduction grid is capped at 1024 blocks,
 * one partial sum each; grid-stride loops cover any n.  The first call on a
 * device looks the array's address up (cudaGetSymbolAddress) and zeroes the
 * ticket, so make that first call before any stream capture; the address is
 * kept for the life of the device's primary context.  Every call shares the
 * array: calls that overlap on the GPU (other streams, other threads) race.
 * Errors: EMRKC_ERR_ARG for a null pointer, n != number of nodes or a
 * method other than emRKC; EMRKC_ERR_CUDA if the set-up or a launch fails.
 * Calls no cudaMalloc / cudaFree and synchronises the solver's stream. */
int emrkc_estimate_rho_F_noalloc(emrkc_solver* s, double* d_v, double* d_w, int64_t n, double rho_warm,
                                 double* rho_out, int* it_out);

/* Set the time and step counter (checkpoint/resume together with set_state). */
int emrkc_set_time(emrkc_solver* s, double t, int64_t steps);

/* Replace the applied stimulus (the I_stim of Eq. monodomain, nodal as in
 * Sec. 2.1) for the following steps: node_mask (n host bytes, nonzero =
 * stimulated; NULL = no stimulus), amplitude in uA/cm^2, active for
 * t_on <= t <= t_off (ms, inclusive).  Stimulation protocols (pacing trains,
 * moving sites) change it between steps.  The mask is copied on the
 * solver's stream before the call returns; the host buffer may be reused at
 * once.  Errors: EMRKC_ERR_ARG (n does not match), EMRKC_ERR_CUDA. */
int emrkc_set_stimulus(emrkc_solver* s, const uint8_t* node_mask, int64_t n, double amplitude, double t_on,
                       double t_off);

/* Pipelined host I/O (not in the paper: the host side of a time-stepping
 * service).  Both calls enqueue work and return without waiting, so a caller
 * can feed each step's input and read each step's result while later steps
 * compute; the copies run on the copy engines, on a second stream of the
 * solver, ordered against the steps by events.
 *
 * emrkc_set_stimulus_async: as emrkc_set_stimulus (same arguments, errors
 * and immediate effect on the amplitude and window), but the n-byte mask is
 * copied into a second device mask buffer that no enqueued step reads; the
 * steps enqueued after the call use it.  node_mask must stay valid and
 * unchanged until emrkc_sync returns (pinned host memory makes the copy
 * asynchronous; pageable memory works but the copy is staged by the driver).
 *
 * emrkc_get_state_async: variable var (0..N-1; not the whole state) of the
 * state after the steps enqueued so far, as n doubles (len must equal n), to
 * host_out.  The variable is first converted into one of two device staging
 * buffers on the solver's stream (a float-float V is joined, FP32 rows are
 * widened); the device-to-host copy then overlaps the following steps.
 * host_out is complete once emrkc_sync returns; it must stay valid until
 * then.  Errors: EMRKC_ERR_ARG (var out of range, null buffer),
 * EMRKC_ERR_STATE (len), EMRKC_ERR_OOM, EMRKC_ERR_CUDA.  emrkc_sync waits for
 * both streams. */
int emrkc_set_stimulus_async(emrkc_solver* s, const uint8_t* node_mask, int64_t n, double amplitude, double t_on,
                             double t_off);
int emrkc_get_state_async(emrkc_solver* s, int var, double* host_out, int64_t len);

int emrkc_get_stats(emrkc_solver* s, emrkc_stats* out);

/* Message of the last error on this solver, or of the last failed create
 * on this thread when s is NULL.  Never NULL. */
const char* emrkc_last_error(const emrkc_solver* s);

void emrkc_destroy(emrkc_solver* s);

/* ---- Batched persistent step --------------------------------------------
 * Many independent monodomain problems (instances) of different sizes,
 * ionic models and stage counts advance one emRKC step each in ONE persistent
 * kernel launch per step (replayed as a CUDA graph).  Every instance is a
 * mixed-precision solver (EMRKC_PREC_MIXED) whose state stays on the device.
 * The rho policy of a batch is EMRKC_RHO_ONCE (Algorithm 5 when an instance
 * takes its first step) or EMRKC_RHO_FIXED; s and m per instance are then
 * fixed while dt is unchanged.  s, m <= 32 and s * m <= 64 per instance.
 * Instances can be added and removed between steps (continuous batching).  */
typedef struct emrkc_batch emrkc_batch;

typedef struct {
  int64_t n;          /* nodes                                   */
  int N;              /* state variables                         */
  int model;          /* ionic model                             */
  int s, m;           /* stage counts (0 before the first step)  */
  double t;           /* time of the instance (ms)               */
  int64_t steps;      /* steps taken                             */
  int64_t device_bytes; /* device memory held by the instance    */
} emrkc_batch_info;

typedef struct {
  int instances;
  int64_t total_nodes;
  int64_t items;        /* work items per step                    */
  int tile, block, grid;/* launch configuration in use            */
  int64_t launches;     /* persistent launches so far             */
  int64_t device_bytes; /* all instances plus the batch tables    */
  int schedule;         /* order of the work list: 0 whole phases,
                           1 / 2 at most 16 / 4 tiles per instance
                           in turn (chosen by the autotuner)       */
  int threads_per_sm;   /* resident threads per SM the persistent
                           kernel is compiled for: 1024, 1536 or
                           2048, a register budget of 64, 40 or 32
                           per thread (chosen by the autotuner)    */
} emrkc_batch_stats;

/* Options: device, cuda_stream, seed, act_threshold, rho_every (ONCE or
 * FIXED with rho_F/rho_S), use_graphs are used; precision is forced to MIXED.
 * opt may be NULL.  The batch starts with tile 1024 nodes, block 128, 1536
 * threads per SM. */
int emrkc_batch_create(const emrkc_options* opt, emrkc_batch** out);
/* Add an instance (copies its inputs; same arguments as emrkc_create).
 * inst_opt (may be NULL: the batch's options) sets the instance's rho policy
 * (ONCE or FIXED, rho_F, rho_S, rho_S_min), seed and activation threshold;
 * precision, stream and device are the batch's.  *id_out receives a
 * batch-unique id.  Takes effect at the next step. */
int emrkc_batch_add(emrkc_batch* b, const emrkc_matrix* mat, const emrkc_tissue* tissue, int ionic_model,
                    const emrkc_stimulus* stim, const emrkc_options* inst_opt, int* id_out);
/* Remove an instance and free its device memory, after waiting for the
 * batch's stream; the work plan is rebuilt at the next step.  Errors:
 * EMRKC_ERR_ARG (unknown id). */
int emrkc_batch_remove(emrkc_batch* b, int id);
/* One emRKC step (Algorithm 3) of size dt (ms) for every instance: one
 * persistent launch, enqueued on the batch's stream (the call does not wait
 * for it).  After instances joined or left, or when dt changes, the work
 * plan is rebuilt first: Algorithm 5 runs for instances that have no
 * estimate yet (EMRKC_RHO_ONCE), Algorithm 1 sets each instance's s and m,
 * and the call waits for the plan's upload.  Errors: EMRKC_ERR_ARG (dt not
 * positive and finite, or an instance's stage counts beyond s, m <= 32,
 * s * m <= 64), EMRKC_ERR_OOM, EMRKC_ERR_CUDA, and the power iteration's
 * errors. */
int emrkc_batch_step(emrkc_batch* b, double dt);
/* Wait for enqueued steps; EMRKC_ERR_NONFINITE if an instance produced a
 * non-finite V, EMRKC_ERR_TIMEOUT if a dependency wait gave up. */
int emrkc_batch_sync(emrkc_batch* b);
/* As emrkc_get_state, emrkc_set_state and emrkc_get_activation_times for
 * the instance id (same arguments, layouts and waits).  Errors:
 * EMRKC_ERR_ARG for an unknown id, then those of the solver call. */
int emrkc_batch_get_state(emrkc_batch* b, int id, int var, double* host_out, int64_t len);
int emrkc_batch_set_state(emrkc_batch* b, int id, int var, const double* host_in, int64_t len);
int emrkc_batch_get_activation_times(emrkc_batch* b, int id, double* host_out, int64_t n);
/* Sizes, stage counts, time and device bytes of one instance (*out, host);
 * EMRKC_ERR_ARG for a NULL out or an unknown id. */
int emrkc_batch_get_info(emrkc_batch* b, int id, emrkc_batch_info* out);
/* Totals and the launch configuration in use (*out, host); EMRKC_ERR_ARG
 * for a NULL out. */
int emrkc_batch_get_stats(emrkc_batch* b, emrkc_batch_stats* out);
/* Launch configuration: tile in {256, 512, ..., 8192} nodes, block 128 or
 * 256 (takes effect at the next step).  EMRKC_ERR_ARG for other values. */
int emrkc_batch_set_config(emrkc_batch* b, int tile, int block);
/* Order of the work list: 0 (default) an instance's whole phase at a time,
 * 1 / 2 at most 16 / 4 tiles of an instance before the next ready one.
 * Every order gives the same results.  EMRKC_ERR_ARG for other values. */
int emrkc_batch_set_schedule(emrkc_batch* b, int schedule);
/* Register budget of the persistent kernel, as resident threads per SM:
 * 1024, 1536 (default) or 2048 (64, 40 or 32 registers per thread).  More
 * resident threads hide more load latency; the two smaller budgets spill
 * some registers to local memory.  Every budget gives the same results.
 * Takes effect at the next step.  EMRKC_ERR_ARG for other values. */
int emrkc_batch_set_occupancy(emrkc_batch* b, int threads_per_sm);
/* Time each (tile, block, work-list order, register budget) candidate over
 * `reps` steps of size dt without advancing any instance (the candidates
 * run with bookkeeping and activation writes disabled) and keep the
 * fastest.  Returns EMRKC_ERR_STATE (configuration unchanged) if an
 * instance has s >= 3, whose dry steps would overwrite its current state
 * buffer, and EMRKC_ERR_TIMEOUT if a dependency wait gave up.  Outputs
 * (the chosen tile and block, the best time per step in ms) may be NULL. */
int emrkc_batch_autotune(emrkc_batch* b, double dt, int reps, int* tile_out, int* block_out, double* ms_out);
/* Diagnostics: polls of a dependency wait before the persistent kernel gives
 * up, records EMRKC_ERR_TIMEOUT (reported by emrkc_batch_sync) and returns;
 * default 2^24 (about 2 s with 100 ns back-off).  limit >= 0. */
int emrkc_batch_set_spin_limit(emrkc_batch* b, int64_t limit);
/* Pipelined host I/O of a whole batch (as emrkc_set_stimulus_async /
 * emrkc_get_state_async for one solver, with the state held on the device
 * as a model's weights are).  The host arrays hold every instance's nodes
 * concatenated in the order returned by emrkc_batch_ids (the order in which
 * the instances were added); len must equal the batch's total node count.
 * emrkc_batch_set_stimulus_async: node masks (one byte per node, nonzero =
 * stimulated), copied from host_masks into one of two device staging
 * buffers on a host-to-device copy stream, then scattered into the
 * instances' mask buffers on the batch's stream; steps enqueued after the
 * call use the new masks (amplitude and time window stay per instance).
 * emrkc_batch_get_V_async: V of every instance after the steps enqueued so
 * far, joined from the float-float pair into one of two device staging
 * buffers on the batch's stream and copied to host_out on a device-to-host
 * copy stream, overlapping the following steps.  Host buffers (pinned
 * memory for overlap) must stay valid, and host_out is complete, once
 * emrkc_batch_sync returns; emrkc_batch_sync waits for both copy streams.
 * Errors: EMRKC_ERR_ARG (null buffer), EMRKC_ERR_STATE (len; get_V_async
 * before the first step after instances joined or left), EMRKC_ERR_OOM,
 * EMRKC_ERR_CUDA. */
int emrkc_batch_set_stimulus_async(emrkc_batch* b, const uint8_t* host_masks, int64_t len);
int emrkc_batch_get_V_async(emrkc_batch* b, double* host_out, int64_t len);
/* As emrkc_batch_get_V_async with V rounded to FP32 (the hi part of the
 * float-float V, its nearest float): half the bytes over the host link. */
int emrkc_batch_get_V32_async(emrkc_batch* b, float* host_out, int64_t len);
/* Instance ids in batch order into ids_out (up to cap entries); returns the
 * number of instances (-1 if b is NULL). */
int emrkc_batch_ids(const emrkc_batch* b, int* ids_out, int cap);
/* Kernel timing: with on != 0 every persistent launch is bracketed by CUDA
 * events on the batch's stream (steps are then launched directly, not as a
 * graph); emrkc_batch_get_kernel_time returns the summed milliseconds and
 * the number of timed launches so far (read at emrkc_batch_sync). */
int emrkc_batch_set_profile(emrkc_batch* b, int on);
int emrkc_batch_get_kernel_time(emrkc_batch* b, double* ms_out, int64_t* launches_out);
/* Device bytes an instance of n nodes with nnz_per_row stored entries per
 * row would hold (for admission control against an HBM budget). */
int64_t emrkc_instance_bytes(int64_t n, double nnz_per_row, int ionic_model);
const char* emrkc_batch_last_error(const emrkc_batch* b);
void emrkc_batch_destroy(emrkc_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* EMRKC_H */
