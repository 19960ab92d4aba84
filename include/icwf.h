/*
 * icwf.h -- C ABI of the GB300 (sm_103a) library for the Interacting Conditional Wavefunction
 * (ICWF) time step of Albareda, Kelly and Rubio, arXiv 1805.11169.
 *
 * The method (paper, Eq. ansatz): the wavefunction of an electron coordinate x and a nuclear or
 * photon coordinate R is expanded as Psi(x,R,t) = sum_a C_a(t) psi_a(x,t) chi_a(R,t) over N
 * stochastic trajectories (x_a, R_a).  One time step advances
 *   - the Bohmian positions with the velocities of Eq. v1/v2,
 *   - every conditional wavefunction (CWF) under its Hermitian-CWF equation (Eq.
 *     conditional_e / conditional_n with the complex eta potentials dropped, as the paper
 *     prescribes for the Hermitian limit), the other coordinate pinned at the trajectory,
 *   - the coefficients by Eq. coeff, S dC/dt = -i Heff C, with S the overlap (Eq. M) and
 *     Heff = W - W1 - W2 (Eq. W, W1, W2), pinned at the ket.
 *
 * Conventions for every call:
 *   - All pointers are HOST pointers.  Inputs are copied; the library never keeps caller memory.
 *     Outputs are written into caller-owned arrays of the documented length.
 *   - Complex arrays are interleaved (re, im) float64 pairs.
 *   - Grids are cell-centred and periodic: x_i = x_min + (i + 1/2) dx, dx = (x_max - x_min)/nx.
 *   - Every call returns an icwf_status; icwf_last_error() gives a one-line description of the
 *     last failure on that handle (or of the last failed create when called with NULL).
 *   - Call-order mistakes (step before init, ...) return ICWF_ERR_STATE and change nothing.
 *   - A non-finite velocity or coefficient, or a failed Cholesky pivot, returns ICWF_ERR_NUMERIC
 *     (detected when the call's device work ends); the handle's state is then not usable and
 *     must be re-initialised.
 *   - Handles are not thread-safe; distinct handles share nothing (except through a pool).
 *   - All device work of a handle runs on the handle's own CUDA stream on the current device at
 *     create time; calls return after that work has finished.
 */
#ifndef ICWF_H
#define ICWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct icwf_ctx* icwf_handle;
typedef struct icwf_pool_ctx* icwf_pool;

typedef enum {
  ICWF_OK = 0,
  ICWF_ERR_ARG = 1,      /* invalid argument (size, pointer, range) */
  ICWF_ERR_STATE = 2,    /* call out of order */
  ICWF_ERR_OOM = 3,      /* device allocation failed or pool HBM budget exceeded */
  ICWF_ERR_CUDA = 4,     /* a CUDA runtime call failed */
  ICWF_ERR_NUMERIC = 5,  /* NaN/Inf in C or S, or Cholesky pivot <= 0 after regularisation */
  ICWF_ERR_TIMEOUT = 6   /* an in-kernel wait gave up (iteration limit reached) */
} icwf_status;

typedef enum {
  ICWF_FP64 = 0,          /* CWFs complex128; matrix elements, Cholesky, triangular solves and
                             RK4 in FP64 (the factorisation's trailing updates in emulated FP64
                             on the tensor cores unless icwf_set_emulated_update turns it off) */
  ICWF_MIXED_BF16X3 = 1,  /* CWFs complex64, FP32 propagation; Grams on tcgen05 tensor cores as
                             three BF16 products (hi*hi + hi*lo + lo*hi), FP32 accumulation;
                             the overlap S as an exact Gram of fixed-point CWFs (positive
                             semidefinite; see overlap_split); S and Heff stored in FP64;
                             S + eps*I formed in FP64; Cholesky and
                             triangular solves in double-float arithmetic (pairs of FP32, about
                             44-48 significant bits) unless solve_fp64 is set; right-hand sides,
                             RK4 update and reductions in FP64 */
  ICWF_MIXED_TF32X3 = 2   /* as above with TF32 operand pieces */
} icwf_precision;

typedef struct {
  int32_t nx, nR;           /* grid sizes; powers of two in [8, 4096] (radix-2 FFT); the mixed
                               modes need nx, nR >= 64 */
  double x_min, x_max;      /* electron grid extent (periodic cell) */
  double R_min, R_max;      /* nuclear / photon grid extent */
  double mass_x, mass_R;    /* masses in atomic units (e.g. 1 and 1836, or 1 and 1) */
  double dt;                /* time step, a.u. */
  int32_t n_traj;           /* N >= 1 trajectories (basis functions) */
  int32_t precision;        /* icwf_precision */
  double svd_rel_cutoff;    /* rank rule for V_c (see icwf_create); 0 keeps every singular value */
  double s_reg_eps;         /* Tikhonov shift eps: the solves use S + eps*I (S_aa = 1) */
  int32_t coeff_scheme;     /* 0: RK4 with S, Heff linear in t over the step (two Cholesky
                               factorisations per step); 1: S, Heff frozen at t_n (one) */
  int32_t max_rank;         /* upper bound on the kept rank k (0: no bound beyond the cutoff) */
  int32_t solve_fp64;       /* mixed modes only: 1 runs the Cholesky factorisations and triangular
                               solves with the FP64 solver (as ICWF_FP64 does; its trailing
                               updates in emulated FP64, see icwf_set_emulated_update) instead of
                               double-float; ignored by ICWF_FP64 */
  int32_t overlap_split;    /* mixed modes only: 0 (default) computes S = S1 o S2 as exact Grams
                               of the CWFs in a 4-digit fixed-point form on the tensor cores, so
                               S is positive semidefinite to FP64 rounding and eps can be as
                               small as in ICWF_FP64; 1 takes S from the same split products
                               with FP32 accumulation as the other Grams (rounding ~1e-6 of S,
                               whose indefinite part needs eps ~1e-3 at N = 1024) */
} icwf_params;

/* Diagnostic facts about a handle. */
typedef struct {
  int32_t rank;             /* kept rank k of the interaction factorisation */
  double tail_rel;          /* ||dropped part of V_c||_F / ||V_c||_F */
  double next_rel;          /* first dropped singular value / largest (0 if none dropped) */
  double sigma_max;         /* largest singular value of V_c */
  size_t device_bytes;      /* device memory held by the handle */
  int64_t steps_done;       /* completed time steps since init */
  double t;                 /* simulated time */
  int64_t kernel_launches;  /* CUDA kernels launched by icwf_step on this handle since create */
  size_t obs_bytes;         /* device memory of the observables work buffers, which
                               icwf_observables allocates on its first call (0 until then) */
  int32_t prop_threads;     /* CTA size of the CWF propagator chosen by the autotuner for this
                               shape (fastest of 64..512 threads, timed at the first create of
                               the shape in the process) */
} icwf_info;

/* Observables of the current state (paper: reduced densities, BO populations and the
 * decoherence indicator of the Shin-Metiu discussion; norm and energy).  Arrays are
 * caller-owned; any of them may be NULL to skip it.
 *   rho_x[nx]  = int dR |Psi(x_i, R)|^2        rho_R[nR] = int dx |Psi(x, R_j)|^2
 *   pop[n_s]   = int dR |chi^(n)(R)|^2,        chi^(n)(R) = int dx phi_n(x; R) Psi(x, R)
 *   decoh[n_s*n_s] = int dR |chi^(n)|^2 |chi^(m)|^2   (row-major n, m)
 *   norm = <Psi|Psi>,  energy = <Psi|T_x + T_R + V|Psi> / <Psi|Psi>.
 * pop and decoh need icwf_set_projectors; otherwise they are left untouched. */
typedef struct {
  double t;
  double norm;
  double energy;
  double* rho_x;
  double* rho_R;
  double* pop;
  double* decoh;
  int32_t n_states;         /* out: number of projectors set (0 if none) */
  int32_t n_clamped;        /* out: cumulative count of positions clamped to the grid */
} icwf_obs;

/* Create a handle for the problem of the paper's Eq. TDSE with 1D x and R and no vector
 * potential: grids, masses, dt and N from *p; V[i*nR + j] = V(x_i, R_j) (float64, host,
 * copied).  Double-centres V = v1(x) + v2(R) + V_c and keeps the smallest rank k of the SVD of
 * V_c whose Frobenius tail is <= svd_rel_cutoff * ||V_c||_F (the factorisation used for the
 * matrix elements of Eq. W, which the paper flags as costly for large ensembles).
 * Allocates every device buffer.  On failure *out is NULL and icwf_last_error(NULL) explains. */
icwf_status icwf_create(const icwf_params* p, const double* V, icwf_handle* out);

/* Real BO states used as population projectors: phi[(n*nR + j)*nx + i] = phi_n(x_i; R_j),
 * n < n_states <= 8 (host, copied).  Optional; may be called at any time after create. */
icwf_status icwf_set_projectors(icwf_handle h, int32_t n_states, const double* phi);

/* Initialise from Psi0: psi0[2*(i*nR + j) + {0,1}] = Psi0(x_i, R_j) (complex128, host, copied).
 * Samples N positions from |Psi0|^2 with SplitMix64(seed) (cell by inverse CDF over the
 * row-major flattened density, then uniform jitter inside the cell), slices the CWFs
 * psi_a = Psi0(., R_a), chi_a = Psi0(x_a, .) by 4-point cubic Lagrange interpolation along the
 * other axis (Eq. CWF1/CWF2), normalises each to 1, assembles S_0 and Heff_0 and sets
 * C_0 = (S_0 + eps I)^-1 <phi_a|Psi0>.  Resets t and the step counter. */
icwf_status icwf_init_from_density(icwf_handle h, const double* psi0, uint64_t seed);

/* As icwf_init_from_density with caller-chosen positions x[N], R[N] (no sampling). */
icwf_status icwf_init_from_positions(icwf_handle h, const double* psi0, const double* x,
                                     const double* R);

/* Advance n_steps >= 0 time steps (velocities, positions, CWF propagation, matrices at
 * t + dt, coefficients).  Returns when the device has finished. */
icwf_status icwf_step(icwf_handle h, int32_t n_steps);

/* Compute observables of the current state into *out (see icwf_obs). */
icwf_status icwf_observables(icwf_handle h, icwf_obs* out);

/* Release the handle and all its device memory.  NULL is a no-op. */
icwf_status icwf_destroy(icwf_handle h);

/* --- diagnostics and tests ---------------------------------------------------------------- */

/* Copy the state out.  C[2N], x[N], R[N] float64; psi[2*nx*N], chi[2*nR*N] complex128 with
 * psi[2*(a*nx + i)] = Re psi_a(x_i) (column a contiguous).  Any pointer may be NULL. */
icwf_status icwf_get_state(icwf_handle h, double* C, double* x, double* R, double* psi,
                           double* chi);

/* Copy the N x N matrices at the current time, row-major complex128 [2*(a*N + b)]:
 * S (Eq. M), H = <phi_a|T_x + T_R + V|phi_b> and Heff = W - W1 - W2.  Any pointer may be NULL;
 * H costs extra Grams and is computed only when requested. */
icwf_status icwf_get_matrices(icwf_handle h, double* S, double* H, double* Heff);

icwf_status icwf_get_info(icwf_handle h, icwf_info* out);

/* --- checkpoint / resume ------------------------------------------------------------------- */

/* Bytes of the handle's time-stepping state as icwf_save_state writes it: a header (sizes,
 * precision, step count, time) and the device state at the current time (CWFs in their storage
 * precision, positions, pinned factor values, C, S, Heff, the Cholesky factor of S + eps I with
 * its inverted diagonal blocks, the clamp counter). */
icwf_status icwf_state_bytes(icwf_handle h, size_t* bytes);

/* Copy the state into buf (host, caller-owned, at least icwf_state_bytes bytes). */
icwf_status icwf_save_state(icwf_handle h, void* buf, size_t bytes);

/* Restore a state saved by icwf_save_state from a handle created with the same parameters and
 * the same V (sizes, rank, precision, scheme and solver are checked, else ICWF_ERR_ARG); the handle
 * is then initialised and continues bit for bit as the saved handle would have.  Projectors are
 * not part of the state. */
icwf_status icwf_load_state(icwf_handle h, const void* buf, size_t bytes);

/* Columns of Heff = W - W1 - W2 (Eq. W, W1, W2) by the full double sum over the grid, without the
 * rank-k factorisation of V:
 *   Heff[a, b] = dx dR sum_ij conj(psi_a(x_i) chi_a(R_j)) [V(x_i,R_j) - V(x_i,R_b) - V(x_b,R_j)]
 *                psi_b(x_i) chi_b(R_j),
 * on the handle's current CWFs and positions, in FP64 arithmetic (the CWFs are read in their
 * storage precision), O(N nx nR) work per column.  It is the reference the factorised assembly's
 * error is reported against (the paper flags this contraction as the costly part of the method
 * for large ensembles).  cols[m] in [0, N) for m < n_cols (1 <= n_cols <= N);
 * out[2*(m*N + a) + {0,1}] = Heff[a, cols[m]] (complex128, host, caller-owned).  Allocates and
 * frees its own device work buffer (about 16 N n_cols (nx/64 + 1) bytes). */
icwf_status icwf_heff_direct(icwf_handle h, int32_t n_cols, const int32_t* cols, double* out);

/* Change the Tikhonov shift eps of the solves (S + eps I) for the following steps.  Any finite
 * value is accepted; a negative eps makes S + eps I indefinite, so the next step's Cholesky
 * fails and returns ICWF_ERR_NUMERIC (the failure path the tests drive on purpose). */
icwf_status icwf_set_regularisation(icwf_handle h, double eps);

/* FP64 solver (ICWF_FP64, or solve_fp64 in the mixed modes): how the blocked Cholesky
 * factorisation forms its trailing updates A_rc -= L_r L_c^H (a Hermitian rank-32 update per block
 * column; the bulk of the factorisation's arithmetic).  on = 1 (default): on the tensor cores in
 * emulated FP64 -- each row of the 32-wide panel is scaled by a power of two and cut into seven
 * 8-bit digits held exactly in BF16; the digit products up to the eighth level are summed exactly
 * in FP32 accumulators (the leading four levels each in their own) and combined in double-float,
 * so every update element carries an error of about 2^-47 of |L_r| |L_c| (an FP64 dot product of
 * 32 terms: up to about 2^-48).  on = 0: FP64 fused multiply-adds.  The diagonal-block factors,
 * the panel solves and the triangular solves stay in FP64 either way.  Ignored by handles whose
 * solver is double-float.  The step graphs are re-recorded on the next step. */
icwf_status icwf_set_emulated_update(icwf_handle h, int32_t on);

/* icwf_step replays each time step as a captured CUDA graph (recorded on the first call, one
 * graph per parity of the ping-pong matrix buffers; re-recorded after icwf_set_regularisation)
 * unless per-kernel timing (icwf_profile_enable) is on.  on = 0 launches the step's kernels
 * directly instead; on = 1 (default) uses the graphs. */
icwf_status icwf_set_step_graphs(icwf_handle h, int32_t on);

/* Diagnostic: poll budget of the in-kernel spin waits on global flags (the look-ahead tickets of
 * the blocked Cholesky factorisation and the block flags of the triangular solves).  polls >= 0:
 * such a wait gives up after that many polls, sets the timeout flag and the kernel continues
 * without its input (results are then meaningless and the call returns ICWF_ERR_TIMEOUT);
 * polls < 0 restores the compiled-in limits (well under a second of polling).  Waits on
 * shared-memory barriers that guard asynchronous copies (the tensor-core assembly, the cluster
 * triangular solve) always keep their 2-second limit, so that no copy can land after its kernel
 * has released its memory.  icwf_init_* reset the budget to the defaults. */
icwf_status icwf_set_wait_limit(icwf_handle h, int64_t polls);

/* The handle's CUDA stream (a cudaStream_t) for callers that record events on it. */
icwf_status icwf_get_stream(icwf_handle h, void** stream);

/* Per-kernel device timing.  While enabled, every kernel launch of icwf_step is bracketed by
 * CUDA events on the handle's stream and its duration accumulated per kernel family.
 * icwf_profile_read fills up to n entries: names (static strings), total ms and launch
 * counts; it returns the number of families in *n_out. */
icwf_status icwf_profile_enable(icwf_handle h, int32_t on);
icwf_status icwf_profile_reset(icwf_handle h);
icwf_status icwf_profile_read(icwf_handle h, int32_t n, const char** names, double* ms,
                              int64_t* launches, int32_t* n_out);

/* Text of the last failure on h (or of the last failed icwf_create / pool call if h is NULL). */
const char* icwf_last_error(icwf_handle h);

/* --- observables without device allocation ------------------------------------------------- */

/* Size of the library's fixed observables work area (bytes) and the largest grid it serves. */
#define ICWF_OBS_STATIC_BYTES 9437184u
#define ICWF_OBS_STATIC_MAX_GRID 524288u

/* Same observables as icwf_observables, computed without allocating any device memory during the
 * call.  For hosts whose allocator policy forbids device allocation after start-up (an application
 * that reserves its device memory in one arena when it starts, or a serving path that must not
 * allocate).  icwf_observables allocates its work buffers on its first call; this entry point uses
 * one fixed work area of ICWF_OBS_STATIC_BYTES bytes compiled into the library as a static device
 * array, which every GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  It copies its results into the caller's host
 * arrays and waits for the handle's stream, so it must be called outside any stream capture.
 * Limits: nx * nR <= ICWF_OBS_STATIC_MAX_GRID and nx, nR <= 4096, else ICWF_ERR_ARG.
 * The first call on a device looks up the work area's device address (once per device, with that
 * device made current for the lookup).  All calls share the one work area, so calls that overlap
 * on the GPU (two handles, streams or threads) race; the caller must serialise them.  Each call
 * overwrites every part of the work area that it reads, so nothing left by an earlier call needs
 * clearing.
 * The paper has no counterpart to this entry point (it is a deployment aid). */
icwf_status icwf_observables_static(icwf_handle h, icwf_obs* out);

/* --- serving pool: continuous batching of independent jobs -------------------------------- */

/* A pool admits jobs while their summed device footprint stays within hbm_budget_bytes and at
 * most max_jobs are live; pending jobs wait in arrival order.  Every icwf_pool_tick advances
 * every live job by one step.  By default each tick is one CUDA graph, instantiated once per live
 * set and parity pattern and launched with a single cudaGraphLaunch: first the grouped kernels,
 * one persistent velocity kernel (Eq. v1/v2 and the Euler positions) and one persistent
 * propagation kernel (the CWF equations' Strang step) per CWF precision, each over every
 * trajectory or CWF of every live job of that precision (a device table of the jobs; ragged N and
 * grids); then every job's remaining step (assembly, factorisations, RK4), captured into CUDA
 * graphs at the job's first tick (one per parity of its ping-pong matrix buffers) and added as
 * child graphs.  The jobs share no memory, so their child graphs overlap on the device.  Job
 * handles are owned by the pool after submission. */
icwf_status icwf_pool_create(size_t hbm_budget_bytes, int32_t max_jobs, icwf_pool* out);

/* Counters of a pool since creation. */
typedef struct {
  int64_t ticks;            /* icwf_pool_tick calls */
  int64_t graph_launches;   /* cudaGraphLaunch calls (at most one per tick) */
  int64_t graph_builds;     /* tick graphs instantiated (live-set or parity changes) */
  int64_t kernel_nodes;     /* kernels executed inside tick graphs */
  int64_t graph_job_steps;  /* job steps run inside tick graphs */
  int64_t eager_job_steps;  /* job steps launched directly (graphs off or capture failed) */
  int64_t group_nodes;      /* grouped (all-job) kernels executed inside tick graphs */
} icwf_pool_stats;

icwf_status icwf_pool_get_stats(icwf_pool pool, icwf_pool_stats* out);

/* on = 0 launches every job's kernels directly on its own streams at each tick (no graphs);
 * on = 1 (default) uses the captured tick graphs. */
icwf_status icwf_pool_set_graphs(icwf_pool pool, int32_t on);

/* on = 1 (default): tick graphs run the live jobs' velocities and propagation as grouped kernels
 * over all jobs (above); on = 0: every job's child graph holds its own velocity and propagation
 * kernels.  max_ctas > 0 caps the CTAs of each grouped kernel (its CTAs then loop over more work
 * items each, leaving SMs to the jobs' other kernels); 0 = one wave at full occupancy.  Results
 * are the same either way (the grouped kernels run the per-job kernels' arithmetic).  Takes effect
 * at the next tick (jobs' step graphs are recorded again when grouping changes). */
icwf_status icwf_pool_set_grouping(icwf_pool pool, int32_t on, int32_t max_ctas);

/* Hand an initialised job to the pool (the pool owns it from now on) to run n_steps steps.
 * *job_id identifies it in icwf_pool_poll. */
icwf_status icwf_pool_submit(icwf_pool pool, icwf_handle job, int64_t n_steps, int32_t* job_id);

/* One step of every live job; admits pending jobs first. *n_live and *n_finished (may be NULL)
 * report the live count after the tick and the jobs that finished in it. */
icwf_status icwf_pool_tick(icwf_pool pool, int32_t* n_live, int32_t* n_finished);

/* *state: 0 pending, 1 live, 2 finished, 3 failed.  When finished, fills *out (if not NULL)
 * with the job's final observables and releases its device memory. */
icwf_status icwf_pool_poll(icwf_pool pool, int32_t job_id, icwf_obs* out, int32_t* state);

icwf_status icwf_pool_destroy(icwf_pool pool);

#ifdef __cplusplus
}
#endif
#endif /* ICWF_H */
