/*
 * fm.h -- C ABI of the GB300 library for monitored free-fermion trajectories
 * (B. Fan, C. Yin, A. M. Garcia-Garcia, "Entanglement dynamics of monitored
 * noninteracting fermions on graphics processing units", arXiv 2508.18468).
 *
 * What is computed.  A trajectory is the Slater determinant of App. A,
 * |psi> = prod_k (sum_j U_jk c_j^dag)|vac>, with U an L x N matrix,
 * U^dag U = 1, on a ring of L sites (Sec. II) or an Lx x Ly torus (Sec. IV),
 * half filled, started from the Neel / checkerboard state (App. A).  One step
 * t -> t + dt is
 *   1. propagation U <- exp(-i H~ dt) U, H~_ij = J on nearest-neighbour bonds
 *      (App. A; H of Sec. II), as a dense complex GEMM;
 *   2. the measurement:
 *      projective (App. A, Eqs. (A1), (A2)): every site is measured with
 *        probability 1 - exp(-gamma dt), sites in ascending order, outcome 1
 *        iff the uniform draw u < p_j = C_jj of the current state; a click
 *        applies n_j, a no-click 1 - n_j (Eq. (A2) read with '+');
 *      homodyne / QSD (App. A, Eq. (A4)): U <- exp(dW + (2<n> - 1) gamma dt) U
 *        with dW_i = sqrt(gamma dt) xi_i, xi_i ~ N(0,1), <n_i> = sum_k |U_ik|^2;
 *   3. re-orthonormalisation (App. A) by CholeskyQR2:
 *      G = U^dag U, G = R^dag R, U <- U R^-1, twice.
 * Observables: the entanglement entropy S_A = -sum f(lambda), f(x) =
 * x ln x + (1-x) ln(1-x), lambda the eigenvalues of C_A = U_A U_A^dag
 * (Sec. II), and the mutual information I = S_A + S_B - S_{A u B} (Sec. IV).
 *
 * Randomness.  Draws come from Philox4x32-10 (Salmon et al., SC'11) at
 * counter (site, step, traj_id_lo, tag | traj_id_hi << 8), key (seed_lo,
 * seed_hi); tag 1 = projective (u_select from words 0-1, u_outcome from words
 * 2-3), tag 2 = homodyne (Box-Muller normal).  A uniform double is
 * ((w_a >> 5) * 2^26 + (w_b >> 6)) * 2^-53.
 *
 * Conventions common to every call.
 *  - Status codes only; nothing throws or aborts across the ABI.
 *  - A CUDA, numeric or timeout error inside a state is sticky: later calls
 *    on that state return FM_ESTATE.  Argument errors (FM_EINVAL) are not
 *    sticky.  fm_last_error() tells what happened.
 *  - Device memory: the caller allocates one device workspace of
 *    fm_workspace_bytes() bytes and owns it; the library never allocates or
 *    frees device memory on the stepping path and never frees caller memory.
 *    The host-side fm_state object is allocated by fm_init_state and freed by
 *    fm_destroy.
 *  - Work is issued on the caller's CUDA stream (cudaStream_t passed as
 *    void*; NULL = legacy default stream).  fm_step is asynchronous; calls
 *    that return host values synchronise that stream.
 *  - Matrices are column-major.  Site indices are 0-based; on the torus site
 *    (x, y) has index x + Lx*y.  Entropies are in nats.
 *  - U is exported as complex128 (interleaved re, im doubles).
 */
#ifndef FM_H
#define FM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FM_OK = 0,
  FM_EINVAL = 1,     /* bad argument (sizes, indices, overlapping A/B, ...) */
  FM_ENOMEM = 2,     /* workspace smaller than fm_workspace_bytes() */
  FM_ECUDA = 3,      /* a CUDA runtime / driver call failed */
  FM_ENUMERIC = 4,   /* non-finite values or a non-positive Cholesky pivot */
  FM_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  FM_ESTATE = 6      /* the state holds an earlier (sticky) error */
} fm_status;

/* FM_PROJECTIVE: projective occupation measurements (Eqs. (A1), (A2)) after the
 * propagation of each fixed step.  FM_HOMODYNE: the QSD protocol of Eq.
 * (QSD_evo) as a split step (propagate, then weight).  FM_HOMODYNE_RK4: the
 * same equation integrated as App. A does, one classical fourth-order
 * Runge-Kutta step with the noise and <n>_t of the step's start held fixed
 * (the hopping enters through H~ itself, nearest neighbours, so no propagator
 * is used); the fixed-dt split step is its dt -> 0 limit.  FM_PROJECTIVE_POISSON:
 * the projective protocol as App. A runs it, in continuous time: events of a
 * Poisson process of total rate gamma N (N = L/2), each measuring one site drawn
 * uniformly, exp(-i H~ tau) between events (stencils of Bessel-function taps);
 * a step advances every trajectory by dt; QR every reorth_interval steps.
 * Draws of event e: Philox counter (e, e >> 32, traj_lo, tag | traj_hi << 8);
 * tag 3: waiting time -ln(1 - u) / (gamma N) with u from words 0-1, site
 * floor(u' L) with u' from words 2-3; tag 4: Born draw from words 0-1 (53-bit
 * uniforms as for the other protocols). */
typedef enum { FM_PROJECTIVE = 0, FM_HOMODYNE = 1, FM_HOMODYNE_RK4 = 2, FM_PROJECTIVE_POISSON = 3 } fm_protocol;

/* FM_FP64: every step in float64 / complex128.
 * FM_MIXED: U held as complex float32; the propagation, Gram and triangular
 * products run on the tensor cores as split-fp16 products with float32
 * accumulation; Cholesky pivots, entropies and eigenvalues in float64. */
typedef enum { FM_FP64 = 0, FM_MIXED = 1 } fm_precision;

typedef struct {
  int32_t Lx, Ly;           /* lattice; Ly == 1 is the ring.  L = Lx*Ly even, N = L/2 */
  int32_t batch;            /* trajectories advanced together, >= 1 */
  int32_t protocol;         /* fm_protocol */
  int32_t precision;        /* fm_precision */
  int32_t reorth_interval;  /* >= 1.  Projective: CholeskyQR2 every k steps.
                               Homodyne: first CholeskyQR pass every step, the
                               second every k steps */
  int32_t event_capacity;   /* projective outcome log entries kept (0 = no log) */
  int32_t tile_config;      /* mixed precision only, 0 = defaults; see FM_TILE_* (fm_autotune picks it) */
  double J, dt, gamma;      /* hopping, time step, monitoring rate (per site) */
  uint64_t seed;            /* Philox key */
  uint64_t traj_id;         /* trajectory b of the batch has id traj_id + b */
} fm_params;

/* fm_params.tile_config of the mixed-precision path: bits 0-1 the output tile
 * width of the propagation and Gram products (0 automatic: 128 up to N = 8192,
 * 256 beyond when N % 256 == 0; 1: 128; 2: 256, needs N % 256 == 0); bits 2-4 g
 * the height of the tile raster groups, 2^(g+1) row tiles (0: 8); bits 5-6 d:
 * with reorth_interval > 1, the first CholeskyQR product of the steps that no
 * second pass follows drains its fp32 tensor-memory accumulators (which round
 * toward zero) into registers every 2^(d+1) K-blocks of 64 (0: 2; 3 is invalid);
 * bit 7: the first CholeskyQR factorisation of a batch of three or more runs as one
 * chain of launches per trajectory (up to four streams) instead of two halves of
 * the batch.  Any other bit set is FM_EINVAL.  Bits 0-4 and 7 do not change a
 * single result (each output is one fixed-order sum per tile, each factor one
 * trajectory's); bits 5-6 change the rounding of U between second passes
 * (U^dag U - 1 stays ~1e-6 there). */
#define FM_TILE_BN_AUTO 0
#define FM_TILE_BN_128 1
#define FM_TILE_BN_256 2
#define FM_TILE_GROUP(g) ((g) << 2)
#define FM_TILE_DRAIN(d) ((d) << 5)
#define FM_TILE_CHOL_CHAINS (1 << 7)

/* One projective measurement: trajectory b of the batch, step index (t/dt
 * before the step), site, the outcome draw u, Born probability p, outcome. */
typedef struct {
  int64_t step;
  int32_t traj;
  int32_t site;
  double u;
  double p;
  int32_t outcome;
  int32_t pad;
} fm_event;

typedef struct fm_state fm_state;

/* Device bytes the state for *p needs; 0 if *p is invalid. */
size_t fm_workspace_bytes(const fm_params* p);

/* Build the propagator on the host (FP64 plane-wave sum, App. A), upload it,
 * and put every trajectory in the Neel / checkerboard state at step 0.
 * d_workspace: caller-owned device buffer of ws_bytes >= fm_workspace_bytes(p),
 * 256-byte aligned.  cuda_stream: cudaStream_t or NULL.  Synchronises. */
fm_status fm_init_state(const fm_params* p, void* d_workspace, size_t ws_bytes,
                        void* cuda_stream, fm_state** out);

/* Advance every trajectory of the batch by nsteps >= 0 steps.  Asynchronous. */
fm_status fm_step(fm_state* s, int32_t nsteps);

/* How fm_step applies exp(-i H~ dt) (App. A).  FM_PROP_DENSE (the default): the
 * dense L x L complex GEMM.  FM_PROP_BANDED: the same product as stencils --
 * the propagator is circulant along each lattice direction (P = P_x (x) P_y on
 * the torus) and its taps fall below 1e-15 beyond a half-width of ~8 sites at
 * dt = 0.05; the taps above 1e-15 are kept (every tap on tiny lattices), so
 * results agree with the dense product to that level.  FM_EINVAL if the
 * stencil would be wider than 41 taps (large J dt).  Synchronises. */
enum { FM_PROP_DENSE = 0, FM_PROP_BANDED = 1 };
fm_status fm_set_propagation(fm_state* s, int32_t mode);

/* Per-trajectory monitoring rates (host array of `batch` doubles >= 0).  Under
 * FM_PROJECTIVE_POISSON the event times of each trajectory become those of the
 * new rate from t = 0 (events already past stay applied). */
fm_status fm_set_gammas(fm_state* s, const double* gammas);

/* Restart trajectory b from the Neel state at step 0 with a new id and rate
 * (continuous batching: a finished slot takes the next request). */
fm_status fm_reset_trajectory(fm_state* s, int32_t b, uint64_t traj_id, double gamma);

/* Steps trajectory b has taken since its (re)start. */
fm_status fm_steps_done(fm_state* s, int32_t b, int64_t* out);

/* S_A (nats) of trajectory b, A = host array of n distinct sites.  FP64
 * Householder tridiagonalisation + bisection on the GPU.  Synchronises.
 * Mixed precision with reorth_interval k > 1: between second CholeskyQR passes
 * U is orthonormal only to ~1e-6..1e-5, so this call, fm_entropy_async,
 * fm_mutual_info, fm_density_correlation, fm_particle_covariance and fm_copy_U
 * first run the pending second pass when the step count is not a multiple of
 * k (span(U) -- the state -- is unchanged; U becomes orthonormal to < 1e-7).
 * fm_occupations, fm_orthonormality_error and fm_save read U as it is. */
fm_status fm_entropy(fm_state* s, int32_t b, const int32_t* sites, int32_t n, double* S_out);

/* Asynchronous S_A of trajectory b at the current point of the step sequence.
 * The rows of A are gathered and C_A is formed on the caller's stream, in
 * order with the steps (one of the workspace's C_A buffers: as many as fit in
 * 4 GiB, between 4 and 64, 16 N^2 bytes each); the FP64
 * eigen-solve (Householder tridiagonalisation, about 5 launches per row of
 * C_A) is issued by library-owned host threads, each onto its own low-priority
 * stream (1 to 4 threads: as many as fit their scratch in 1 GiB, so that small
 * eigen-solves run side by side; tickets may then complete out of order).
 * From the first call on, fm_step runs its kernels on a high-priority stream
 * ordered after and before the caller's stream by events, so later steps
 * proceed while the eigen-solve fills what their kernels leave of each SM.
 * *ticket identifies the result for fm_entropy_wait.  Up to 64 results may be
 * outstanding (a 65th call first waits for the oldest); a call while every
 * C_A buffer still waits for its eigen-solve makes the caller's stream wait
 * for the oldest to release its buffer.  Results live in a small pinned host
 * buffer the state allocates on first use.  A launch error of the library
 * thread is reported by fm_entropy_wait (FM_ECUDA, sticky). */
fm_status fm_entropy_async(fm_state* s, int32_t b, const int32_t* sites, int32_t n, int64_t* ticket);

/* *ready = 1 if the entropy of `ticket` is ready (fm_entropy_wait then returns
 * without waiting for it), else 0.  Never blocks. */
fm_status fm_entropy_ready(fm_state* s, int64_t ticket, int32_t* ready);

/* Block until the entropy of `ticket` is ready and return it. */
fm_status fm_entropy_wait(fm_state* s, int64_t ticket, double* S_out);

/* How fm_entropy, fm_entropy_async and fm_mutual_info compute S_A.
 * FM_EE_FULL (default): the eigenvalues lambda of C_A as above.
 * FM_EE_SKETCH (mixed precision only): for orthonormal orbitals C is a
 * projector, so lambda (1 - lambda) = sigma^2 with sigma the singular values of
 * the cross block C_AB = U_A U_B^dag (B the complement of A), and the terms of
 * S_A (Sec. II) depend on sigma^2 only.  A randomized subspace iteration on C_AB
 * (complex64 products with U, float64 orthonormal bases, rank r = 128, 256,
 * ... up to min(1024, N/2)) finds the sigma above the noise, whose squares are
 * the FP64 eigenvalues of an r x r Rayleigh-Ritz matrix formed with exact
 * products.  The rank grows until the (r/8)-th smallest sigma^2 is below 1e-9;
 * if it never is, the full method runs instead.  Subsystems or complements
 * below 512 sites always take the full method.  The state keeps a snapshot of
 * U for this (asynchronous tickets keep theirs in their C_A buffer).
 * FM_EE_AUTO (mixed precision): the sketch when A and its complement both
 * have at least 1024 sites, the full method otherwise (the measured crossover:
 * at 512 sites the full method is faster).  FM_EINVAL for FM_EE_SKETCH or
 * FM_EE_AUTO on an FP64 state, or an unknown method.  Synchronises. */
enum { FM_EE_FULL = 0, FM_EE_SKETCH = 1, FM_EE_AUTO = 2 };
fm_status fm_set_entropy_method(fm_state* s, int32_t method);

/* The last synchronous FM_EE_SKETCH entropy: the rank it settled on (0 if the
 * full method ran), its convergence value (the (r/8)-th smallest sigma^2) and
 * whether it fell back to the full method.  Any pointer may be NULL. */
fm_status fm_entropy_sketch_info(fm_state* s, int32_t* rank, double* check, int32_t* fell_back);

/* I = S_A + S_B - S_{A u B} for trajectory b; A and B disjoint host arrays. */
fm_status fm_mutual_info(fm_state* s, int32_t b, const int32_t* A, int32_t nA,
                         const int32_t* B, int32_t nB, double* I_out);

/* Density-density correlation of Eq. (2) for trajectory b, per displacement:
 * c_out[d] = (1/L) sum_i C_{i,i+d}, C_ij = -D_ij D_ji = -|(U U^dag)_ij|^2, the
 * partner site i + d taken with periodic wrap in x and y, d = dx + Lx dy
 * (0 <= dx < Lx, 0 <= dy < Ly); c_out[0] = 0 (the paper uses i != j only).
 * On the ring C(r) = c_out[r], r = 1 .. L/2.  c_out: host array of L doubles.
 * C is formed in the state's precision (complex128 or complex64 products),
 * accumulated in float64.  Synchronises. */
fm_status fm_density_correlation(fm_state* s, int32_t b, double* c_out);

/* Particle-number covariance of Eq. (GAB) for trajectory b, the integral read
 * as the lattice sum: G_AB = -sum_{i in A, j in B} C_ij = sum |(U_A U_B^dag)_ij|^2
 * for disjoint host site lists A and B (overlap: FM_EINVAL).  Synchronises. */
fm_status fm_particle_covariance(fm_state* s, int32_t b, const int32_t* A, int32_t nA, const int32_t* B,
                                 int32_t nB, double* G_out);

/* U of trajectory b -> host complex128 array with leading dimension ld >= L. */
fm_status fm_copy_U(fm_state* s, int32_t b, void* host_c128, int64_t ld);

/* Overwrite U of trajectory b from host complex128 (checkpoint restore, tests). */
fm_status fm_set_U(fm_state* s, int32_t b, const void* host_c128, int64_t ld);

/* <n_i> = sum_k |U_ik|^2 of trajectory b -> host array of L doubles. */
fm_status fm_occupations(fm_state* s, int32_t b, double* host_n);

/* max_kl |(U^dag U - 1)_kl| of trajectory b over the columns k in `cols`
 * (host array, 1 <= ncols <= min(N, 64) entries; all l), in float64 on the GPU. */
fm_status fm_orthonormality_error(fm_state* s, int32_t b, const int32_t* cols, int32_t ncols,
                                  double* err);

/* Move up to `cap` logged projective events into host `out`, oldest first;
 * *count = number written, *dropped = events lost to a full log since the
 * last call.  Synchronises. */
fm_status fm_take_events(fm_state* s, fm_event* out, int32_t cap, int32_t* count, int64_t* dropped);

/* Replay mode for the fixed-step projective protocol (App. A, Born rule and Eqs.
 * (A1), (A2)): from the next fm_step on, the measurement of site `site` by trajectory
 * `traj` at step index `step` (t/dt before the step, as in fm_event) takes the listed
 * `outcome` (0 or 1) instead of comparing its Philox draw with the Born weight.  Which
 * sites are measured still follows the Philox selection draws; listed measurements
 * that the selection does not make are ignored.  The u and p fields of the entries
 * are ignored, so the events another state logged (fm_take_events) can be passed
 * straight in, e.g. to hold a mixed-precision run on the outcome sequence of an FP64
 * run through near ties.  A forced measurement is logged with u = -1 (a forced click)
 * or u = 2 (a forced no-click).  Forcing an outcome of Born weight 0 (a click where
 * C_jj = 0, a no-click where C_jj = 1) is undefined and ends in FM_ENUMERIC.
 * events: host array of n <= fm_params.event_capacity entries (the list is kept in
 * the workspace), 0 <= step < 2^31, each (step, traj, site) at most once; n = 0
 * clears the list.  FM_EINVAL for other protocols.  Synchronises. */
fm_status fm_force_outcomes(fm_state* s, const fm_event* events, int32_t n);

/* Checkpoint: U (as stored), step counters, rates and ids to / from a file.
 * Philox is counter based, so a restored run continues bit-identically. */
fm_status fm_save(fm_state* s, const char* path);
fm_status fm_load(fm_state* s, const char* path);

/* CUDA graphs.  When enabled, fm_step replays captured graphs of whole step
 * periods (2 * reorth_interval steps, started at a multiple of the period;
 * the remaining steps run eagerly), removing per-kernel launch overhead.
 * The first replay captures the graph (on a library-owned stream) and
 * synchronises.  Results are bit-identical to eager stepping.  Phase timing
 * is not recorded inside graphs.  Projective states whose measurements read
 * the step's event count back to size their launches -- the grid-wide FP64
 * per-event kernels (few trajectories or L > 2048) and the mixed-precision
 * block update -- and continuous-time states always step eagerly. */
fm_status fm_set_graphs(fm_state* s, int32_t enable);

/* Phase timing (tracing).  When enabled, each phase of fm_step and fm_entropy
 * is bracketed by CUDA events on the state's stream.  fm_phase_times
 * synchronises, adds the elapsed milliseconds of every completed phase since
 * the last call into ms[0..FM_NPHASES-1] and the number of timed launches
 * into counts[] (either may be NULL), then resets.  Phases: */
enum { FM_PH_PROPAGATE = 0, FM_PH_MEASURE = 1, FM_PH_GRAM = 2, FM_PH_CHOLESKY = 3, FM_PH_TRMM = 4,
       FM_PH_ENTROPY = 5, FM_NPHASES = 6 };
fm_status fm_set_timing(fm_state* s, int32_t enable);
fm_status fm_phase_times(fm_state* s, double* ms, int64_t* counts);

/* The guard of the mixed-precision second CholeskyQR pass (App. A, "QR after each
 * step").  The second pass factors G = U^dag U = 1 + E to first order (T = 1 - F, F
 * the strict upper part of E plus half its diagonal, E measured in float64 on the
 * diagonal); that leaves U^dag U - 1 = -(F^dag F + F^2 + F^dag^2) + O(E^3), whose
 * entries are at most 3 (N o^2 + o d) + (3/4) d^2 with d, o the largest diagonal and
 * off-diagonal |E|.  The Gram's epilogue records d and o per trajectory; when that
 * bound exceeds 1e-7 for any trajectory of the batch, one more closed-form pass runs
 * (decided on the device, so graphs replay it too); if the E it then measures still
 * exceeds the bound, the state fails with FM_ENUMERIC rather than continue less
 * orthonormal than 1e-6.
 * *checks: second passes run since init; *extra_passes: of which needed the extra
 * pass; maxima[0..3] (host array of 4, may be NULL): the largest d and o seen by the
 * second passes, then by the extra passes, since the previous call (reset by the
 * call).  FP64 states (a float64 Cholesky every pass) report zeros.  Synchronises. */
fm_status fm_reorth_stats(fm_state* s, int64_t* checks, int64_t* extra_passes, double* maxima);

/* Result of fm_autotune. */
typedef struct {
  int32_t tile_config;      /* best fm_params.tile_config */
  int32_t reorth_interval;  /* best fm_params.reorth_interval */
  double ms_per_step;       /* its device time per step of the whole batch */
  double ortho_err;         /* its largest max|U^dag U - 1| after the checked steps that end a
                               period (a second CholeskyQR pass) */
  int32_t tried;            /* configurations timed */
  int32_t rejected;         /* of which over the orthonormality tolerance */
  double ortho_mid;         /* the same after the checked steps inside a period (first pass only) */
} fm_tuning;

/* Pick tile_config and reorth_interval for the workload *p by measurement
 * (the re-orthonormalisation interval of App. A is a free parameter of the
 * method; the tile shape is not part of it).  One state of *p is built in the
 * caller's workspace (ws_bytes >= fm_workspace_bytes(p), any tile_config);
 * for every candidate -- tile width 128 / 256 (mixed precision; 256 only when
 * N % 256 == 0) x raster groups of 8 / 16 / 32 row tiles x reorth_interval
 * 1, 2, 4, ... <= max_reorth -- the trajectories restart from the Neel state,
 * run 2 * reorth_interval warm-up steps, then `steps` timed steps (rounded up
 * to a whole number of 2 * reorth_interval; CUDA events on the stream, CUDA
 * graphs when use_graphs != 0), then 2 * reorth_interval single steps after
 * each of which max|U^dag U - 1| over 64 sampled columns of the first and
 * last trajectory is measured.  The fastest candidate whose error stays
 * <= ortho_tol after the steps that end a period (second pass done) and
 * <= 100 ortho_tol after the others wins (observables first complete a
 * period that is still open, see fm_entropy); if none does, the fastest with
 * reorth_interval = 1.  Mixed precision then also measures, against the winner,
 * its first-pass drain intervals of 4 and 8 K-blocks (reorth_interval > 1) and
 * then one Cholesky chain per trajectory (batches of three or more).
 * Synchronises; the workspace holds nothing useful afterwards. */
fm_status fm_autotune(const fm_params* p, void* d_workspace, size_t ws_bytes, void* cuda_stream,
                      int32_t steps, int32_t max_reorth, double ortho_tol, int32_t use_graphs,
                      fm_tuning* out);

/* Limits of fm_entropy_noalloc. */
#define FM_NOALLOC_MAX_SITES 1024
#define FM_NOALLOC_MAX_N 512

/* S_A (nats) of a Slater determinant held by the caller, computed without
 * allocating any device memory.  The paper has no counterpart of this call: it
 * serves callers that cannot call cudaMalloc, such as an application whose own
 * memory pool already holds nearly all of the device memory, or a loop that
 * must not pay the device-wide synchronisation that freeing memory implies.
 *   d_U    device complex128 U, L x N column-major (ld = L), read only;
 *   sites  host array of n distinct site indices in [0, L);
 *   d_S    device double receiving S_A;
 *   cuda_stream  cudaStream_t or NULL; the call is asynchronous on it.
 * Limits: n <= FM_NOALLOC_MAX_SITES, N <= FM_NOALLOC_MAX_N, L <= 65536;
 * larger sizes return FM_EINVAL without touching the GPU.  The scratch is one
 * fixed array of about 13 MB in the library's static device memory that every
 * GPU loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  Each call writes every scratch word it
 * reads, so nothing carries over from the previous call.  The site list is
 * copied into the gather kernel's launch parameters, so `sites` may be freed
 * as soon as the call returns, and the call makes no host-to-device copy.
 * n == 0 writes S = 0.  The same FP64 Householder + bisection method as
 * fm_entropy. */
fm_status fm_entropy_noalloc(const void* d_U, int32_t L, int32_t N, const int32_t* sites, int32_t n,
                             double* d_S, void* cuda_stream);

/* Several states in one CUDA graph (App. A's step, batched across lattice sizes).
 * A group captures one period of every member state -- P steps, P the least common
 * multiple of the members' 2 * reorth_interval -- into a single graph in which each
 * state's kernels form their own branch, so that the batches of different L (and
 * protocol or precision) advance together in one cudaGraphLaunch and their kernels
 * overlap on the device.  The states keep their workspaces and streams; the group
 * owns only its streams, events and graph.  Member states must be graph-capable:
 * not FM_PROJECTIVE_POISSON, and no projective state whose measurements read event
 * counts back (mixed precision, or the grid-wide FP64 path: fewer than 64
 * trajectories or L > 2048); P <= 256.  FM_EINVAL otherwise, or for a state listed
 * twice.  cuda_stream: the stream the graph replays on (cudaStream_t or NULL). */
typedef struct fm_group fm_group;
fm_status fm_group_create(fm_state* const* states, int32_t n, void* cuda_stream, fm_group** out);

/* Advance every member by nsteps, a multiple of the group period, from a step count
 * that is a multiple of it (FM_EINVAL otherwise).  The first call, and the first after
 * a member's propagation, forced outcomes or tuning changed, captures the graph
 * (synchronising the members' streams); later calls only replay it, nsteps / P
 * launches.  The caller's stream first waits for every member's stream, and every
 * member's stream then waits for the replays, so other calls on a member stay in
 * order.  Results are bit-identical to stepping each state alone.  Asynchronous. */
fm_status fm_group_step(fm_group* g, int32_t nsteps);

/* The group period P (0 for NULL); the last error message of the group. */
int32_t fm_group_period(const fm_group* g);
const char* fm_group_last_error(const fm_group* g);

/* Synchronise the replay stream and free the group (not its states).  NULL is allowed. */
void fm_group_destroy(fm_group* g);

/* Launches of library kernels issued on this state since init. */
int64_t fm_kernel_launches(const fm_state* s);

/* Last error message of this state ("" if none); valid until the next call. */
const char* fm_last_error(const fm_state* s);

/* Free the host-side state (not the caller's workspace).  NULL is allowed. */
void fm_destroy(fm_state* s);

/* Library version string. */
const char* fm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FM_H */
