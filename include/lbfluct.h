/*
 * lbfluct.h -- C ABI of the GB300 (sm_103a) fluctuating lattice Boltzmann library.
 *
 * The library steps a periodic D2Q9 lattice of the modified-equilibrium non-ideal
 * fluid model with thermal noise that satisfies the lattice fluctuation-dissipation
 * theorem of Gross, Adhikari, Cates & Varnik, "Thermal fluctuations in the lattice
 * Boltzmann method for non-ideal fluids", arXiv:1009.0254 (cited below as [GACV]).
 *
 * Conventions shared by every entry point
 *   - Return value: LB_OK (0) on success, a negative LB_E* code on failure.  Nothing
 *     aborts; lb_last_error(ctx) returns a message for the last failure on ctx.
 *   - Populations cross the ABI as FP64 arrays f[i][y][x] (index i*nx*ny + y*nx + x),
 *     i = 0..8 in the velocity order of [GACV] Eq. (Tmat): c = (0,0), (1,0), (0,1),
 *     (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).  They are the pre-collision
 *     populations f_i(r, t), i.e. the state right after streaming.
 *   - Moments are m_a = sum_i T_ai f_i with T of [GACV] Table I, a = 0..8 for the
 *     paper's a = 1..9 (rho, jx, jy, e, p_ww, p_xy, qx, qy, eps).
 *   - `loc` says where a caller buffer lives: LB_HOST (pageable or pinned host memory)
 *     or LB_DEVICE (device memory of the context's GPU).  The caller owns every
 *     buffer it passes; the library keeps no pointer to it after the call returns.
 *   - All GPU work is issued on the context's stream (lb_set_stream, default: the
 *     legacy default stream).  Calls that return data to the host synchronise that
 *     stream; lb_step does not.
 *   - One context may be used by one host thread at a time.
 */
#ifndef LBFLUCT_H
#define LBFLUCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define LB_OK 0
#define LB_EINVAL (-1)     /* argument out of range or inconsistent */
#define LB_ENOTPSD (-2)    /* noise covariance Xi(k) not positive semidefinite */
#define LB_ENOMEM (-3)     /* device allocation failed or workspace too small */
#define LB_ECUDA (-4)      /* a CUDA runtime call failed (message in lb_last_error) */
#define LB_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define LB_ESTATE (-6)     /* call out of order (e.g. lb_step before lb_set_params) */
#define LB_ENONFINITE (-7) /* a result holds NaN or infinity (served simulations) */
#define LB_ECANCELED (-8)  /* the request was cancelled (served simulations) */

/* storage precision of the populations */
#define LB_FP32 0          /* FP32 deviations f_i - fbar_i (72 bytes moved per node update) */
#define LB_FP16DEV 1       /* FP16 deviations, stored as (f_i - fbar_i) / w_i (36 bytes per node update);
                              arithmetic stays FP32; rounding to FP16 each step makes the mass
                              conserved only to that rounding */
#define LB_FP64 2          /* FP64 deviations and FP64 arithmetic throughout the step (the
                              correlated noise too, which then needs ny <= 4096); the sampled
                              spectra are FP32 transforms accumulated in FP64 */

/* noise modes, [GACV] Sec. IV */
#define LB_NOISE_OFF 0     /* deterministic (kT ignored) */
#define LB_NOISE_LW 1      /* spatially uncorrelated, covariance Xi(0), Eq. (noise-matrix-k0) */
#define LB_NOISE_FULL 2    /* spatially correlated, covariance Xi(k), Eq. (noise-yeo);
                              needs nx, ny powers of two, ny <= 8192 */
#define LB_NOISE_DIAG 3    /* "ideal gas-like": LW with the off-diagonal Xi_49 dropped */
#define LB_NOISE_FULL_RS 4 /* spatially correlated, covariance Xi(k) of Eq. (noise-yeo) at every k,
                              built in real space: Xi depends on k only through the lattice k^2 s
                              (Appendix B), affinely, so four white 2-vector fields nu_ab drawn per
                              node, each times a factor L_ab of Xi at s = 0, 4, 4, 16/3 and summed
                              over the 2x2 box {r, r-e_x, r-e_y, r-e_x-e_y} with the signs
                              a^dx b^dy (a, b = +-1), give xi_4, xi_9 with exactly that covariance
                              (no transform; any lattice size).  Needs Xi positive semidefinite
                              at s = 0 and s = 16/3.  Modes 5..8 as LB_NOISE_LW. */
#define LB_NOISE_LW_LOCAL 5 /* spatially uncorrelated with Xi(0) evaluated at each node's own
                              density rho(r) and sound speed c_s^2(rho(r)) (Sec. IV: the
                              uncorrelated noise applies to inhomogeneous systems with the local
                              values; Sec. V B): Cholesky of the local (4,9) block, a negative
                              pivot (a node in the spinodal region of an interface, where the
                              local block is not positive semidefinite) clamped to zero; same
                              draws as LB_NOISE_LW, identical to it at uniform density. */

/* equations of state, [GACV] Sec. II A (lb_set_eos) */
#define LB_EOS_LINEAR 0       /* p0 = cs2 rho (the linearised equation of state; default) */
#define LB_EOS_DOUBLE_WELL 1  /* Landau double well f0 = beta (rho - rhoV)^2 (rho - rhoL)^2,
                                 Eq. (f0-bulk): p0 = rho df0/drho - f0, c_s^2 = rho d2f0/drho2 */

/* factorisation of the noise matrix, [GACV] Sec. IV (xi = L nu with L L^T = Xi) */
#define LB_FACTOR_CHOLESKY 0   /* Cholesky of the lower-right block (default) */
#define LB_FACTOR_EIGEN 1      /* eigen-decomposition L = S diag(sqrt(e)) */

/* buffer locations */
#define LB_HOST 0
#define LB_DEVICE 1

/* warning bits returned by lb_warnings() */
#define LB_WARN_LOW_MACH 1 /* kT >= 0.1 sigma_s^2 rho0, [GACV] Eq. (low-mach) */

typedef struct lb_ctx lb_ctx;

/*
 * Device bytes a context of this size needs (populations, noise and statistics
 * scratch).  Pass a buffer of at least this size to lb_create to keep all device
 * memory under the caller's allocator.  Returns 0 for invalid sizes.
 */
size_t lb_workspace_bytes(int nx, int ny, int precision);

/*
 * Creates a context for a periodic nx x ny lattice (nx, ny >= 2) at rest with
 * uniform density rho0: f_i = fbar_i, the equilibrium of [GACV] Table II at u = 0
 * with the linearised equation of state p0 = cs2 rho (cs2 is the thermodynamic
 * sound speed squared; 1/3 gives fbar_i = w_i rho0).  `seed` keys the Philox4x32-10
 * noise: key = (seed mod 2^32, seed div 2^32).
 * workspace: device buffer of >= lb_workspace_bytes() bytes owned by the caller and
 * kept alive until lb_destroy, or NULL to let the library cudaMalloc its own.
 * The context uses the device that is current when lb_create is called.
 * Errors: LB_EINVAL (sizes, rho0 <= 0, cs2 <= 0, precision), LB_ENOMEM, LB_ECUDA.
 */
int lb_create(int nx, int ny, int precision, uint64_t seed, double rho0, double cs2,
              void* workspace, size_t workspace_bytes, lb_ctx** out);

/* Releases the context (and its own device memory, if it allocated any). */
int lb_destroy(lb_ctx* ctx);

/* Issue all later GPU work of ctx on `stream` (a cudaStream_t; NULL = legacy default). */
int lb_set_stream(lb_ctx* ctx, void* stream);

/*
 * Relaxation and noise, [GACV] Sec. III-IV.  lambda_a = -1/tau_a with tau_s for the
 * shear modes p_ww, p_xy, tau_b for the bulk mode e and tau_ghost for q_x, q_y and eps
 * (Table I).  Every tau must exceed 1/2 (Sec. III A), kT >= 0, kappa >= 0.
 * For noise_mode != LB_NOISE_OFF with kT > 0 the noise covariance Xi(k) of
 * Eq. (noise-yeo) must be positive semidefinite at every wavevector of this lattice
 * (Sec. III C, Fig. 5), else LB_ENOTPSD; its factors are computed here in FP64.
 * May be called again between steps; the lattice state is kept.
 */
int lb_set_params(lb_ctx* ctx, double kT, double kappa, double tau_s, double tau_b,
                  double tau_ghost, int noise_mode);

/*
 * Equation of state, [GACV] Sec. II A.  eos = LB_EOS_LINEAR restores p0 = cs2 rho with the
 * cs2 of lb_create; eos = LB_EOS_DOUBLE_WELL takes p0 = rho df0/drho - f0 of the Landau
 * double well f0 = beta (rho - rhoV)^2 (rho - rhoL)^2 (beta > 0, 0 <= rhoV < rhoL) in the
 * Table II equilibrium at every node.  The uniform rest state becomes the equilibrium at rho0
 * with p0(rho0); the linear theory about rho0 that sets the noise of the LW, DIAG, FULL and
 * FULL_RS modes takes c_s^2 = rho0 d2f0/drho2 (rho0) (it must be > 0 for those modes), and
 * LB_NOISE_LW_LOCAL takes c_s^2(rho(r)) at every node.  The populations are kept (their
 * stored deviations are re-based on the new rest state); the parameters of the last
 * lb_set_params are re-applied.  With FP32 storage a double-well lattice is stepped by the
 * TMA-staged kernel's double-well variant (the default tile of its noise mode), with FP16 and
 * FP64 storage by the plain step kernel.  LB_EINVAL for bad
 * arguments; FP16 and FP32 storage keep deviations from the rest state, so large density
 * contrasts lose more to rounding in FP16.
 */
int lb_set_eos(lb_ctx* ctx, int eos, double beta, double rhoV, double rhoL);

/*
 * lb_set_noise_factor: how the noise matrix is factored, [GACV] Sec. IV: LB_FACTOR_CHOLESKY
 * (default) or LB_FACTOR_EIGEN, L = S diag(sqrt(e)) with e the eigenvalues (largest first)
 * and S = [[cos t, -sin t], [sin t, cos t]], t in [0, pi) with tan 2t = 2 Xi49 / (Xi44 -
 * Xi99), of the coupled (4,9) block (Xi(0) for the uncorrelated modes, Xi(k) at
 * every k for the correlated mode); the other modes are uncoupled.  Both give noise of
 * covariance Xi; the realisations differ.  Applies to the current parameters and to later
 * lb_set_params calls.  LB_EINVAL for an unknown factor.
 */
int lb_set_noise_factor(lb_ctx* ctx, int factor);

/*
 * Advances nsteps >= 0 time steps of [GACV] Eq. (fluct-lin-lbe): stream (pull),
 * collide in moment space with the Table II equilibrium (Appendix B Laplacian),
 * add the noise of the chosen mode, transform back.  The collision at time t draws
 * its random numbers with counter (node y*nx+x, t mod 2^32, t div 2^32, tag): tag 0 per
 * node (words 0, 1: nu_5..nu_8, word 2: nu_4, nu_9), tag 2 per wavevector pair
 * (LB_NOISE_FULL), tag 3 per node (LB_NOISE_FULL_RS: word w gives field w of ++, +-, -+, --).  If
 * sampling is on (lb_set_sampling) the spectra are accumulated after every step
 * that brings the time to a multiple of `every`.  Asynchronous on the stream.
 * Errors: LB_ESTATE before lb_set_params, LB_ECUDA on launch failure.
 */
int lb_step(lb_ctx* ctx, int64_t nsteps);

/* Time index t of the current state (number of collisions done since t = 0). */
int lb_get_time(lb_ctx* ctx, int64_t* t);

/*
 * Replaces the state by pre-collision populations f (FP64, 9*nx*ny, layout above) and
 * sets the time index to t (which keys the next collision's noise).  Values are
 * rounded to the storage precision as deviations from fbar_i.
 */
int lb_set_populations(lb_ctx* ctx, const double* f, int loc, int64_t t);

/* Copies the current pre-collision populations (FP64, 9*nx*ny) into f. */
int lb_get_populations(lb_ctx* ctx, double* f, int loc);

/*
 * Moments of the current state.  If m != NULL it receives m_a(r) (FP64, 9*nx*ny,
 * m[a*nx*ny + y*nx + x]).  If sums != NULL it receives the FP64 lattice sums
 * {sum rho, sum jx, sum jy}, accumulated on the device in FP64 (Table I: these
 * three are conserved by the collision).
 */
int lb_moments(lb_ctx* ctx, double* m, int loc, double sums[3]);

/*
 * Turns on sampling of the spectra every `every` >= 1 steps into `nbins` >= 1 radial
 * bins of |k| over [0, pi sqrt(2)] (k components wrapped to (-pi, pi], k = 0 left
 * out); every = 0 turns sampling off.  Needs nx and ny powers of two (the transform
 * is a radix-2 FFT).  Resets the accumulators.
 */
int lb_set_sampling(lb_ctx* ctx, int every, int nbins);

/*
 * Running FP64 averages over the samples taken so far, per bin b < nbins:
 *   S_rho[b] = < |drho(k)|^2 >,  S_jl[b] = < |k.j(k)|^2 / k^2 >,
 *   S_jt[b]  = < |k x j(k)|^2 / k^2 >,  counts[b] = wavevectors in bin b,
 * with the unitary transform a(k) = n^-1/2 sum_r exp(i k.r) a(r) of [GACV] Sec. III
 * and drho = rho - rho0.  Their theories are Eqs. (struct-fact) and (momtm-fluct).
 * Any output pointer may be NULL.  *nsamples receives the number of samples.
 */
int lb_structure_factor(lb_ctx* ctx, int nbins, double* S_rho, double* S_jl, double* S_jt,
                        int64_t* counts, int64_t* nsamples);

/* Bitmask of LB_WARN_* raised by the last lb_set_params. */
int lb_warnings(lb_ctx* ctx);

/* Message of the last failure on ctx ("" if none); ctx == NULL gives the last
 * failure of a call that had no context (lb_create, lb_conserved_sums_static). */
const char* lb_last_error(lb_ctx* ctx);

/* Waits for all work issued on the context's stream. */
int lb_synchronize(lb_ctx* ctx);

/*
 * Kernel timing for roofline measurements: with every = k >= 1, CUDA events are recorded
 * on the context's stream around every k-th launch of the fused step kernel (k = 1: all of
 * them; a sample keeps the events' own cost out of a whole-run timing); 0 turns it off.
 * lb_kernel_time synchronises and returns the summed event time (ms) and the number of
 * timed launches since timing was set.  LB_EINVAL for every < 0.
 */
int lb_set_kernel_timing(lb_ctx* ctx, int every);
int lb_kernel_time(lb_ctx* ctx, double* ms, int64_t* launches);

/* Number of kernels this context has launched since lb_create (all kinds). */
int lb_launch_count(lb_ctx* ctx, int64_t* launches);

/* Row capacity of the static scratch used by lb_conserved_sums_static. */
#define LB_STATIC_MAX_ROWS 16384

/*
 * Allocation-free conserved sums, for callers that cannot call cudaMalloc (their device
 * memory is wholly owned by another allocator, or a latency-critical loop must not risk
 * the device-wide synchronisation of an allocation).  The paper has no counterpart: this
 * is the FP64 reduction behind lb_moments' sums, applied to populations the caller owns.
 *   f:      device pointer, FP64 populations f[i][y][x] (layout above), nx*ny*9 values
 *   sums:   device pointer, receives {sum rho, sum jx, sum jy} (FP64) when the stream
 *           reaches the work; nothing is copied to the host
 *   stream: a cudaStream_t (NULL = legacy default stream); the call returns without
 *           waiting for the result
 * Needs no context and allocates nothing: the per-row partial sums live in one static
 * device array of LB_STATIC_MAX_ROWS rows (384 KB) that every GPU which loads the library
 * holds until the process exits.  nx >= 1, 1 <= ny <= LB_STATIC_MAX_ROWS, else LB_EINVAL
 * (message in lb_last_error(NULL)).  The first call on a device looks up the array's
 * device address with the device current (no allocation); make that first call before
 * any stream capture.  All calls share the array, each writing the rows it reads, so two
 * calls whose GPU work overlaps (different streams, or different host threads on the
 * same device) race and may return wrong sums; order them on one stream.
 */
int lb_conserved_sums_static(const double* f, int nx, int ny, double* sums, void* stream);

/*
 * Batched ensembles: many independent periodic lattices ("replicas") stepped together.
 * Every replica is the model of [GACV] Sec. III with the noise of Sec. IV (any noise mode;
 * LB_NOISE_FULL needs nx, ny powers of two and ny <= 8192), in FP32 storage, with its own
 * size, seed and parameters, and follows the trajectory that lb_create/lb_step with the
 * same size, seed and parameters would give it (bitwise for a replica whatever the other
 * replicas are; up to FP32 rounding order against lb_step).  The step kernel covers every
 * replica in one persistent launch per time step; replicas with correlated noise add two
 * launches per size class (k-space synthesis, transform back) before it.  The noise
 * factor is Cholesky.
 *
 * lb_batch_workspace_bytes: device bytes of an ensemble of `count` lattices of sizes
 *   nx[r] x ny[r] (each side in [2, 8192]); 0 if the sizes are invalid.
 * lb_batch_create: like lb_create for every replica: seeds[r] keys replica r's Philox
 *   stream; rho0 and cs2 are common.  workspace NULL: the library allocates and owns
 *   device memory; else a 256-byte aligned caller buffer of at least
 *   lb_batch_workspace_bytes() that the caller keeps alive until lb_batch_destroy.
 *   Every replica starts at rest at time 0.
 * lb_batch_set_params: lb_set_params for replica `replica`, or for every replica when
 *   replica == -1; the same validation (lb_check_params), LB_EINVAL for LB_NOISE_FULL on
 *   a lattice whose sides are not powers of two.
 * lb_batch_autotune: times every tile shape of the batched step kernel on the whole
 *   ensemble (three runs of `steps` steps each, the fastest run counts) and keeps the
 *   fastest shape, then puts every replica back at
 *   rest at time 0 (populations set before are lost).  Needs parameters for every
 *   replica; synchronises the stream.
 * lb_batch_step: advances every replica by nsteps (asynchronous, one kernel per size
 *   class and one counter update per step, plus the spectra samples).
 * lb_batch_step_graph: the same, with the steps issued through a CUDA graph of
 *   steps_per_graph steps (captured on first use, replayed afterwards; a multiple of the
 *   sampling interval when sampling is on); leftovers run as lb_batch_step.  Results
 *   are identical to lb_batch_step.
 * lb_batch_get_time: the time t of replica `replica`.
 * lb_batch_set_populations / lb_batch_get_populations: as lb_set_populations /
 *   lb_get_populations for one replica (f holds nx[r]*ny[r]*9 doubles); setting also
 *   sets that replica's time to t.  Synchronise the stream.
 * lb_batch_sums: FP64 sums of (rho, jx, jy) of one replica.  Synchronises.
 * lb_batch_set_sampling: every `every` steps, the radial spectra of [GACV] Sec. V of
 *   every replica are accumulated (every = 0: off); nbins in [1, 1024]; every lattice
 *   side must be a power of two.  Clears the accumulated spectra.
 * lb_batch_structure_factor: as lb_structure_factor for one replica.
 * lb_batch_launch_count: kernels launched on behalf of the ensemble so far (a graph
 *   replay counts the kernels it contains).
 * lb_batch_tuning: the tile shape of the step kernel in use (tile_x x tile_y nodes per
 *   tile, `threads` threads per CTA) and the time per step lb_batch_autotune measured
 *   for it (0 before any autotune); any output pointer may be NULL.
 * lb_batch_last_error: message of the last failure on b (NULL b: of the last failed
 *   lb_batch_create, as lb_last_error(NULL)).
 */
typedef struct lb_batch lb_batch;
size_t lb_batch_workspace_bytes(int count, const int* nx, const int* ny);
int lb_batch_create(int count, const int* nx, const int* ny, const uint64_t* seeds, double rho0,
                    double cs2, void* workspace, size_t workspace_bytes, lb_batch** out);
int lb_batch_destroy(lb_batch* b);
int lb_batch_set_stream(lb_batch* b, void* stream);
int lb_batch_set_params(lb_batch* b, int replica, double kT, double kappa, double tau_s,
                        double tau_b, double tau_ghost, int noise_mode);
int lb_batch_autotune(lb_batch* b, int steps);
int lb_batch_step(lb_batch* b, int64_t nsteps);
int lb_batch_step_graph(lb_batch* b, int64_t nsteps, int64_t steps_per_graph);
int lb_batch_get_time(lb_batch* b, int replica, int64_t* t);
int lb_batch_set_populations(lb_batch* b, int replica, const double* f, int loc, int64_t t);
int lb_batch_get_populations(lb_batch* b, int replica, double* f, int loc);
int lb_batch_sums(lb_batch* b, int replica, double* sums);
int lb_batch_set_sampling(lb_batch* b, int every, int nbins);
int lb_batch_structure_factor(lb_batch* b, int replica, int nbins, double* S_rho, double* S_jl,
                              double* S_jt, int64_t* counts, int64_t* nsamples);
int lb_batch_launch_count(lb_batch* b, int64_t* launches);
int lb_batch_tuning(lb_batch* b, int* tile_x, int* tile_y, int* threads, double* ms_per_step);
const char* lb_batch_last_error(lb_batch* b);

/*
 * Request server: continuous batching of independent simulations.
 * Each request is one periodic lattice of the model of [GACV] Sec. III started at time 0,
 * at rest (uniform density rho0, zero velocity) or from the populations in `init`, with
 * the noise of Sec. IV in any mode
 * (LB_NOISE_OFF, LB_NOISE_LW, LB_NOISE_DIAG, or LB_NOISE_FULL for nx, ny powers of two and
 * ny <= 8192) keyed by its own seed, FP32 storage, advanced by `steps` time steps.  Its
 * trajectory is exactly the one lb_batch_* (and, up to FP32 rounding order, lb_step) gives
 * the same lattice, whatever else is served with it.  Correlated requests of one size share
 * one pair of k-space synthesis launches per step (Sec. IV, Eq. (noise-yeo)).
 *
 * lb_server_request_bytes: device bytes one request of that size and noise mode holds
 *   while admitted (both population buffers, plus the (xi_4, xi_9) field for
 *   LB_NOISE_FULL); 0 for an invalid size (sides in [2, 16384]).
 * lb_server_create: starts a scheduler thread on the current device.  hbm_budget_bytes
 *   bounds the sum of lb_server_request_bytes over admitted requests (their memory comes
 *   from a stream-ordered pool that keeps up to the budget cached); max_active bounds the
 *   number admitted at once (device tables are sized for it); max_chunk_steps bounds the
 *   steps issued between two admission decisions.  Requests are admitted in arrival order;
 *   one that does not fit the remaining budget lets later, smaller ones pass.
 * lb_server_submit: queues a request (thread-safe) and returns its id (> 0).  Validation
 *   happens here: LB_EINVAL for bad sizes/steps/parameters or LB_NOISE_FULL on a size
 *   that is not a power of two on both sides (or ny > 8192), LB_ENOTPSD
 *   as lb_check_params, LB_ENOMEM if the request alone exceeds the budget.
 * lb_server_poll: moves up to max_results completed results (oldest first) into out.
 * lb_server_wait: blocks until request `id` has completed (id <= 0: until every request
 *   submitted so far has) or timeout_s seconds have passed (LB_ETIMEOUT; < 0: no limit).
 * lb_server_fetch_populations: for a completed request submitted with keep_state = 1,
 *   copies its final FP64 populations (9*nx*ny doubles, layout as lb_get_populations) to
 *   host memory f and releases its device memory.  Until then that memory stays counted
 *   against the budget.  LB_EINVAL if the request is unknown, not finished or not kept.
 * lb_server_get_stats: counters since creation (times in seconds since lb_server_create).
 * lb_server_cancel: withdraws request `id`: a queued one at once, an admitted one at the
 *   next chunk boundary (its memory is released); its result then has status
 *   LB_ECANCELED.  LB_EINVAL if it is unknown or already completed.
 * lb_server_set_admission: requests of at least `large_nodes` lattice nodes (nx * ny) are
 *   admitted at most `max_large` at a time (later, smaller requests pass one that waits);
 *   max_large = 0 removes the limit (the default).  A lattice that fills the GPU alone gains
 *   no throughput from sharing it with another such lattice, and sharing delays both: with
 *   a limit the large requests complete in arrival order while small ones still run in
 *   the same launches.  LB_EINVAL for large_nodes < 1 or max_large < 0.
 * lb_server_inject_alloc_failures: fault injection on the host: the next `count`
 *   admissions behave as if the device allocation failed.  A failed allocation, injected
 *   or real (the pool could not grow), completes that request with status LB_ENOMEM
 *   without running, returns its budget and slot, and the server carries on.  A request
 *   with `init` also takes an FP64 staging plane (8*nx*ny bytes) from the pool while its
 *   state is uploaded at admission.
 * lb_server_destroy: drops queued requests, finishes the admitted ones, frees everything.
 * lb_server_last_error: message of the last failure of s (NULL s: of the last failed
 *   lb_server_create or lb_server_submit validation).
 * Results carry the FP64 conserved sums (rho, jx, jy) of the final state and the host
 * times of submission, admission and completion (completion = when the host saw the GPU
 * finish the chunk holding the request's last step).  A result whose sums are not finite
 * (a diverged run) has status LB_ENONFINITE.
 */
typedef struct lb_request {
    int nx, ny;
    int64_t steps;
    double rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost;
    int noise_mode;
    int keep_state;
    uint64_t seed;
    const double* init;   /* NULL: start at rest; else host FP64 pre-collision populations
                             f[i][y][x] (9*nx*ny, layout above) to start from at time 0,
                             copied by lb_server_submit (the caller may free it on return) */
} lb_request;

typedef struct lb_result {
    int64_t id;
    int status;           /* LB_OK, or LB_ETIMEOUT if a kernel gave up a bounded wait */
    int nx, ny;
    int state_kept;
    int64_t steps;
    double sums[3];
    double t_submit, t_admit, t_complete;
} lb_result;

typedef struct lb_server_stats {
    int64_t submitted, completed, queued, steps_issued;
    size_t bytes_in_use, bytes_peak, bytes_budget;
    double node_updates;  /* lattice node updates issued */
    double gpu_busy_s;    /* sum of the chunks' device durations */
    double t_first_admit, t_last_complete;
} lb_server_stats;

typedef struct lb_server lb_server;
size_t lb_server_request_bytes(int nx, int ny, int noise_mode);
int lb_server_create(size_t hbm_budget_bytes, int max_active, int max_chunk_steps, lb_server** out);
int lb_server_submit(lb_server* s, const lb_request* r, int64_t* id);
int lb_server_poll(lb_server* s, lb_result* out, int max_results, int* n);
int lb_server_wait(lb_server* s, int64_t id, double timeout_s, lb_result* out);
int lb_server_fetch_populations(lb_server* s, int64_t id, double* f);
int lb_server_get_stats(lb_server* s, lb_server_stats* st);
int lb_server_cancel(lb_server* s, int64_t id);
int lb_server_set_admission(lb_server* s, int64_t large_nodes, int max_large);
int lb_server_inject_alloc_failures(lb_server* s, int count);
int lb_server_destroy(lb_server* s);
const char* lb_server_last_error(lb_server* s);

/*
 * Host-only helpers (no GPU needed).
 * lb_noise_matrix: the 9x9 noise covariance Xi(k) of [GACV] Eq. (noise-yeo) for the
 * given parameters at wavevector (kx, ky), with k^2 the lattice symbol of Appendix B;
 * row-major into xi[81].
 * lb_check_params: the validation lb_set_params performs for an nx x ny lattice.
 */
/*
 * Self-test of the device-side timeout path (no fault involved): one CTA waits, with the
 * bounded wait the TMA step kernels use and a limit of limit_s seconds (0 < limit_s <= 10),
 * on an mbarrier armed for a transfer that is never issued.  Returns LB_ETIMEOUT and sets
 * *gave_up = 1 when the wait gave up as designed; the CUDA context stays usable.
 */
int lb_selftest_bounded_wait(double limit_s, int* gave_up);

int lb_noise_matrix(double rho0, double cs2, double kT, double kappa, double tau_s,
                    double tau_b, double tau_ghost, double kx, double ky, double* xi);
int lb_check_params(int nx, int ny, double rho0, double cs2, double kT, double kappa,
                    double tau_s, double tau_b, double tau_ghost, int noise_mode);

#ifdef __cplusplus
}
#endif

#endif /* LBFLUCT_H */
