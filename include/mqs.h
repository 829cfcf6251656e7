/*
 * mqs.h -- C ABI of the GB300 library for batched implicit-Euler time stepping
 * of the 2D eddy-current (magnetoquasistatic) finite-element model across
 * Multi-Level Monte Carlo samples and Parareal time slices.
 *
 * Method: Hahn & Schoeps, "Multi-Level Monte Carlo sampling with Parallel-in-
 * Time Integration for Uncertainty Quantification in Electric Machine
 * Simulation" (arXiv 2507.19246).  Sec. II-A (Eq. 1-7): the semi-discrete
 * Galerkin system M da/dt + K a = r advanced by implicit Euler,
 *     (M/dt + K) a_{k+1} = (M/dt) a_k + r(t_{k+1});
 * Sec. II-B (Eq. 8-9): Monte Carlo and telescoping MLMC estimators;
 * Sec. II-C (Eq. 12): the Parareal update.
 *
 * Conventions for every entry point:
 *  - Return value: MQS_OK (0) or a negative MQS_E* code.  On error the
 *    message of mqs_last_error() (thread-local, owned by the library, valid
 *    until the next call from the same thread) says what failed.  Errors leave
 *    the context usable unless the code is MQS_ECUDA from a sticky CUDA error.
 *  - Host arrays passed in are read during the call and stay owned by the
 *    caller.  Pointers documented as "host or device" may point to host memory
 *    or to device memory of the context's GPU; the library detects which.
 *  - Device state (meshes, batches, results) is owned by the context and lives
 *    until the matching free call or mqs_destroy.
 *  - Work is enqueued on the context's CUDA stream and runs asynchronously;
 *    calls that return values to host memory synchronise that stream.
 *  - All floating-point data are IEEE binary64 unless stated otherwise.
 */
#ifndef MQS_H
#define MQS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MQS_OK        0
#define MQS_EINVAL   -1   /* invalid argument (size, index, handle, order of calls) */
#define MQS_ENOMEM   -2   /* device or host allocation failed */
#define MQS_ECUDA    -3   /* CUDA runtime error */
#define MQS_ENOTCONV -4   /* a linear solve hit its iteration limit (strict mode only) */

/* arithmetic of the linear solves */
#define MQS_FP64   0      /* FP64 Jacobi-PCG */
#define MQS_MIXED  1      /* FP32 matrix values and SpMV inside FP64 PCG, FP64 residual replacement */

/* linear solver of the implicit-Euler systems (mqs_set_solver) */
#define MQS_SOLVER_PCG    0  /* batched Jacobi-preconditioned CG (default) */
#define MQS_SOLVER_BANDED 1  /* band Cholesky in reverse Cuthill-McKee order */

/* quantity of interest */
#define MQS_QOI_ENERGY 0  /* (1/N) sum_{k=1..N} 1/2 a_k^T K a_k (time-averaged magnetic energy) */
#define MQS_QOI_JOULE  1  /* (1/T) sum_k (a_{k+1}-a_k)^T M (a_{k+1}-a_k) / dt  (Eq. 26, mean joule loss) */

/* per-sample status bits returned by mqs_read_qoi */
#define MQS_ST_NOTCONV 1  /* some step's linear solve stopped at the iteration limit */
#define MQS_ST_NONFINITE 2 /* a residual norm became NaN or Inf */
#define MQS_ST_NOTSPD  4  /* a band Cholesky factorisation met a non-positive pivot */
#define MQS_ST_TIMEOUT 8  /* a wait between the CTAs of a cluster ran out of its iteration
                             limit; the lane's results are invalid */

typedef struct mqs_ctx mqs_ctx;

/* Last error message of the calling thread ("" if none). */
const char* mqs_last_error(void);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (e.g. a PyTorch stream handle) or NULL for the legacy default stream; the
 * stream is not owned.  *out receives the handle. */
int mqs_create(mqs_ctx** out, int device, void* cuda_stream);

/* Change the stream later calls enqueue on (not owned; NULL = default). */
int mqs_set_stream(mqs_ctx* ctx, void* cuda_stream);

/* Free all device state of the context and the context itself. */
int mqs_destroy(mqs_ctx* ctx);

/* Upload a P1 triangle mesh and build its shared sparsity pattern and the
 * per-region reference matrices (Sec. II-A, Eq. 4-5): for every material
 * region r, M_r = int_{region r} N_i N_j and K_r = int_{region r} grad N_i .
 * grad N_j, and for every source phase p the load vector F_p = sum over the
 * phase's triangles of coef_T int_T N_i.  Dirichlet nodes (A_z = 0) are
 * eliminated; the unknowns are the remaining ("free") nodes in increasing
 * node id.
 *   n_nodes, xy        host, [n_nodes][2] node coordinates (m)
 *   n_tri, tri         host, [n_tri][3] node ids (0-based)
 *   region             host, [n_tri] material region in [0, n_regions)
 *   n_regions          1..16
 *   dirichlet          host, [n_nodes] 1 = homogeneous Dirichlet node
 *   src_phase          host, [n_tri] source phase in [0, n_phases) or -1
 *   src_coef           host, [n_tri] winding sign / fill factor of the source
 *   n_phases           0..4
 *   mesh_id            out: handle
 * Errors: MQS_EINVAL for out-of-range ids, degenerate triangles, no free node,
 * or a free node with more than 32 neighbours. */
int mqs_upload_mesh(mqs_ctx* ctx, int32_t n_nodes, const double* xy,
                    int32_t n_tri, const int32_t* tri, const int32_t* region,
                    int32_t n_regions, const uint8_t* dirichlet,
                    const int32_t* src_phase, const double* src_coef,
                    int32_t n_phases, int32_t* mesh_id);

/* Free unknowns and nonzeros of the pattern of a mesh. */
int mqs_mesh_info(mqs_ctx* ctx, int32_t mesh_id, int32_t* n_free, int64_t* nnz);

/* Upload a batch of sample parameters xi (Sec. II-B).  Layout per sample:
 *   [sigma_0..sigma_{R-1}, nu_0..nu_{R-1}, J0, amp_0..amp_{P-1}, phase_0..phase_{P-1}]
 * (n_params = 2R + 1 + 2P), conductivity sigma_r (S/m) and reluctivity
 * nu_r = 1/mu_r (m/H) per region, current density scale J0 (A/m^2) and per
 * phase amplitude and phase shift (rad).  Phase p carries
 *   J_p(t) = J0 amp_p sin(2 pi f t - 2 pi p / P + phase_p).
 *   params      host or device, [n_samples][n_params], n_samples >= 1
 *   batch_id    out: handle */
int mqs_set_samples(mqs_ctx* ctx, int32_t mesh_id, int32_t n_samples, int32_t n_params,
                    const double* params, int32_t* batch_id);

/* Time window [t0, t_end] (s), supply frequency f (Hz) and QoI kind
 * (MQS_QOI_*) of a batch.  Must be called before mqs_propagate. */
int mqs_set_time(mqs_ctx* ctx, int32_t batch_id, double t0, double t_end,
                 double freq_hz, int32_t qoi_kind);

/* Select the linear solver used by later mqs_propagate calls on a batch
 * (MQS_SOLVER_PCG or MQS_SOLVER_BANDED).  Both solve Eq. 7's system
 * (M/dt + K) a_{k+1} = b each step.  The banded solver factors M/dt + K once
 * per sample and step size (band Cholesky after a reverse Cuthill-McKee
 * ordering of the free unknowns, n x (bw+1) doubles per factor) and then does
 * one forward and one backward substitution per step.  MQS_FP64: the factor
 * and the substitutions are FP64 (cg_tol and cg_max_iters are ignored).
 * MQS_MIXED: the factor and substitutions are FP32 and each step refines in
 * FP64 -- residual r = b - A x with the FP64 matrix, x += (L L^T)^-1 r --
 * until ||r||_2 <= cg_tol ||b||_2 or cg_max_iters sweeps (MQS_ST_NOTCONV). */
int mqs_set_solver(mqs_ctx* ctx, int32_t batch_id, int32_t solver);

/* Bandwidth of a mesh's reverse Cuthill-McKee ordering (used by the banded solver). */
int mqs_mesh_bandwidth(mqs_ctx* ctx, int32_t mesh_id, int32_t* bandwidth);

/* Run one MLMC level for every sample of the batch (Eq. 7, Eq. 9, Eq. 12):
 * the level-l solve with step dt_level and, if dt_prev > 0, the companion
 * level-(l-1) solve with step dt_prev on the same sample (Q_{l-1} of Eq. 9).
 * Both start from a(t0) = 0.  Step counts are (t_end - t0)/dt and must be
 * integers (relative tolerance 1e-9).
 *   level          MLMC level of the batch (recorded for mqs_mlmc_accumulate)
 *   n_slices       1: sequential time stepping; M > 1: the level-l solve runs
 *                  Parareal (Eq. 12) on M slices, coarse step coarse_factor *
 *                  dt_level; the step count must be a multiple of
 *                  M * coarse_factor
 *   max_par_iters  Parareal iteration limit (<= M)
 *   par_tol        Parareal stop: max_n ||U_n^k - U_n^{k-1}||_2 / max_n ||U_n^k||_2 <= par_tol
 *   precision      MQS_FP64 or MQS_MIXED
 *   cg_tol         per-step PCG stop: ||b - A a||_2 <= cg_tol ||b||_2
 *   cg_max_iters   per-step PCG iteration limit (>= 1)
 *   par_iters_out  out (may be NULL): Parareal iterations taken (max over samples), 0 if sequential
 * A sample whose solve hits cg_max_iters gets status MQS_ST_NOTCONV; the call
 * still returns MQS_OK.  The call synchronises the stream only when Parareal
 * runs (to test the stopping rule once per iteration). */
int mqs_propagate(mqs_ctx* ctx, int32_t batch_id, int32_t level, double dt_level,
                  double dt_prev, int32_t n_slices, int32_t coarse_factor,
                  int32_t max_par_iters, double par_tol, int32_t precision,
                  double cg_tol, int32_t cg_max_iters, int32_t* par_iters_out);

/* Quantities of interest of the last propagate: qoi[s][0] = Q_l, qoi[s][1] =
 * Q_{l-1} (0 when dt_prev was 0), status[s] = MQS_ST_* bits.
 *   qoi      host or device, [n_samples][2]
 *   status   host or device, [n_samples] (may be NULL)
 * Synchronises the stream when a destination is host memory. */
int mqs_read_qoi(mqs_ctx* ctx, int32_t batch_id, double* qoi, int32_t* status);

/* Final state a(t_end) of the last propagate: which = 0 the level-l solve,
 * 1 the level-(l-1) solve.  a: host or device, [n_samples][n_free], free
 * unknowns in increasing node id. */
int mqs_read_state(mqs_ctx* ctx, int32_t batch_id, int32_t which, double* a);

/* Solver counters of the last propagate (host array of MQS_N_STATS):
 *   [0] PCG iterations summed over all lanes
 *   [1] implicit-Euler solve-steps executed (Parareal: every fine and coarse step run)
 *   [2] serial-equivalent solve-steps (the sequential solves this replaces)
 *   [3] free unknowns n_free
 *   [4] lane-iterations / [6] lane-steps of the sequential-stepping kernel
 *   [5] lane-iterations / [7] lane-steps of the Parareal coarse-sweep kernel */
#define MQS_N_STATS 8
int mqs_read_stats(mqs_ctx* ctx, int32_t batch_id, double* stats);

/* Instrumentation.  mqs_profile(ctx, 1) clears and starts recording CUDA-event
 * timings around every launch of the two time-stepping kernels on the
 * stream of each launch; 0 stops.  mqs_profile_read fills out[7] (host):
 *   [0] kernels launched by this library in this process since it was loaded
 *   [1] recorded launches / [2] their summed duration (ms) of the stepping kernel
 *   [3] recorded launches / [4] their summed duration (ms) of the coarse-sweep kernel
 *   [5] / [6] time (ms) during which at least one stepping / coarse-sweep
 *       launch ran (launches on several streams overlap, so this can be less
 *       than the sum)
 * and synchronises the stream. */
int mqs_profile(mqs_ctx* ctx, int32_t enable);
int mqs_profile_read(mqs_ctx* ctx, double* out);
/* Measured arithmetic peak of device `device` (restored as current device
 * afterwards): fused multiply-add chains on every SM, timed with CUDA events on
 * `cuda_stream` (NULL: default stream).  precision MQS_FP64 measures the FP64
 * rate (the roofline of the FP64 stepping kernels), MQS_MIXED the FP32 rate.
 * *tflops receives TFLOP/s (2 flop per FMA).  About 0.1 s; allocates and frees
 * 8 bytes of device memory.  Instrumentation, not part of the method. */
int mqs_measure_peak(int32_t device, void* cuda_stream, int32_t precision, double* tflops);

/* Launch intervals of the recorded launches of one kind (0 stepping, 1
 * coarse sweep): out[2 j], out[2 j + 1] = start and end (ms) of launch j
 * relative to the mqs_profile(ctx, 1) call, for j < min(*count, max_launches);
 * *count receives the number recorded.  Synchronises the stream. */
int mqs_profile_trace(mqs_ctx* ctx, int32_t kind, double* out, int32_t max_launches,
                      int32_t* count);

/* Apply a sample's matrix: y[s] = X_s x[s] with X = M (which = 0), K (1) or
 * A = M/dt + K (2) for every sample s of the batch; x, y host or device,
 * [n_samples][n_free]. */
int mqs_apply(mqs_ctx* ctx, int32_t batch_id, int32_t which, double dt,
              const double* x, double* y);

/* MLMC estimator state (Eq. 9).  mqs_mlmc_reset clears n_levels level
 * records; mqs_mlmc_accumulate adds the batch's Y = Q_l - Q_{l-1} (Q_0 alone
 * on level 0) to the record of `level` (compensated two-pass mean and
 * sum of squared deviations per batch, merged across batches by the pairwise
 * update of Chan, Golub & LeVeque); mqs_mlmc_readout returns per level
 * [N_l, mean_l, var_l (unbiased)] in levels[n_levels][3] (host), the estimate
 * sum_l mean_l and the statistical RMSE sqrt(sum_l var_l / N_l). */
int mqs_mlmc_reset(mqs_ctx* ctx, int32_t n_levels);
int mqs_mlmc_accumulate(mqs_ctx* ctx, int32_t batch_id, int32_t level);
int mqs_mlmc_readout(mqs_ctx* ctx, double* levels, double* estimate, double* rmse);

/* Sequential implicit-Euler stepping that allocates no memory.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory while they run -- a host application driving
 * the GPU from a real-time or signal-safe path, where cudaMalloc may block or
 * take locks, or a runtime that partitions all device memory into its own
 * pools at start-up, so that a cudaMalloc would fail or compete with them.
 * They own every input and output; the library works in a static device
 * scratch array of 32 MiB that each GPU loading the library holds until the
 * process exits.
 *
 * It runs the same stepping kernel as mqs_propagate on n_lanes independent
 * lanes from a(t0) = 0 (Eq. 7 with the same Jacobi-PCG and the same QoI
 * definitions), with matrices the caller has assembled:
 *   device          CUDA device ordinal (current during the call; the caller's
 *                   current device is restored before the call returns)
 *   cuda_stream     cudaStream_t or NULL; all work is enqueued on it
 *   n, rowptr, colidx, nnz   device, CSR pattern of the n x n free-unknown matrices
 *                   (int32, columns ascending within a row, at most 32 per row)
 *   n_lanes         lanes (samples) >= 1
 *   A, M, K         device, values [nnz][n_lanes] (lane fastest) of A = M/dt + K,
 *                   of M, and of K (K only for MQS_QOI_ENERGY, else may be NULL)
 *   Dinv            device, [n][n_lanes] inverse diagonal of A
 *   n_phases, F     0..4 phases; device [n_phases][n] load vectors
 *   src_amp, src_phase  host or device, [n_lanes][n_phases]: J0 amp_p and phase_p
 *                   of each lane (J_p(t) = amp sin(2 pi f t - 2 pi p / P + phase))
 *   t0, dt, n_steps, freq_hz, qoi_kind, cg_tol, cg_max_iters   as in mqs_propagate
 *   a_out           device, [n][n_lanes]: final state (also used as work space)
 *   qoi_out         device, [n_lanes]: the quantity of interest
 *   status_out      device, [n_lanes] MQS_ST_* bits, or NULL
 * Limit: 6 * n * n_lanes doubles plus about 72 bytes per lane and the tile
 * table must fit in the 32 MiB array (for example n = 19584 with 32 lanes);
 * larger problems return MQS_EINVAL with the required size in the message.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call reuses the same array and leaves its contents behind; the call clears
 * the parts that must start at zero itself.  Calls whose work overlaps on the
 * GPU (different streams or threads without ordering) race on the array. */
int mqs_propagate_noalloc(int32_t device, void* cuda_stream, int32_t n, const int32_t* rowptr,
                          const int32_t* colidx, int64_t nnz, int32_t n_lanes, const double* A,
                          const double* M, const double* K, const double* Dinv,
                          int32_t n_phases, const double* F, const double* src_amp,
                          const double* src_phase, double t0, double dt, int32_t n_steps,
                          double freq_hz, int32_t qoi_kind, double cg_tol, int32_t cg_max_iters,
                          double* a_out, double* qoi_out, int32_t* status_out);

/* Lane slots: how many independent sample solves ("lanes") the banded
 * stepping keeps resident on the GPU at once in its throughput form (one
 * 256-thread CTA per lane, several per SM).  These are the "cores" n_c of the
 * paper's batching model (Sec. II-D, Eq. 24-25): a level with N samples runs
 * in about N (1 + C_{l-1}/C_l) / slots batches, and the finest level can give
 * each sample floor(slots / (N_L (1 + C_{L-1}/C_L))) lanes for Parareal slices. */
int mqs_lane_slots(mqs_ctx* ctx, int32_t precision, int32_t* slots);

/* Test hook, for tests of the failure path only (0 = off, the default).
 * MQS_TEST_HOOK_STALL: on this context, the first wait of every banded
 * stepping lane that runs as one CTA per lane (cluster kernels with one CTA)
 * waits on a count that nothing reaches, so that the bounded wait runs out
 * and the lane reports MQS_ST_TIMEOUT with an invalid result.  Other contexts
 * and other launch shapes are not affected. */
#define MQS_TEST_HOOK_STALL 1
int mqs_set_test_hook(mqs_ctx* ctx, int32_t hook);

/* ---------------------------------------------------------------- serving
 * A request server on a context: continuous batching of independent sample
 * solves of different meshes and step counts (the MLMC samples of Sec. II-B
 * and the Parareal slices of Sec. II-C as separate requests).
 *
 * Requests wait in arrival order.  mqs_server_progress admits them, in that
 * order, while their device footprint (per-sample values, a band Cholesky
 * factor per step size, lane vectors) fits the HBM budget, as one batch per
 * free stream; batches on different streams run at the same time, so a
 * request admitted while others run starts as soon as SMs free up.  Every
 * lane finishes on its own and reports through host-mapped memory, so a
 * request completes when its own solves have, whatever its batch still does.
 * All lanes use one launch shape (a 256-thread CTA each, work vector in L2),
 * so a request's result does not depend on the other requests it ran with.
 * Solves are FP64 with the banded direct solver (Eq. 7).  The server holds
 * the context's meshes by id: do not free a mesh while its requests live.
 * Single-threaded: call the server functions from one thread. */
typedef struct mqs_server mqs_server;

#define MQS_REQ_LEVEL 0   /* MLMC level sample: the level solve (dt, n_steps) from a(t0) = 0
                             and, if dt_prev > 0, the level-(l-1) solve (dt_prev, n_steps_prev)
                             on the same parameters; qoi = finished Q_l, Q_{l-1} (Eq. 9, 26) */
#define MQS_REQ_SLICE 1   /* Parareal slice: n_steps fine steps (dt) from global step k0,
                             starting from a_init (or zero); qoi[0] = the slice's raw QoI
                             sum (what Parareal adds over slices), final state into a_out */

/* hbm_budget: bytes of device memory admitted requests may hold (<= 0: 80%
 * of the free memory at creation); n_streams: batches in flight (1..32);
 * max_batch_lanes: lanes per batch (a level sample with a companion solve has
 * two); freq_hz: supply frequency f of the source (Eq. 5). */
int mqs_server_create(mqs_ctx* ctx, int64_t hbm_budget, int32_t n_streams,
                      int32_t max_batch_lanes, double freq_hz, mqs_server** out);
int mqs_server_destroy(mqs_server* srv);

/* Queue one request; *request_id receives its id.  params: host,
 * [n_params] in the layout of mqs_set_samples (copied).  a_init: host [n_free]
 * (copied) or NULL; a_out: device [n_free] (caller-owned, written before the
 * request completes) or NULL; both only for MQS_REQ_SLICE.  MQS_EINVAL for bad
 * arguments or a footprint larger than the whole budget. */
int mqs_server_submit(mqs_server* srv, int32_t mesh_id, int32_t n_params, const double* params,
                      int32_t kind, int32_t qoi_kind, double t0, double dt, int32_t n_steps,
                      double dt_prev, int32_t n_steps_prev, int64_t k0, const double* a_init,
                      double* a_out, int64_t* request_id);

/* Device bytes a request with `lanes` solves (1, or 2 for a level sample with
 * its companion) on mesh_id holds while admitted. */
int mqs_server_footprint(mqs_server* srv, int32_t mesh_id, int32_t qoi_kind, int32_t lanes,
                         int64_t* bytes);

/* Non-blocking scheduler pass (retire, release, admit, launch); *in_flight and
 * *queued (may be NULL) receive the request counts afterwards. */
int mqs_server_progress(mqs_server* srv, int32_t* in_flight, int32_t* queued);

/* Up to max completed requests since the last call, in completion order:
 * ids[c], qoi[c][2], status[c] (MQS_ST_* bits, may be NULL), times[c][3] =
 * submit, admit and completion time (s, host clock from server creation; may
 * be NULL); *count receives how many. */
int mqs_server_poll(mqs_server* srv, int32_t max, int64_t* ids, double* qoi, int32_t* status,
                    double* times, int32_t* count);

/* Release a batch or a mesh (a mesh must have no live batch). */
int mqs_free_batch(mqs_ctx* ctx, int32_t batch_id);
int mqs_free_mesh(mqs_ctx* ctx, int32_t mesh_id);

#ifdef __cplusplus
}
#endif
#endif /* MQS_H */
