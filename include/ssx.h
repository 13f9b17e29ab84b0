/*
 * ssx.h -- C ABI of the GB300 surface-source-extension solver.
 *
 * The library solves the source subproblem of W. W. Symes, "Efficient
 * Computation of Extended Surface Sources" (arXiv 2203.16573), eqn:esis:
 *
 *     given the medium, choose h on the line z = z_s minimising
 *     || S h - d ||^2 + alpha || A h ||^2,   (A h)(x, t) = |x - x_s| h(x, t)
 *
 * by Algorithm 1 (preconditioned CG on the weighted normal equation
 * eqn:normpart) with the time-reversal preconditioner of eqn:defprecond /
 * eqn:winvcomp, or by plain CG on the Euclidean normal equation.
 *
 * Conventions shared by every call
 * --------------------------------
 * Units: km, s, km/s, g/cm^3 (kappa = rho v^2 in GPa). All gathers are
 * row-major [nt][n] float64 arrays in DEVICE memory (time-major: sample n of
 * every trace is contiguous). The caller owns every buffer it passes and keeps
 * it alive until the call's work on `stream` has finished; the library owns
 * its internal wavefields, slabs and Krylov vectors (allocated by
 * ssx_set_geometry / ssx_set_velocity_model, freed by ssx_destroy).
 * Every call is enqueued on the caller's stream (ordered after the caller's
 * prior work on it, and the caller's later work is ordered after it); calls
 * that return host results (ssx_solve_source_subproblem) synchronise.
 * No call throws; each returns an ssx_status. The message of the last failure
 * is available from ssx_last_error. A context is not thread-safe.
 * Environment: SSX_GRAPHS=0 makes contexts created afterwards launch every
 * time step directly instead of replaying captured CUDA graphs (same kernels
 * and results; for profilers, which rebuild a graph on every replay).
 * SSX_LOG_TUNING=1 makes them print, to stderr, the time per step of every
 * tile configuration the phase autotuner tries (a diagnostic).
 *
 * Discretisation (section "Synthetic models and simulation"): staggered grid,
 * order 2 in time and 2k in space, fields FP32 on the device; sampling by
 * linear interpolation in depth, injection by its adjoint; an absorbing
 * sponge of n_sponge points padded outside the physical grid. The discrete
 * transpose is exact (Appendix A; dot-product test to FP32 rounding).
 */
#ifndef SSX_H
#define SSX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssx_ctx ssx_ctx;

typedef enum {
    SSX_OK = 0,
    SSX_ERR_ARG = 1,            /* invalid argument or call order        */
    SSX_ERR_CUDA = 2,           /* a CUDA runtime call failed            */
    SSX_ERR_CFL = 3,            /* time step violates the CFL bound      */
    SSX_ERR_OOM = 4,            /* device allocation failed              */
    SSX_ERR_BREAKDOWN = 5,      /* <p,q> <= 0 or <g,r> <= 0 in Algorithm 1 */
    SSX_ERR_NONFINITE = 6,      /* a Krylov scalar became NaN/Inf        */
    SSX_ERR_NOT_CONVERGED = 7   /* maxit reached above rtol (h is valid) */
} ssx_status;

/* Solver modes of ssx_solve_source_subproblem / ssx_normal_apply. */
enum {
    SSX_MODE_PCG = 0,   /* the paper's method: weighted normal equation
                           (eqn:normpart) + preconditioner (eqn:defprecond) */
    SSX_MODE_CG = 1     /* plain CG, W_m = W_d = I, M = I (the paper's
                           comparison in "Preconditioned CG iteration")     */
};

/* Weight operators of ssx_weight_apply. */
enum {
    SSX_W_D = 0,        /* W~_d at the receiver line (eqn:wdef)                  */
    SSX_W_M = 1,        /* W~_m on the source line (wcomp, prefactor -1)         */
    SSX_W_M_INV = 2     /* W~_m^{-1} = sym Lambda~ on the source line (eqn:winvcomp) */
};

typedef struct {
    int nx, nz;          /* physical grid points (x, z), each >= 8             */
    double h;            /* grid step, km (same in x and z)                    */
    double dt;           /* time step, s                                       */
    int nt;              /* time steps = samples per trace                     */
    int space_order;     /* 2k in {2, 4, 6, 8}                                 */
    int n_sponge;        /* absorbing points padded on every side, >= 0        */
} ssx_grid_desc;

typedef struct {
    double z_s;          /* extended-source line depth, km                     */
    int ix_line0;        /* first physical column of the source line           */
    int n_line;          /* source-line points (columns ix_line0 ..)           */
    double z_r;          /* receiver line depth, km (!= z_s)                   */
    int ix_rec0;         /* first physical column of the receivers             */
    int n_rec;           /* receivers                                          */
    double x_s;          /* physical source position for A (eqn:penop), km     */
    double dz_datum;     /* thin-slab datum distance, km (paper: 0.1)          */
} ssx_geom_desc;

typedef struct {
    long long kernel_launches;   /* kernels enqueued by this context (graph nodes counted) */
    long long point_updates;     /* grid-point steps of all sweeps (one v + p update each) */
    long long sweeps;            /* forward + adjoint sweeps                               */
    double sweep_ms;             /* event-timed device time of the sweeps (timing mode)    */
    long long timed_steps;       /* step-kernel launches inside timed sweeps               */
    double timed_point_updates;  /* grid-point steps inside timed sweeps                   */
    int tile_cfg[6];             /* chosen configuration of the full grid, z_s slab, z_r slab
                                    (forward, adjoint each): cfg + 16 if the sweep is one
                                    cooperative launch, -1 if not chosen yet               */
} ssx_stats;

/* Version string of the library. */
const char *ssx_version(void);

/* Create a context for one grid. `stream` is a cudaStream_t (NULL = legacy
 * default stream). Returns SSX_ERR_ARG for out-of-range descriptors. */
int ssx_create(ssx_ctx **out, const ssx_grid_desc *grid, void *stream);

/* Free the context and every device buffer it owns (synchronises). */
int ssx_destroy(ssx_ctx *ctx);

/* Message of the last failing call on ctx ("" if none). Owned by ctx. */
const char *ssx_last_error(const ssx_ctx *ctx);

/* Set the medium: v_dev is the physical velocity v[nz][nx] (km/s, float32,
 * device, row-major), rho the constant density (g/cm^3). kappa = rho v^2
 * (section "Synthetic models and simulation", constant density as in the
 * paper's models). Checks the CFL bound v_max dt/h * sqrt(2) sum|c_m| < 1
 * (SSX_ERR_CFL). */
int ssx_set_velocity_model(ssx_ctx *ctx, const float *v_dev, double rho);

/* Set the acquisition: the source line z = z_s and receiver line z = z_r
 * (eqn:fwd's P_s, P_r), the penalty centre x_s (eqn:penop) and the thin-slab
 * datum distance (eqn:lamnear). Allocates the two thin slabs and the Krylov
 * vectors. Lines must lie at least k + 1 rows inside the padded grid. */
int ssx_set_geometry(ssx_ctx *ctx, const ssx_geom_desc *geom);

/* d = S h: pressure-source gather h [nt][n_line] on z_s -> pressure gather
 * d [nt][n_rec] on z_r (eqn:sdef; one forward sweep from rest). */
int ssx_forward(ssx_ctx *ctx, const double *h_dev, double *d_dev);

/* h = S^T d: exact discrete transpose of ssx_forward (eqn:sadj1, Appendix A;
 * one reverse-time sweep). */
int ssx_adjoint(ssx_ctx *ctx, const double *d_dev, double *h_dev);

/* out = W in for which in {SSX_W_D, SSX_W_M, SSX_W_M_INV} (eqn:winvcomp,
 * wcomp, eqn:wdef): one forward and one adjoint sweep on the thin slab.
 * Gathers are [nt][n_rec] for SSX_W_D, [nt][n_line] otherwise. */
int ssx_weight_apply(ssx_ctx *ctx, int which, const double *in_dev, double *out_dev);

/* out = Lambda~ in (transpose = 0, eqn:lamtilde) or Lambda~^T in (transpose =
 * 1, eqn:lamtransp): the unsymmetrised thin-slab pressure-to-source map on
 * the source line, -8 (V+_{zs,zs+dz})^T Pi_0 S+ Pi_1^T and its exact
 * transpose. Their mean is W~_m^{-1}. Gathers [nt][n_line]. */
int ssx_lambda_apply(ssx_ctx *ctx, int transpose, const double *in_dev, double *out_dev);

/* h = 4 (V+_{zs,zr})^T d: the time-reversal approximate inverse of S
 * (eqn:approxinv; "multiply by -2, apply the transpose of V+, multiply by
 * -2"): d [nt][n_rec] injected as a vertical load at the receivers, one
 * reverse-time sweep, v_z read out on the source line into h [nt][n_line]. */
int ssx_time_reversal_inverse(ssx_ctx *ctx, const double *d_dev, double *h_dev);

/* g = M^{-1} r = D W~_m^{-1} D r, D = (I + alpha A^T A)^{-1/2}
 * (eqn:defprecond). alpha >= 0 multiplies ||A h||^2. */
int ssx_precond_apply(ssx_ctx *ctx, double alpha, const double *r_dev, double *g_dev);

/* q = N p: SSX_MODE_PCG: S^T W~_d S p + alpha A^T W~_m A p (eqn:normpart);
 * SSX_MODE_CG: S^T S p + alpha A^T A p. */
int ssx_normal_apply(ssx_ctx *ctx, int mode, double alpha, const double *p_dev, double *q_dev);

/* Solve the source subproblem by Algorithm 1 from h_0 = 0 with
 * r_0 = S^* d (S^T W~_d d for SSX_MODE_PCG, S^T d for SSX_MODE_CG).
 * Stops when ||r_k||_2 <= rtol ||r_0||_2 or after maxit updates of h.
 * d_dev [nt][n_rec] in; h_out_dev [nt][n_line] out (device).
 * resid_hist_host (host, maxit + 1 doubles, may be NULL) receives ||r_k||_2;
 * iters_out (host, may be NULL) the number of updates made. Krylov vectors,
 * scalars and reductions are float64 on the device; one 56-byte device-to-host
 * read per iteration (the 7 Krylov scalars) decides the stop. Returns SSX_ERR_NOT_CONVERGED if maxit
 * was reached above rtol (h_out is still the last iterate), SSX_ERR_BREAKDOWN
 * if <p_k,q_k> <= 0 or <g_k,r_k> <= 0 (h_out holds the last good iterate). */
int ssx_solve_source_subproblem(ssx_ctx *ctx, const double *d_dev, double alpha,
                                int maxit, double rtol, int mode, double *h_out_dev,
                                double *resid_hist_host, int *iters_out);

/* Solve n independent source subproblems at once (a survey's shots, or the
 * requests of a server), one per context (ctxs[i]: model and geometry set;
 * grids, nt and geometry may differ, the space order may not; no context twice).
 * Every phase of Algorithm 1 runs as one kernel launch per time step over all
 * active shots' sweeps (one shot's forward and adjoint sweeps advance in
 * lockstep inside those launches); the Krylov vectors, scalars and stopping
 * tests are per shot and a shot leaves the launches once it has stopped, so
 * each result equals the shot's solo ssx_solve_source_subproblem.
 * d_dev[i] / h_out_dev[i]: device gathers of shot i; alphas[i] host array;
 * hist (host, may be NULL): n x (maxit + 1) residual norms, row i for shot i;
 * iters / status (host, may be NULL): per-shot updates and ssx_status.
 * All work runs on ctxs[0]'s stream, ordered after every shot's stream.
 * Returns SSX_OK if the batch ran (per-shot outcomes in status). */
int ssx_solve_batch(ssx_ctx *const *ctxs, int n, const double *const *d_dev, const double *alphas,
                    int maxit, double rtol, int mode, double *const *h_out_dev, double *hist,
                    int *iters, int *status);

/* Gradient in the velocity model of Phi(c, h) = ||S[c] h - d||^2 +
 * alpha ||A h||^2 at fixed h (eqn:esis). At h = the subproblem's minimiser
 * (ssx_solve_source_subproblem with SSX_MODE_CG solves that Euclidean
 * problem) Phi is stationary in h, so this is the gradient of the reduced
 * objective that variable projection minimises over c (eqn:esi and the
 * paragraph after eqn:esis). Computed by the discrete adjoint state method
 * (the route the paper takes to exact adjoints): a forward sweep of S h
 * keeping the wavefield before every checkpoint_every-th step, then the
 * transposed sweep driven by 2 (S h - d), segment by segment backwards, each
 * segment's forward pressures recomputed from its checkpoint, accumulating
 * sum_n pbar^{n+1} (p^{n+1} - A_p p^n) / kappa in FP64 (kappa = rho c^2 enters
 * only the pressure update), folded onto the physical model through
 * kappa = rho c^2 and the sponge's edge replication. The sponge strength
 * (set from max c) is held fixed. Results do not depend on checkpoint_every.
 * h_dev [nt][n_line], d_dev [nt][n_rec] in (device); grad_dev [nz][nx]
 * float64 out (device, dPhi/dc in the units of the model); objective_host
 * (may be NULL) receives Phi and makes the call synchronise; with NULL the
 * call returns once its work is queued on the context's stream (ordered
 * before later work on the caller's stream), so the gradients of several
 * contexts (a survey's shots) run concurrently. Device memory:
 * (nt / checkpoint_every) x 3 + checkpoint_every + 11 padded fields, kept by
 * the context for reuse. Errors: SSX_ERR_ARG for null pointers,
 * checkpoint_every < 1 or alpha < 0. */
int ssx_velocity_gradient(ssx_ctx *ctx, const double *h_dev, const double *d_dev, double alpha,
                          int checkpoint_every, double *grad_dev, double *objective_host);

/* Phi of the context's last ssx_velocity_gradient (synchronises the context's
 * stream). SSX_ERR_ARG if no gradient was computed yet. */
int ssx_last_objective(ssx_ctx *ctx, double *objective_host);

/* A solve server with continuous batching. Requests (each a full source
 * subproblem: grid, geometry, model, data, alpha, stopping rule, output
 * buffer) queue in submission order and are admitted while their estimated
 * device memory fits hbm_budget_bytes; admitted requests join the solves
 * already running at the next round and share every kernel launch with them
 * (ssx_solve_batch's engine); a finished request releases its memory for the
 * queue. Each result equals the request's solo ssx_solve_source_subproblem.
 * All requests use the server's space order. Caller-owned buffers (model,
 * data, output) must stay valid until the request is done. Not thread-safe. */
typedef struct ssx_server ssx_server;
int ssx_server_create(ssx_server **out, int space_order, size_t hbm_budget_bytes, void *stream);
/* Queue one request; *id_out identifies it. No device work until admission. */
int ssx_server_submit(ssx_server *sv, const ssx_grid_desc *grid, const ssx_geom_desc *geom,
                      const float *v_dev, double rho, const double *d_dev, double alpha, int maxit,
                      double rtol, int mode, double *h_out_dev, int *id_out);
/* Admit what fits, run one round (four phases) of every admitted solve,
 * retire the finished ones. Synchronises. */
int ssx_server_step(ssx_server *sv, int *n_active, int *n_queued);
/* done = 1 once the request's h is in its output buffer; status, iterations,
 * submit-to-done latency and submit-to-admit wait in ms (host clock). */
int ssx_server_poll(ssx_server *sv, int id, int *done, int *status, int *iters, double *latency_ms,
                    double *queue_ms);
/* Working-set admission: besides the memory budget, requests are admitted
 * (first in, first out) only while the active requests' grids -- the fields
 * their sweeps step through -- fit in `bytes`, so that a batch stays close to
 * the L2 cache's size instead of growing into one long all-request round
 * that streams from HBM; a request that does not fit waits until it fits or
 * would run alone. The default is four times the device's L2 size; 0
 * switches the limit off (admission by the memory budget alone). */
int ssx_server_set_cache_budget(ssx_server *sv, size_t bytes);
/* Instrumentation of the server's shared launches: ssx_server_set_timing
 * brackets them with CUDA events (as ssx_set_timing does for a context);
 * ssx_server_get_stats returns their counters since creation (kernel
 * launches, point updates, event-timed phase time; synchronises when timing)
 * and, if not NULL, the engine rounds run and the requests in them summed
 * over the rounds. */
int ssx_server_set_timing(ssx_server *sv, int on);
int ssx_server_get_stats(ssx_server *sv, ssx_stats *out, long long *rounds, long long *request_rounds);
int ssx_server_destroy(ssx_server *sv);
const char *ssx_server_last_error(const ssx_server *sv);

/* d = pressure gather on z_r of a point pressure source w(t) delta(x - x_d)
 * delta(z - z_d) (fixture of the section "Creating downgoing fields").
 * wavelet_dev: nt float64 samples (device), sample n integrated over the
 * pressure update n -> n+1. x_d must fall on a grid column. */
int ssx_point_source_data(ssx_ctx *ctx, double x_d, double z_d,
                          const double *wavelet_dev, double *d_dev);

/* How a sweep (nt time steps of one grid) is launched:
 * SSX_SWEEP_AUTO (default): one cooperative launch for the whole sweep when
 *   every tile's CTA can be resident at once (each CTA steps its tile and
 *   waits, with a 2 s bound, only for its four edge neighbours); otherwise
 *   SSX_SWEEP_STEP.
 * SSX_SWEEP_STEP: one launch per time step, replayed from a CUDA graph.
 * SSX_SWEEP_PERSISTENT: cooperative launch or SSX_ERR_ARG if it cannot fit.
 * Both launch forms run the same per-tile arithmetic. A neighbour wait that
 * times out makes the call return SSX_ERR_CUDA ("timed out") instead of
 * hanging; the context stays usable.
 * SSX_SWEEP_TEST_STALL (test hook, not a mode): in the next persistent sweep
 *   one tile never signals its neighbours, whose waits then run out after
 *   0.2 s; or, if the next multi-sweep phase runs on the TMA-staged kernel,
 *   the copies of its first tile in its first step are never issued, so that
 *   CTA's mbarrier wait runs out after 0.2 s. Either way the timeout path is
 *   exercised without a fault, and the call returns SSX_ERR_CUDA.
 * After a wait that timed out for a real reason (not the test hook), treat
 * the context as unusable and destroy it: a CTA that gave up on tensor copies
 * which were merely slow waits once more (bounded) and then leaves, and copies
 * still in flight after that would land in shared memory the CTA no longer
 * owns, so the context's fields and captured graphs are no longer trusted.
 * The test hook withholds the copies entirely, which is why its context
 * stays usable. */
enum { SSX_SWEEP_AUTO = 0, SSX_SWEEP_STEP = 1, SSX_SWEEP_PERSISTENT = 2, SSX_SWEEP_TEST_STALL = 3 };
int ssx_set_sweep_mode(ssx_ctx *ctx, int mode);

/* Failure injection for tests, on the host-visible scalar path (no GPU
 * fault): in the next solve on this context (ssx_solve_source_subproblem, or
 * this context's shot in ssx_solve_batch / a server), the curvature
 * <p_k, q_k> of iteration k is overwritten on the device right after it is
 * formed, before alpha_k: with 0 (SSX_HOOK_BREAKDOWN), so Algorithm 1's
 * breakdown test fires and the solve returns SSX_ERR_BREAKDOWN; or with a NaN
 * (SSX_HOOK_NONFINITE), so it returns SSX_ERR_NONFINITE. Either way h_out then
 * holds h_k, the last good iterate, and k updates are reported. The hook
 * fires once. SSX_HOOK_NONE clears it. SSX_ERR_ARG for an unknown hook or
 * k < 0. */
enum { SSX_HOOK_NONE = 0, SSX_HOOK_BREAKDOWN = 1, SSX_HOOK_NONFINITE = 2 };
int ssx_set_test_hook(ssx_ctx *ctx, int hook, int k);

/* Tile configuration of the step kernels: -1 (default) lets the library time
 * every configuration on each grid's first sweep in each direction and keep
 * the fastest; 0..13 fixes one shape: 0..7 step by column strips (tile
 * 64x16/256 threads, 64x16/512, 32x32/256, 64x32/512, 64x32/1024, 128x16/512,
 * 128x32/1024, 32x16/256), 8..13 by quads, one thread per four consecutive
 * columns with 16-byte vector operands (64x16/256, 32x32/256, 64x32/512,
 * 128x16/512, 128x32/1024 with one row a thread; 64x16/128 with two; for
 * space order 8, other orders run them as strips); 14 + k fixes shape k with
 * the multi-sweep steps run by the TMA-staged kernel (operand tiles copied by
 * the tensor memory accelerator into a two-stage shared-memory pipeline,
 * persistent CTAs), available for space order 8; for other orders 14 + k
 * runs shape k; 28 + m fixes the marching kernel of shape m (tiles of
 * 64 x 128, 128 x 64, 128 x 128, 128 x 32 points, one thread per column
 * walking down it in blocks of 8 rows fed by tensor copies), available for
 * space order 8 (else shape 0 runs); 32 + m fixes, for the phases of a
 * single sweep, the two-step kernel of shape m (tiles of 32 x 16 with 256 or
 * 512 threads, 32 x 32 with 512: temporal blocking, two time steps per launch
 * with the intermediate step kept in shared memory), available for space
 * order 8 (other phases run shape 0). All configurations compute identical results. */
#define SSX_NUM_TILE_CONFIGS 14
#define SSX_NUM_MARCH_CONFIGS 4
#define SSX_NUM_TWO_CONFIGS 3
int ssx_set_tile_config(ssx_ctx *ctx, int cfg);

/* Timing mode: when on, every sweep is bracketed by CUDA events on the
 * launching stream; ssx_get_stats then reports their summed device time. */
int ssx_set_timing(ssx_ctx *ctx, int on);

/* Counters since creation or the last reset (synchronises when timing). */
int ssx_get_stats(ssx_ctx *ctx, ssx_stats *out);
int ssx_reset_stats(ssx_ctx *ctx);

/* Per-phase breakdown of the timed sweeps (timing mode), since creation or
 * the last reset. A phase is one set of sweeps stepped together, one launch a
 * time step (the solve's phases e1-e4 of Algorithm 1's operators); phases of
 * the same name, sweep count, tile count and kernel configuration share a
 * row. Row k (from 0, in order of first appearance): the phase's name
 * (NUL-terminated, truncated to name_len - 1 characters), its sweeps, the
 * tiles of its largest launch, its tile configuration (0-13 plain kernel,
 * 14-27 TMA-staged, 28-31 marching, 32-34 two steps per launch), its dependent-launch chain length (every
 * chain-th launch an ordinary launch; 0: one chain a span), its event-timed
 * device time and its time steps (launches). SSX_ERR_ARG for k past the
 * last row or a NULL output. Synchronises. */
int ssx_get_phase_stats(ssx_ctx *ctx, int k, char *name, int name_len, int *sweeps, int *tiles,
                        int *tile_cfg, int *chain, double *ms, long long *steps);

/* Capacity, in floats (16 MiB), of the fixed device scratch array used by
 * ssx_forward_noalloc. */
#define SSX_NOALLOC_MAX_FLOATS 4194304

/* d = S h, like ssx_forward, for callers that cannot allocate device memory.
 * The paper has no counterpart: this entry point exists for integration only.
 *
 * Some callers cannot call cudaMalloc: a plug-in inside a framework that owns
 * the device's whole memory pool, code running under a fixed memory budget,
 * or code that must not allocate (and risk an implicit synchronisation) in
 * the middle of its own work. Here the caller passes the grid and geometry
 * descriptors, the model v_dev [nz][nx] (float32, device), rho, the source
 * gather h_dev [nt][n_line] and the output d_dev [nt][n_rec] (float64,
 * device); no context is needed. All scratch (padded kappa field, two
 * ping-pong wavefield triples, sponge tables, the model maximum) lives in
 * one file-scope device array of SSX_NOALLOC_MAX_FLOATS floats. A GPU
 * reserves the array when the library's module is first used on it (with
 * CUDA's lazy module loading that can be inside this call's first use) and
 * holds it until the process exits. Nothing is allocated or freed.
 *
 * The grid must fit: 7 P Q + 2 (nx + nz + 4 n_sponge) + 64 <= SSX_NOALLOC_MAX_FLOATS
 * with P = roundup(roundup(nx + 2 n_sponge, 128) + 64, 32) and
 * Q = roundup(nz + 2 n_sponge, 32) + 16 (the 601 x 301 grid with a
 * 40-point sponge uses 2.33 M floats); larger grids (including descriptors
 * whose padded size overflows an int) return SSX_ERR_ARG before any device
 * work. Results are bit-identical to ssx_forward's on the same inputs. Other errors: SSX_ERR_ARG for invalid arguments,
 * SSX_ERR_CFL, SSX_ERR_CUDA; there is no message string.
 *
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture. The call enqueues its work on `stream` and
 * synchronises that stream once (a 4-byte read of the model maximum for the
 * CFL check). Every call shares the one array, which keeps the last call's
 * contents; each call clears what must start at zero. Calls whose work
 * overlaps on the GPU (other streams or threads) race on the array and must
 * be serialised by the caller. */
int ssx_forward_noalloc(const ssx_grid_desc *grid, const ssx_geom_desc *geom,
                        const float *v_dev, double rho, const double *h_dev,
                        double *d_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SSX_H */
