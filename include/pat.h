/*
 * pat.h - C ABI of the GB300 library for joint reconstruction of initial
 * pressure p0 and speed of sound c in 2-D photoacoustic tomography.
 *
 * The library computes, for K photoacoustic data sets that share one speed
 * of sound map:
 *   - the forward operator f^i : (p0^i, c) -> y^i of the observation model
 *     y = f(x) + e (Sec. 2.2, Eq. ObservationModel), a k-space
 *     pseudospectral solve of the acoustic initial value problem
 *     (Sec. 2.1, Eq. WaveEquation) with a PML and point sensors;
 *   - the data term of the objective (Eq. Minimised_functional) and its
 *     exact discrete adjoint gradient with respect to every p0^i and c
 *     (Sec. 3, Eqs. AdjointEquation, gradient_p0, gradient_sos);
 *   - the projected L-BFGS reconstruction with backtracking (Eq.
 *     BFGS_iterations, Algorithm 1, Eq. bound_constraints) over a
 *     coarse-to-fine multigrid schedule (Sec. 3.1).
 *
 * Discretisation (the paper names the k-space method but does not restate
 * it): first-order split-field staggered k-space leapfrog, wavenumbers
 * k = 2 pi/(Ng dx) {-Ng/2 .. Ng/2-1}, correction kappa = sinc(c_ref |k| dt/2),
 * staggering shifts exp(+-i k dx/2), PML alpha = pml_alpha (c_ref/dx)
 * (depth/P)^4 applied as exp(-alpha dt/2) twice per update, uniform density
 * rho0, p = c^2 (rho_x + rho_y), initial velocity u^{-1/2} = dt/(2 rho0) G p0.
 *
 * Conventions for every call:
 *   - Fields are row-major [y][x] (x fastest), float32.  p0 and c cover the
 *     N x N domain only; the PML (P cells per side) lies outside it and has
 *     c = c_bg there.  Traces are [K][nt][m] (time-major).
 *   - Pointers named d_* are DEVICE pointers owned by the caller; pointers
 *     named h_* are host pointers.  Nothing returned to the caller is
 *     allocated by the library; plans own their own small tables.
 *   - Calls are asynchronous on the given CUDA stream (passed as void*, a
 *     cudaStream_t; NULL = legacy default stream) unless stated.
 *   - Return value: PAT_OK (0) or a negative PAT_E* code; pat_last_error()
 *     gives a message for the calling thread.  Arguments are validated
 *     before anything is launched.
 *   - A plan is used by one host thread at a time (it holds its graph
 *     cache, its second stream and the record of which workspace keeps the
 *     last pressure history); distinct plans may run on distinct threads.
 *     Calls that share a workspace must be ordered on the GPU (issued on
 *     one stream, or the caller synchronises between streams): a workspace
 *     holds the running state of the time stepping.
 */
#ifndef PAT_H
#define PAT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PAT_OK 0
#define PAT_EINVAL (-1)       /* bad shape, size, range or pointer */
#define PAT_ENOMEM (-2)       /* workspace too small or allocation failed */
#define PAT_ECUDA (-3)        /* a CUDA call failed */
#define PAT_ENONFINITE (-4)   /* NaN/Inf met in the objective */
#define PAT_ETIMEOUT (-5)     /* a bounded device wait gave up */
#define PAT_ELINESEARCH (-6)  /* line search failed (reported, not fatal) */

/* Discretisation of one grid level (Sec. 2.1; Table 1 style parameters).
 * n: domain side N (cells), >= 2.  pml: PML width P (cells), >= 0; the FFT
 * grid side Ng = n + 2 pml must be even, 5-smooth (factors 2, 3, 5) and
 * <= 1024.  dx: cell size (m).  dt: time step (s).
 * nt: number of time samples t_n = n dt, n = 0..nt-1 (>= 1).  c_ref:
 * reference speed of kappa and of the PML (the upper bound of c).  rho0:
 * uniform density.  pml_alpha: PML strength (nepers per cell at the outer
 * edge; 0 disables absorption).  c_bg: speed of sound outside the domain. */
typedef struct {
    int n;
    int pml;
    double dx;
    double dt;
    int nt;
    double c_ref;
    double rho0;
    double pml_alpha;
    double c_bg;
} pat_grid;

typedef struct pat_plan_s* pat_plan;

/* Create a plan for K data sets with m point sensors (Sec. 4: point-like
 * sensors; sampled by bilinear interpolation at their physical positions).
 * h_sensor_xy: host [m][2] (x, y) in metres in the domain frame (origin at
 * the lower-left corner of the domain, cell (iy, ix) centred at
 * ((ix+0.5) dx, (iy+0.5) dx)); every sensor's 2x2 stencil must lie inside
 * the FFT grid.  ckpt_every: wavefield checkpoint interval s used by the
 * gradient (store the state every s steps, recompute in between); s >= nt
 * stores the whole pressure history instead.  Tables (wavenumbers, kappa,
 * PML, twiddles, sensor stencils) are computed in FP64 and stored in FP32
 * on the current device.  *out receives the plan; destroy it with
 * pat_plan_destroy (NULL is accepted). */
int pat_plan_create(pat_plan* out, const pat_grid* grid, int m, const double* h_sensor_xy,
                    int K, int ckpt_every);

/* A plan for ninst independent reconstructions that share one grid and one
 * sensor set (a batch: one launch per pass serves all of them).  Instance i
 * has h_K[i] >= 1 data sets; the K = sum h_K[i] data sets are numbered
 * instance by instance.  In every call of such a plan the speed of sound
 * d_c and its gradient d_grad_c are [ninst][N][N], J is [ninst], and p0,
 * traces, weights and dJ/dp0 are indexed by data set as usual.
 * pat_plan_create(..., K, ...) is the one-instance case. */
int pat_plan_create_batched(pat_plan* out, const pat_grid* grid, int m, const double* h_sensor_xy, int ninst,
                            const int* h_K, int ckpt_every);
void pat_plan_destroy(pat_plan plan);

/* Number of instances and of data sets (all instances) of a plan. */
int pat_plan_shape(pat_plan plan, int* ninst, int* K);

/* FFT grid side Ng and PML width of a plan (for callers that size buffers). */
int pat_plan_ng(pat_plan plan);

/* Kernel variants of a plan.  Grid sides with a compiled two-level FFT
 * (108, 144, 180, 200, 240, 300 = N1 x N2) have fixed-size variants (eight
 * for 108-240, eleven for 300), all one launch per pass:
 *   0  column and velocity passes on the N1 x N2 factorisation, density
 *      passes on N2 x N1 (4 rows / 4 spectral columns per CTA); the column
 *      passes of the forward sweep, which runs alone on the GPU, take 8
 *      columns per CTA;
 *   1  all passes N1 x N2, 4 rows / 4 columns per CTA;
 *   2  all passes N1 x N2, 8 rows / 2 columns per CTA;
 *   3  as 1 with the row passes' state staged in shared memory by TMA bulk
 *      copies instead of registers;
 *   4  all passes N2 x N1, 4 rows / 4 columns per CTA;
 *   5  as 0 with 8 rows per CTA in the row passes;
 *   6  as 0 with the segment recompute's row passes (which share the GPU
 *      with the adjoint) staged by TMA as in 3, so that they need fewer
 *      registers;
 *   7  (108-240) as 5 with column passes that form their multipliers where
 *      they use them (less shared memory: faster when a launch has many
 *      waves of CTAs);
 *   7, 8 (300) as 5 with the column passes on a three-level 5 x 10 x 6
 *      register FFT (60 threads per column), 4 / 8 and 2 / 4 columns per CTA;
 *   9  (300) as 5 with 4-column tiles in the forward sweep's column passes;
 *   10 (300) as 5 with the column passes of 7 (108-240).
 * Every side also has the generic shared-memory Stockham passes (variant
 * -1).  All variants compute the same scheme.  A new plan uses variant 0
 * when it exists, else -1.  pat_plan_variants returns the number of
 * fixed-size variants; pat_plan_set_variant selects one (PAT_EINVAL if it
 * does not exist); pat_plan_variant returns the current one. */
int pat_plan_variants(pat_plan plan);
int pat_plan_set_variant(pat_plan plan, int variant);
int pat_plan_variant(pat_plan plan);

/* Persistent forward sweep (grid sides 108, 144, 180, 200, 240, 300): with
 * enable != 0 every forward sweep of the plan (pat_forward, the forward part
 * of pat_adjoint_grad, the objective evaluations of the reconstruction) is
 * one launch instead of four per time step.  Its CTAs stay resident and take
 * work items (pass, data set, tile) of all data sets of all instances from a
 * counter in the workspace; an item waits only for its own data set's
 * earlier passes, so data sets and instances advance independently.  Each
 * wait is bounded: if one gives up (after 1 s) the status word gets
 * PAT_STATUS_QUEUE (pat_status) and the results of that call are invalid.
 * Same results as the launched passes.  PAT_EINVAL for other grid sides.
 * pat_plan_persistent returns 1 if enabled, 0 if not, -1 for a NULL plan. */
int pat_plan_set_persistent(pat_plan plan, int enable);
int pat_plan_persistent(pat_plan plan);

/* Cluster-resident stepping (Sec. 2.1 scheme; grid side 300): with enable != 0
 * every forward sweep of the plan and every segment recompute of the reverse
 * sweep runs as one launch of one thread-block cluster of 16 CTAs per data
 * set, which keeps the data set's wavefield in registers and shared memory
 * for all its time steps and exchanges row and column spectra through
 * distributed shared memory (four cluster barriers per step).  Same scheme
 * and results as the launched passes to FP32 rounding; traces, checkpoints,
 * pressure history and the final state are written as by the launched
 * sweep.  Clusters that do not fit on the GPU at once run after the others.
 * PAT_EINVAL for other grid sides; PAT_ECUDA if the GPU cannot run a
 * 16-CTA cluster of this size.  pat_plan_cluster returns 1 if enabled, 0 if
 * not, -1 for a NULL plan; pat_plan_cluster_capacity the number of such
 * clusters (data sets) the current GPU runs at once (0 if none or no
 * cluster-resident stepping for the plan's grid side; PAT_EINVAL for a NULL
 * plan).  The launched passes are faster on GB300 at every K measured (the
 * cluster form is an option, off by default).  With the persistent sweep also
 * enabled, forward sweeps use the persistent sweep and segment recomputes the
 * cluster form. */
int pat_plan_set_cluster(pat_plan plan, int enable);
int pat_plan_cluster(pat_plan plan);
int pat_plan_cluster_capacity(pat_plan plan);

/* CUDA graphs: with enable != 0, the first pat_forward / pat_adjoint_grad
 * (or objective evaluation of pat_reconstruct) on a non-default stream with
 * a given set of buffers and kernel variant is captured into a CUDA graph and
 * every later call with the same buffers replays it (one launch for the
 * whole call).  Buffers are keyed by address: a caller that reuses
 * addresses for new data gets the new data.  A plan keeps at most 16
 * graphs; capturing another one first frees the least recently replayed.
 * enable = 0 frees the graphs. */
int pat_plan_set_graphs(pat_plan plan, int enable);

/* Autotuner: times every variant of the plan (generic and fixed-size) on
 * this GPU and keeps the fastest (median of three timings per variant).
 * With a gradient workspace (ws_bytes >=
 * PAT_WS_GRADIENT size) it times one whole gradient evaluation per variant
 * (forward sweep with checkpoints, reverse sweep with the recompute stream;
 * c = c_ref, p0 = 0, zero residual), otherwise 32 forward steps on a forward
 * workspace (d_ws NULL: a temporary one is allocated and freed on the
 * stream).  The workspace contents are overwritten.  h_ms: host array of
 * pat_plan_variants(plan)+1 entries (may be NULL) receiving, for variants
 * -1, 0, ..., the ms per gradient evaluation or per forward step.
 * Synchronises the stream; with no fixed-size variant it selects -1. */
int pat_plan_autotune(pat_plan plan, void* d_ws, size_t ws_bytes, double* h_ms, void* stream);

/* Smallest PML width >= min_pml for which n + 2 P satisfies the grid rules
 * above (Sec. 4.1.1: PML sized so the grid has small prime factors);
 * returns -1 if none <= 1024 exists. */
int pat_pml_auto(int n, int min_pml);

/* Workspace sizes in bytes (caller allocates, 256-byte aligned device
 * memory).  PAT_WS_FORWARD suffices for pat_forward; PAT_WS_GRADIENT holds
 * the checkpoints and the adjoint state as well. */
#define PAT_WS_FORWARD 0
#define PAT_WS_GRADIENT 1
size_t pat_workspace_bytes(pat_plan plan, int kind);

/* Forward operator (Eq. ObservationModel without noise): d_y[k][n][m] =
 * S p_k^n for the K initial pressures d_p0 [K][N][N] and the speed of sound
 * d_c [N][N].  d_y [K][nt][m] is overwritten.  If ws_bytes >=
 * pat_workspace_bytes(plan, PAT_WS_GRADIENT) the checkpoints needed by a
 * following pat_vjp with the same c and p0 are kept in d_ws. */
int pat_forward(pat_plan plan, const float* d_c, const float* d_p0, float* d_y,
                void* d_ws, size_t ws_bytes, void* stream);

/* Forward operator without any allocation, for callers that cannot
 * allocate device memory at the time they run the model (for example an
 * acquisition process whose device memory budget is fixed at start-up, or a
 * host program whose device memory is owned by another allocator; cudaMalloc
 * can also synchronise the device, which a latency-critical loop cannot
 * afford).  The paper has no counterpart: this is a deployment variant of
 * pat_forward.  Same arguments and results as pat_forward without the
 * workspace: the scratch is a static device array of
 * PAT_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library
 * holds until exit.  Plans whose forward workspace
 * (pat_workspace_bytes(plan, PAT_WS_FORWARD)) exceeds it are rejected with
 * PAT_EINVAL and a message.  The plan's device must be current.  The array's
 * device address is looked up in the current context on every call (after a
 * cudaDeviceReset it may move); the first call in a context loads the
 * library's device code (set-up), so make it before any stream capture.  All
 * calls share the array and it keeps the last call's contents; calls that
 * overlap on the GPU (other streams, other threads, other plans) race on it.
 * No checkpoints are kept, so it cannot precede pat_vjp. */
#define PAT_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
int pat_forward_noalloc(pat_plan plan, const float* d_c, const float* d_p0, float* d_y, void* stream);

/* Status of the last pat_forward_noalloc with this plan, read from the
 * static array after synchronising the stream: *h_flag gets PAT_STATUS_WAIT
 * if a staged row pass (variant 3) gave up its bounded wait, and (debug
 * build) PAT_STATUS_BOUNDS if a bounds check failed, so that the traces of
 * that call are invalid; 0 otherwise.  The array is shared, so
 * the answer concerns the last allocation-free call of any plan. */
int pat_forward_noalloc_status(pat_plan plan, int* h_flag, void* stream);

/* Data term and its gradient (Eq. Minimised_functional without priors;
 * Eqs. gradient_p0 and gradient_sos for the discrete scheme):
 *   J = sum_k w_k/2 || y_pred_k - y_meas_k ||^2,
 *   d_grad_p0 [K][N][N] = dJ/dp0_k,  d_grad_c [N][N] = dJ/dc summed over k.
 * d_w: device [K] float weights w_k = 1/sigma_k^2 (L_e^T L_e = w_k I).
 * d_J: device double[ninst] (may be NULL) receives J per instance.  d_y_pred: device
 * [K][nt][m] (may be NULL) receives the predicted traces.  The workspace
 * must hold PAT_WS_GRADIENT bytes.  A NaN or Inf in J is reported by
 * pat_status (PAT_STATUS_NONFINITE), not by the return value: the call
 * stays asynchronous. */
int pat_adjoint_grad(pat_plan plan, const float* d_c, const float* d_p0, const float* d_y_meas,
                     const float* d_w, float* d_grad_p0, float* d_grad_c, double* d_J,
                     float* d_y_pred, void* d_ws, size_t ws_bytes, void* stream);

/* Vector-Jacobian product of the forward operator: given d_ybar [K][nt][m]
 * (the adjoint source, e.g. dL/dy), returns d_grad_p0 = (df/dp0)^T ybar and
 * d_grad_c = sum_k (df_k/dc)^T ybar_k.  Requires that d_ws holds the
 * checkpoints of a pat_forward with the same d_c and d_p0 and a
 * PAT_WS_GRADIENT workspace; calls in between that use other workspaces are
 * allowed (the last segment's pressure history is then recomputed). */
int pat_vjp(pat_plan plan, const float* d_c, const float* d_p0, const float* d_ybar,
            float* d_grad_p0, float* d_grad_c, void* d_ws, size_t ws_bytes, void* stream);

/* Status of the last calls on this workspace, after synchronising the
 * stream: *h_flag bit 0 (PAT_STATUS_NONFINITE) if the last objective met a
 * NaN/Inf in J or a residual; bit 1 (PAT_STATUS_WAIT) if a kernel of the last
 * pat_forward / pat_adjoint_grad / pat_vjp gave up a bounded wait for its
 * staged copies (variant 3); bit 2 (PAT_STATUS_QUEUE) if a persistent sweep
 * gave up waiting for a work item (the results of that call are then
 * invalid in both cases). */
#define PAT_STATUS_NONFINITE 1
#define PAT_STATUS_WAIT 2
#define PAT_STATUS_QUEUE 4
/* Bit 4 (PAT_STATUS_BOUNDS), debug build only (pat_debug_bounds() == 1): a
 * device-side bounds check of the last forward / gradient / vjp failed on an
 * index taken from run-time data (a sensor stencil entry, the time step, the
 * history slot); the access was skipped or redirected to an index in range,
 * so the results of that call are invalid. */
#define PAT_STATUS_BOUNDS 16

/* 1 if this library was built with the device-side bounds checks
 * (-DPAT_DEBUG_BOUNDS: libpat_debug.so), 0 for the release build, whose
 * checks compile to nothing.  Not from the paper: a debugging aid. */
int pat_debug_bounds(void);

/* Self-test of the bounds check behind PAT_STATUS_BOUNDS: one CTA checks an
 * index one past the end of a shared-memory array (which has one spare
 * element, so the guarded store stays in bounds whichever build runs it).
 * The debug build ORs PAT_STATUS_BOUNDS into the device int *d_status and
 * skips the store; the release build leaves *d_status unchanged.  PAT_EINVAL
 * for a NULL pointer. */
int pat_selftest_bounds(int* d_status, void* stream);

/* Self-test of the bounded wait behind PAT_STATUS_WAIT: launches one CTA on
 * the stream whose threads wait for an mbarrier phase that never completes
 * (nothing arrives, no copy is in flight), give up after timeout_us
 * microseconds (1..1000000) and OR PAT_STATUS_WAIT into the device int
 * *d_status.  No fault and no hang: the context stays usable.  PAT_EINVAL
 * for a NULL pointer or a timeout out of range. */
int pat_selftest_wait(int* d_status, unsigned timeout_us, void* stream);

/* Self-test of the bounded dependency wait behind PAT_STATUS_QUEUE: zeroes
 * the device int[3] d_queue (ticket counter, abort flag, items done of one
 * data set), then launches one CTA that waits for an item of that data set
 * which nothing produces, gives up after timeout_us microseconds
 * (1..1000000), ORs PAT_STATUS_QUEUE into *d_status and sets the abort flag
 * d_queue[1].  No fault and no hang.  PAT_EINVAL for a NULL pointer or a
 * timeout out of range. */
int pat_selftest_queue(int* d_queue, int* d_status, unsigned timeout_us, void* stream);
int pat_status(pat_plan plan, const void* d_ws, int* h_flag, void* stream);

/* ---- Ornstein-Uhlenbeck prior (Eq. Minimised_functional, Sec. 4.1.2) ---- */

/* The regularising terms of the objective: for a field z on an n x n pixel
 * grid of spacing dx (m), P(z) = 1/2 (z - eta)^T Xi^{-1} (z - eta) / sigma^2
 * with the unit covariance Xi_ij = exp(-|r_i - r_j| / tau), r_i the pixel
 * centres, tau the characteristic length (m); dP/dz = Xi^{-1}(z - eta)/sigma^2.
 * Xi v is computed exactly as a linear convolution through a zero-padded FFT
 * of side M >= 2n - 1; Xi^{-1} b by preconditioned conjugate gradients (the
 * padded circulant's inverse as preconditioner), batched over fields, FP32
 * vectors with FP64 dot products.  Fields are device arrays [nf][n][n]
 * float, nf <= max_fields.  All calls run on `stream`; pat_prior_solve and
 * pat_prior_eval synchronise it (convergence checks).  A prior object owns
 * its device buffers (about 5 max_fields n^2 floats plus the transforms);
 * calls on one object must not overlap. */
typedef struct pat_prior_s* pat_prior;

/* Create for the current device: 2 <= n <= 512, dx > 0, tau > 0,
 * 1 <= max_fields <= 1024 (PAT_EINVAL otherwise).  Builds the spectrum of
 * the embedding on the host in FP64 (O(M^3), about 0.3 s at n = 256). */
int pat_prior_create(int n, double dx, double tau, int max_fields, pat_prior* out);
int pat_prior_destroy(pat_prior prior);

/* d_out = Xi d_v for nf fields. */
int pat_prior_xi(pat_prior prior, const float* d_v, float* d_out, int nf, void* stream);

/* Solve Xi d_z = d_b for nf fields to a relative residual |r| <= tol |b|
 * per field, at most maxit iterations; warm != 0 starts from d_z's contents,
 * else from zero.  *h_iters (may be NULL) receives the iterations taken. */
int pat_prior_solve(pat_prior prior, const float* d_b, float* d_z, int nf, double tol, int maxit, int warm,
                    int* h_iters, void* stream);

/* Prior terms of nf fields d_x with means h_eta[nf] and standard deviations
 * h_sigma[nf] (host arrays): d_z [nf][n][n] receives Xi^{-1}(x - eta) (warm:
 * start from its contents); *d_J (device double, may be NULL) is increased by
 * sum_f P(x_f); d_grad (may be NULL) is increased by gscale_f dP/dx_f
 * (h_gscale may be NULL: 1).  tol, maxit, warm, h_iters as in
 * pat_prior_solve. */
int pat_prior_eval(pat_prior prior, const float* d_x, int nf, const double* h_eta, const double* h_sigma,
                   const double* h_gscale, float* d_z, float* d_grad, double* d_J, double tol, int maxit,
                   int warm, int* h_iters, void* stream);

/* ---- reconstruction (Sec. 3, Sec. 3.1) ---- */

/* Configuration of pat_reconstruct.  levels[nlevels]: domain sides N_l,
 * coarse to fine, all covering the same physical side L (m), dx_l = L/N_l,
 * dt_l = cfl dx_l / c_hi, nt_l = round(T/dt_l) + 1 with T = (nt_data-1)
 * dt_data; PML >= min_pml cells per side.  Bounds: p0 >= p0_lo (no upper
 * bound), c in [c_lo, c_hi] (Eq. bound_constraints); c_hi is also c_ref.
 * mem: L-BFGS memory l (0 = projected Barzilai-Borwein gradient).  iters:
 * iterations per level; a level also stops when the relative decrease of J
 * is below rtol.  alpha0: first step in block-scaled units; c1: Armijo
 * constant; max_halvings: backtracking halvings per line search; sigma_p0:
 * block scale of p0 (c uses (c_hi - c_lo)/4).  ckpt_every: checkpoint
 * interval of the gradient solves. */
typedef struct {
    int nlevels;
    const int* levels;
    double L;
    double dt_data;
    int nt_data;
    int m;
    const double* h_sensor_xy;
    int K;
    double cfl;
    double c_lo, c_hi;
    double p0_lo;
    double c_bg;
    double rho0;
    double pml_alpha;
    int min_pml;
    int mem;
    int iters;
    int max_halvings;
    int ckpt_every;
    double rtol;
    double alpha0;
    double c1;
    double sigma_p0;
    int autotune;   /* nonzero: run pat_plan_autotune on every level's plan (forward-step timing) */
    /* Ornstein-Uhlenbeck prior terms of Eq. Minimised_functional (Sec. 4.1.2):
     * prior_tau > 0 (m) adds, on every level's grid, 1/2 |L_c (c - eta_c)|^2
     * and 1/2 |L_p0 (p0_k - eta_p0)|^2 for every k to J (see pat_prior_eval;
     * prior means and standard deviations below, sigmas > 0); 0: data term only. */
    double prior_tau;
    double prior_eta_c, prior_sigma_c;
    double prior_eta_p0, prior_sigma_p0;
    int persistent;  /* nonzero: forward sweeps of every level whose grid side has one run as one
                        persistent launch (pat_plan_set_persistent); other sides keep the passes */
} pat_recon_cfg;

/* One row per L-BFGS iteration. */
typedef struct {
    int level;
    int iter;
    double J;       /* objective before the step */
    double gnorm;   /* ||g|| in block-scaled variables before the step */
    double alpha;   /* accepted step (0 if the line search failed) */
    int trials;     /* objective evaluations in the line search */
    double J_new;   /* objective after the step */
    double ms;      /* wall time of the iteration */
    double Ec;      /* E_c (%, Eq. RelativeError) after the step against the instance's
                       true c resampled to the level, or -1 without a true c */
    double Ep0;     /* E_p0 (%, Eq. RelativeError over all K data sets stacked) after the
                       step against the true p0 resampled to the level, or -1 without one */
} pat_iter_report;

typedef struct {
    int capacity;              /* rows available in iters (caller-owned host array) */
    int count;                 /* rows written */
    pat_iter_report* iters;
    int status;                /* PAT_OK or PAT_ELINESEARCH if a level stopped on a failed search */
    double total_ms;
} pat_report;

/* Joint reconstruction of p0_1..K and c (Sec. 3, 3.1).  d_y_meas: device
 * [K][nt_data][m] data at t = n dt_data; d_w: device [K] weights.  d_c_io:
 * device [N][N] on the finest level (N = levels[nlevels-1]); on input the
 * initial guess (resampled bilinearly to the coarsest level), on output the
 * reconstruction.  d_p0_io: device [K][N][N], same semantics.  The call
 * synchronises the stream once per objective evaluation to read J (FP64
 * line-search decisions on the host) and allocates its level buffers with
 * stream-ordered allocation, freed before it returns. */
int pat_reconstruct(const pat_recon_cfg* cfg, const float* d_y_meas, const float* d_w,
                    float* d_c_io, float* d_p0_io, pat_report* report, void* stream);

/* The two transfers of the multigrid schedule, as pat_reconstruct applies
 * them between levels (Sec. 3.1: the parameters of a converged level are
 * interpolated to the next finer grid; Sec. 4.1.2: the data are interpolated
 * linearly to each level's time grid).
 * pat_prolong: bilinear resampling of nb fields d_src [nb][n_src][n_src] to
 * d_dst [nb][n_dst][n_dst] on the cell-centred coordinates of the same
 * physical square, constant beyond the outermost source cell centres.
 * pat_time_interp: d_out [K][nt_dst][m] = linear interpolation in time of
 * d_y [K][nt_src][m] (samples at n dt_src) at t = n dt_dst, held at the last
 * sample beyond it.  Device buffers, asynchronous on the stream; PAT_EINVAL
 * for a NULL buffer, a size < 1 or a time step that is not positive. */
int pat_prolong(const float* d_src, float* d_dst, int nb, int n_src, int n_dst, void* stream);
int pat_time_interp(const float* d_y, float* d_out, int K, int nt_src, int nt_dst, int m, double dt_src,
                    double dt_dst, void* stream);

/* ---- instrumentation (benchmarking; not thread-safe) ---- */

/* Kernel classes that can be timed. */
#define PAT_K_ROW_RHO 1       /* forward density / pressure row pass (incl. sensor gather) */
#define PAT_K_ROW_U 2         /* forward velocity row pass */
#define PAT_K_COL_GRAD 3      /* column pass, one spectrum in, two out (forward G) */
#define PAT_K_COL_PAIR 4      /* column pass, two in, two out (forward D, adjoint G) */
#define PAT_K_COL_SUM 5       /* column pass, two in, one out (adjoint D) */
#define PAT_K_ROW_ADJ_RHO 6   /* adjoint density row pass (incl. scatter, dJ/dc) */
#define PAT_K_ROW_ADJ_U 7     /* adjoint velocity row pass */
#define PAT_K_LAST 7

/* Total number of kernels this library has launched in the process. */
unsigned long long pat_kernel_launches(void);

/* Record a pair of CUDA events on the launching stream around every
 * every-th launch of kernel class cls (at most max_launches pairs; cls 0
 * disables).  Events are created here, outside any timed region.  Sampling
 * keeps the perturbation of the timed work small: an event between two
 * kernels removes their programmatic launch overlap. */
int pat_timing_enable(int cls, int max_launches, int every);

/* Sum of the recorded launch durations (ms) and their count; waits for the
 * last recorded event and resets the counter. */
int pat_timing_read(double* total_ms, long long* launches);

/* One instance of a batched reconstruction: its data d_y_meas
 * [K][nt_data][m], weights d_w [K], finest-level c (in: initial guess, out:
 * result) d_c_io [N][N] and p0 d_p0_io [K][N][N] (same semantics), and an
 * optional report. */
typedef struct {
    const float* d_y_meas;
    const float* d_w;
    float* d_c_io;
    float* d_p0_io;
    int K;
    pat_report* report;
    const float* d_c_true;   /* optional [N][N]: report E_c per iteration */
    double ec_target;        /* > 0 with d_c_true: target of E_c */
    const float* d_p0_true;  /* optional [K][N][N]: report E_p0 per iteration */
    double ep0_target;       /* > 0 with d_p0_true: target of E_p0 */
    /* an instance with targets leaves a level (the finest: stops) once it meets all of them */
} pat_instance;

/* Several independent reconstructions that share cfg (levels, domain,
 * sensors, time grid, bounds, optimiser settings; cfg->K is ignored), solved
 * together: every objective or gradient evaluation is one batched solve over
 * all instances (a plan from pat_plan_create_batched per level), each
 * instance keeps its own L-BFGS state and FP64 line search, and the
 * instances advance in lockstep (an instance that has converged or failed
 * keeps its point).  Results are those of pat_reconstruct on each instance
 * alone.  Synchronises the stream once per evaluation round. */
int pat_reconstruct_batched(const pat_recon_cfg* cfg, int ninst, const pat_instance* inst, void* stream);

/* ---- learned warm start (an extension: the paper has no network) ----
 * A U-Net mapping K back-projected images (adjoint solves at a constant
 * speed of sound, i.e. pat_vjp with c = c0) to an initial speed-of-sound map
 * for pat_reconstruct; the iterative solve still decides the result.
 * Encoder level l (0..levels-1): two 3x3 convolutions + ReLU with base*2^l
 * channels and 2x2 max pooling between levels; decoder: nearest 2x
 * upsampling, concatenation [upsampled, encoder] and two 3x3 convolutions +
 * ReLU; a final 1x1 convolution to one channel.  BF16 activations and
 * weights on the tensor cores, FP32 accumulation, FP32 master parameters
 * and Adam.  The model owns its buffers (allocated at creation for
 * max_batch images). */
typedef struct pat_unet_s* pat_unet;
int pat_unet_create(pat_unet* out, int levels, int base, int in_ch, int H, int W, int max_batch);
void pat_unet_destroy(pat_unet net);
/* Number of FP32 parameters.  Layout: for every convolution in forward order
 * (encoder a/b per level, decoder a/b per level from the deepest, final),
 * weights [cout][k*k][cin] then bias [cout]; cin of the first convolution is
 * in_ch rounded up to 8 (weights of the padding channels must be 0). */
size_t pat_unet_param_count(pat_unet net);
/* h_desc: host int[6 * n_convs] (may be NULL): cin, cout, k, weight offset,
 * bias offset, spatial side of each convolution. */
int pat_unet_param_layout(pat_unet net, int* n_convs, int* h_desc);
/* Device FP32 parameters in / out (set also resets the Adam moments). */
int pat_unet_set_params(pat_unet net, const float* d_params, void* stream);
int pat_unet_get_params(pat_unet net, float* d_params, void* stream);
/* d_in: device [B][in_ch][H][W] FP32; d_out: device [B][H][W] FP32. */
int pat_unet_forward(pat_unet net, const float* d_in, int B, float* d_out, void* stream);
/* MSE loss mean((out - target)^2) (device double, may be NULL) and the FP32
 * parameter gradients (device, parameter layout; may be NULL). */
int pat_unet_grads(pat_unet net, const float* d_in, const float* d_target, int B, float* d_grad, double* d_loss,
                   void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr. */
int pat_unet_train_step(pat_unet net, const float* d_in, const float* d_target, int B, float lr, double* d_loss,
                        void* stream);

/* Tensor-core path of the network's GEMMs: 0 the warp-level BF16 MMA
 * (mma.sync m16n8k16, operands staged by cp.async); 1 (default) the
 * fifth-generation tensor cores: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in
 * tensor memory) on 128 x 128 tiles whose 128 x 64 operand blocks are copied
 * by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a 4-stage ring of
 * shared memory; GEMMs whose operands the TMA cannot address (K < 64,
 * pitches not multiples of 8, unaligned bases) keep the warp-level path.
 * Every wait of the tcgen05 kernel is bounded: if one gives up, the network's
 * status word gets PAT_STATUS_TC05 (pat_unet_status; the results of that
 * call are invalid). */
#define PAT_STATUS_TC05 8
int pat_unet_set_gemm_path(pat_unet net, int path);
int pat_unet_status(pat_unet net, int* h_flag, void* stream);

/* The network's BF16 GEMM on its own, for tests and measurement:
 * d_C[M][N] (FP32, row pitch ldc) = d_A[M][K] . d_B[N][K]^T with BF16
 * operands in row-major storage (row pitches lda, ldb in elements), FP32
 * accumulation.  path 0: warp-level MMA (K, lda, ldb multiples of 8);
 * path 1: tcgen05 (K >= 64, lda and ldb multiples of 8, 16-byte aligned
 * operands; PAT_EINVAL otherwise).  d_status (device int, may be NULL) gets
 * PAT_STATUS_TC05 if a bounded wait of the tcgen05 kernel gave up.
 * Asynchronous on the stream. */
int pat_gemm_bf16(const void* d_A, int lda, const void* d_B, int ldb, int M, int N, int K, float* d_C, int ldc,
                  int path, int* d_status, void* stream);

/* Message describing the last error on the calling thread. */
const char* pat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PAT_H */
