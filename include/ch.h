/*
 * ch.h -- C ABI of the GB300 (sm_103a) library for the explicit Cahn-Hilliard time
 * integrators of M.A. Botchev, "Explicit adaptive time stepping for the Cahn-Hilliard
 * equation by exponential Krylov subspace and Chebyshev polynomial methods",
 * arXiv:2502.14589.
 *
 * Problem (Sec. 2, Eq. IVP): y'(t) = -A (F'(y) + eps^2 A y), F'(y) = y^3 - y, where -A is the
 * second-order finite-difference Laplacian on a periodic grid of the unit square (dim = 2)
 * or cube (dim = 3), h_a = 1/n_a, points stored x fastest: index = i0 + n0 (i1 + n1 i2).
 * Linearisation at y^n (Sec. 3.1, Eqs. J, A_g):
 *   J_n = 3 diag((y^n)^2) - I,   A_hat_n = A (J_n + eps^2 A),   g_hat^n = A (J_n y^n - F'(y^n));
 * with the Eyre splitting (Sec. 3.2, Eq. A_g_cs) A_hat_n gains + A and g_hat^n gains + A y^n.
 *
 * Conventions for every call below:
 *  - Vector arguments are CALLER-OWNED DEVICE pointers to N = n0 n1 n2 contiguous doubles
 *    (FP64 at the boundary in every precision mode), 8-byte aligned.  The library keeps
 *    no reference to them after the call returns.
 *  - The grid owns all workspace (Krylov basis, Hessenberg matrix, scratch vectors),
 *    allocated once by ch_create_grid; no call allocates device memory afterwards.
 *  - Work is queued on the grid's CUDA stream.  Calls that return host scalars
 *    (norms, tau_used, est, p_used, lambda_max, stats) synchronise that stream before
 *    returning; ch_rhs / ch_jacvec with NULL scalar outputs are asynchronous.
 *  - Errors are returned as ch_status codes; no C++ exception crosses the ABI.  The
 *    message of the last error on the calling thread is available from ch_last_error().
 *    Device-side failures (non-finite values, Krylov non-convergence, bounded-wait
 *    timeouts) are written to a device status word and returned by the next call that
 *    synchronises.
 *  - A grid may be used by one host thread at a time.
 */
#ifndef CH_H_
#define CH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CH_OK = 0,
    CH_EINVAL = 1,        /* invalid argument (sizes, pointers, parameters) */
    CH_ENOMEM = 2,        /* device or pinned-host allocation failed at create time */
    CH_ECUDA = 3,         /* a CUDA runtime call failed */
    CH_ENOTCONV = 4,      /* Krylov run found no admissible step, or step/restart cap hit */
    CH_ENONFINITE = 5,    /* a NaN or Inf appeared in a reduction or in the solution */
    CH_ETIMEOUT = 6       /* a bounded device-side wait gave up */
} ch_status;

typedef enum {
    CH_FP64 = 0,          /* every vector, stencil and reduction in FP64 */
    CH_MIXED = 1          /* FP32 stencil arithmetic and Krylov basis; FP64 solution,
                             inner products, norms, Hessenberg matrix, projected phi,
                             Chebyshev coefficients and step control */
} ch_precision;

typedef enum { CH_EE2 = 0, CH_LIM = 1 } ch_scheme;

typedef struct ch_grid ch_grid;       /* opaque */

/* Parameters of a time integration; the "Given" boxes of Fig. 3 (LIM) and Fig. 4 (EE2). */
typedef struct {
    int scheme;           /* CH_EE2 or CH_LIM */
    int adaptive;         /* 1: adaptive tau (Figs. 3, 4); 0: constant tau = tau0 */
    double T;             /* final time */
    double tau0;          /* initial (adaptive) or constant step size */
    double tol;           /* accuracy tolerance of Eqs. (LIMdt), (EEdt), (tol_phi) */
    int mmax;             /* Krylov dimension m_max (EE2), 1 <= mmax <= capacity */
    double tol_phi;       /* > 0: fixed Krylov tolerance; <= 0: Eq. (tol_phi) */
    int eyre;             /* 1: Eyre-splitting A_hat, g_hat of Eq. (A_g_cs) */
    int64_t max_steps;    /* cap on accepted steps (CH_ENOTCONV when reached before T) */
} ch_params;

/* Work counters; "matvecs" counts products with A_hat_n as the paper does (Sec. 5.1):
 * LIM 2p-1 per step, EE2 one per Arnoldi iteration plus one per Krylov start vector. */
typedef struct {
    int64_t steps, matvecs, rhs_evals, krylov_iters, restarts, tau_shrinks, phi_evals;
    double t;             /* time reached */
    double tau_next;      /* step size the controller proposes next */
    double last_est;      /* est of the last step (Eq. LIMest) */
} ch_stats;

/* Create a periodic grid on the unit square (dim 2) or cube (dim 3) with n[a] >= 4 points
 * per axis (n[2] ignored when dim == 2), parameter eps > 0 of Eq. (IVP), precision mode,
 * and Krylov basis capacity mmax_capacity (1..128; the basis holds mmax_capacity + 1
 * vectors).  `cuda_stream` is a cudaStream_t (NULL = legacy default stream) on which all
 * work of this grid is queued.  Allocates all workspace.  *out receives the handle.     */
ch_status ch_create_grid(int dim, const int64_t n[3], double eps, int precision,
                         int mmax_capacity, void *cuda_stream, ch_grid **out);

/* Boundary conditions of a grid.  CH_BC_NEUMANN: the homogeneous Neumann conditions of
 * Eq. (CH) on cell-centred nodes (Sec. 5.1, x_i = (i - 1/2) h_a), where the neighbour beyond
 * a boundary face is the mirror image of the point inside, i.e. the point itself, so every
 * difference across the boundary vanishes. */
typedef enum { CH_BC_PERIODIC = 0, CH_BC_NEUMANN = 1 } ch_bc;

typedef struct {
    int bc;                 /* CH_BC_PERIODIC (default) or CH_BC_NEUMANN */
    int variable_mobility;  /* 1: reserve the workspace of ch_set_mobility at creation */
} ch_grid_options;

/* ch_create_grid with options (NULL = periodic, unit mobility).  Same domain, spacing,
 * precision modes and errors as ch_create_grid; CH_EINVAL for an unknown bc.            */
ch_status ch_create_grid_ex(int dim, const int64_t n[3], double eps, int precision,
                            int mmax_capacity, const ch_grid_options *opts, void *cuda_stream,
                            ch_grid **out);
ch_status ch_destroy_grid(ch_grid *g);

/* The Remark on Eq. (CHmob): a variable mobility M(c) replaces the outer operator A by
 * A_M(y^n), the flux form of -div(M grad .) frozen over a step:
 *   (A_M t)_i = sum_a (1/h_a^2) sum_{+-} (M_i + M_{i+-e_a})/2 (t_i - t_{i+-e_a}),
 * so A_hat = A_M (J + eps^2 A [+ I]), g_hat = A_M (J y - F'(y) [+ y]) and f = -A_M (F'(y) +
 * eps^2 A y); the inner eps^2 A and the energy keep the constant-mobility Laplacian.  M is a
 * caller-owned device array of N nodal values M_i >= 0 (for instance M(y^n_i) = 1 - (y^n_i)^2),
 * read on the grid's stream before the call returns control of it; the face values are kept
 * in the grid's workspace and used by every later call on the grid (rhs, jacvec,
 * lambda_max, estimate, Krylov runs, EE2 / LIM steps, integrate) until the next
 * ch_set_mobility.  To freeze the mobility at each step, call it before each step.  M = NULL
 * restores unit mobility.  CH_EINVAL when the grid was not created with variable_mobility. */
ch_status ch_set_mobility(ch_grid *g, const double *M);

/* Sec. 2, Eq. (IVP): f = -A (F'(y) + eps^2 A y).  Optional host outputs: norm_f = ||f||_2
 * and norm_ghat = ||g_hat(y)||_2 with g_hat of Eq. (A_g) (or Eq. A_g_cs when `eyre`).     */
ch_status ch_rhs(ch_grid *g, const double *y, double *f, int eyre, double *norm_f,
                 double *norm_ghat);

/* Eq. (A_g) / (A_g_cs): w = A_hat(y_lin) v = A (J + eps^2 A [+ I]) v.  Asynchronous.      */
ch_status ch_jacvec(ch_grid *g, const double *y_lin, const double *v, double *w, int eyre);

/* Fig. 1, spectral bound: lambda_max = ||A_hat(y)||_1 (host output, synchronises).  Closed
 * form from the extremes of y^2 on periodic constant-mobility grids, else the maximum of
 * the explicitly formed column sums (Neumann boundaries, variable mobility).             */
ch_status ch_lambda_max(ch_grid *g, const double *y, int eyre, double *lambda_max);

/* Host-only (no GPU needed).  The spectral bound of Fig. 1 in the closed form the GPU path
 * evaluates:
 * every column of A_hat has an absolute sum g(d_j), d_j = 3 y_j^2 - 1 (+1 with Eyre), and g
 * is convex, so ||A_hat||_1 = max(g(d_min), g(d_max)) from the extreme values y2min, y2max
 * of y^2.  Periodic grid of dim 2/3 with n[a] in [4, 2^20] points per axis (n[2] ignored
 * for dim 2), eps > 0.  CH_EINVAL for invalid arguments or y2min > y2max.               */
ch_status ch_lambda_max_bound(int dim, const int64_t n[3], double eps, int eyre, double y2min,
                              double y2max, double *lambda_max);

/* Host-only (no GPU needed).  The schedule of one LIM step as the GPU path runs it
 * (Fig. 1): *p = the Chebyshev order of Eq. (p) for tau * lambda_max; order[k] (k < p,
 * 1-based m) = the parameter used by the k-th iteration of the first sweep m = 1..p (the
 * second sweep m = 2..p reuses order[1..p-1]); a[m-1] = a_m.  order and a are caller-owned host
 * arrays of `capacity` entries (either may be NULL).  capacity = 0 only reports p;
 * 0 < capacity < p is CH_EINVAL.  CH_EINVAL also for tau not finite and > 0, a negative
 * lambda_max or p above 10^6; CH_ENONFINITE for a non-finite lambda_max.                */
ch_status ch_lim_schedule(double tau, double lambda_max, int capacity, int *p, int *order,
                          double *a);

/* Eq. (LIMest): est = ||y1 - y_PC|| / ||y_PC|| with
 * y_PC = y0 - (tau/2) A (F'(y0) + F'(y1) + eps^2 A (y0 + y1)).  Synchronises.             */
ch_status ch_estimate(ch_grid *g, const double *y0, const double *y1, double tau, double *est);

/* Fig. 2: one Krylov run for the linearised IVP (Eq. IVPlin) at y_n with tentative step
 * tau0, tolerance tol_phi (> 0) and dimension mmax.  linear_restart = 0: the run may cut
 * tau (residual-time step choice, Eq. phi_stop) and *tau_used returns the step taken;
 * linear_restart = 1: linear residual-time restarting covers all of tau0 (constant-step
 * use, end of Sec. 4.1).  y_next may not alias y_n.  `stats` (optional) is incremented.
 * CH_EINVAL when tau0 is not finite and > 0, tol_phi <= 0 or mmax is outside [1, capacity]. */
ch_status ch_phi_krylov(ch_grid *g, const double *y_n, double tau0, double tol_phi, int mmax,
                        int linear_restart, int eyre, double *y_next, double *tau_used,
                        ch_stats *stats);

/* One EE2 step (Sec. 4, Eqs. IVPlin, EE2) with the Krylov tolerance of prm (Eq. tol_phi
 * when prm->tol_phi <= 0), linear restarting when prm->adaptive == 0, and the error
 * estimate of Eq. (LIMest) for the step actually taken.  Synchronises.  CH_EINVAL when tau
 * is not finite and > 0 or prm is invalid.                                                */
ch_status ch_ee_step(ch_grid *g, const double *y_n, double tau, const ch_params *prm,
                     double *y_next, double *tau_used, double *est);

/* One LIM step (Sec. 3.1, Fig. 1).  Returns the Chebyshev order p and lambda_max.
 * CH_EINVAL when tau is not finite and > 0 or p of Eq. (p) would exceed 10^6;
 * CH_ENONFINITE when lambda_max is not finite (non-finite y_n).                          */
ch_status ch_lim_step(ch_grid *g, const double *y_n, double tau, int eyre, double *y_next,
                      int *p_used, double *lambda_max);

/* Figs. 3 / 4 (adaptive) or constant-step integration of y from t = 0 to T, in place.
 * Constant steps: ceil(T/tau0) steps, the last one ending exactly at T.  Per-step records
 * are kept for ch_get_records.                                                            */
ch_status ch_integrate(ch_grid *g, const ch_params *prm, double *y, ch_stats *stats);

/* Per-step records of the last ch_integrate (host arrays of length >= max; any may be
 * NULL): step size taken, Krylov dimension at exit of the last run, linear restarts,
 * 1 if the Krylov residual test cut the step, LIM order p, est.  *count = records kept
 * (at most the capacity given to ch_set_record_capacity, default 0 = none).              */
ch_status ch_set_record_capacity(ch_grid *g, int64_t capacity);
ch_status ch_get_records(ch_grid *g, int64_t max, double *tau, int *jexit, int *restarts,
                         int *shrunk, int *p, double *est, int64_t *count);

/* Checkpoint state of an integration: time reached and next step size.  ch_set_state
 * makes the next ch_integrate resume from (t, tau) instead of (0, tau0).                  */
ch_status ch_get_state(ch_grid *g, double *t, double *tau);
ch_status ch_set_state(ch_grid *g, double t, double tau);

/* Diagnostics of Sec. 5.2: discrete energy E_h (Eq. Ediscr, read as h^d [sum F(y) +
 * eps^2/2 sum_a sum ((y_{i+e_a} - y_i)/h_a)^2]) and mass h^d sum y (Eq. m).  Synchronises. */
ch_status ch_energy_mass(ch_grid *g, const double *y, double *energy, double *mass);

/* Number of kernel launches this grid has issued since creation (for launch accounting). */
int64_t ch_kernel_launches(const ch_grid *g);

/* ---- Batches of independent instances ---------------------------------------------------
 * `count` periodic grids of the same dim with their own sizes (n[3i + a], a < dim, each
 * >= 4) and eps[i], advanced together with adaptive EE2 (Fig. 4) by ch_integrate_batch: every
 * instance keeps its own time, step size, Krylov run and controller; one kernel launch serves
 * all instances still before T.  The states are concatenated in one caller-owned device array
 * of FP64 values: instance i occupies [offsets[i], offsets[i] + N_i) (offsets from
 * ch_batch_layout; gaps between instances are ignored).  precision CH_MIXED keeps the Krylov
 * basis and stencil arithmetic in FP32 as for a single grid.  mmax_capacity <= 63.         */
typedef struct ch_batch ch_batch;
ch_status ch_create_batch(int dim, int count, const int64_t *n, const double *eps, int precision,
                          int mmax_capacity, void *cuda_stream, ch_batch **out);
ch_status ch_destroy_batch(ch_batch *b);
/* offsets: count + 1 entries (last = total length of the concatenated array); chunk_len:
 * values per thread block picked by the creation-time tuner.  Either may be NULL.          */
ch_status ch_batch_layout(const ch_batch *b, int64_t *offsets, int *chunk_len);
/* prm: scheme CH_EE2, adaptive 1, no Eyre.  stats (optional) receives `count` entries.
 * When prm->max_steps batch steps pass before every instance reaches T, the call returns
 * CH_ENOTCONV with y and stats holding the state reached (each instance's own t).  Batch
 * steps are counted per scheduling group (below).                                         */
ch_status ch_integrate_batch(ch_batch *b, const ch_params *prm, double *y, ch_stats *stats);
int64_t ch_batch_kernel_launches(const ch_batch *b);
/* Scheduling groups of the batch (1 or 2; 0 for NULL).  With the environment variable
 * CH_BATCH_GROUPS=2 at creation, a batch of at least 16 instances whose instances within a
 * factor 2 of the largest stiffness estimate eps^2 (sum_a 4 n_a^2)^2 + sum_a 4 n_a^2 (the
 * leading terms of ||A_hat||_1 at d = -1, Sec. 3.2) number at most an eighth of it
 * integrates those as a second group, concurrently with the others, on a stream of higher
 * priority; both groups start after earlier work on the batch's stream and the batch's
 * stream waits for both.  Each instance's arithmetic does not depend on its group.  Without
 * the variable every batch is one group.                                                  */
int ch_batch_groups(const ch_batch *b);

/* Kernel classes of the hot path, for launch accounting and timing (no counterpart in the
 * paper: these report where the time of Figs. 1-4 goes on the GPU). */
typedef enum {
    CH_K_PREP = 0,      /* D, G and min/max of y^2 from y^n (linearisation, bound of Fig. 1) */
    CH_K_TSTAGE,        /* stage 1 of the Arnoldi product A_hat v (Fig. 2) */
    CH_K_WSTAGE,        /* stage 2 of A_hat v, fused with h_{1j} */
    CH_K_MGS,           /* one modified Gram-Schmidt pass (Fig. 2) */
    CH_K_PHI,           /* projected phi, residual test, step trace (Fig. 2) */
    CH_K_COMBINE,       /* y^n + V_j (beta u), the Krylov combine (Fig. 2) */
    CH_K_RHS1,          /* stage 1 of f(y) (Eq. IVP) */
    CH_K_RHS2,          /* stage 2 of f(y), fused with norms and Eq. (LIMest) sums */
    CH_K_RESID1,        /* stage 1 of g_hat - A_hat x (LIM update of Fig. 1, restarts) */
    CH_K_RESID2,        /* stage 2 of g_hat - A_hat x with its norm (restart vector) */
    CH_K_LIM2,          /* stage 2 fused with the LIM update (Fig. 1) */
    CH_K_ENERGY,        /* energy and mass */
    CH_K_ARM,           /* Krylov start: beta, tol_phi (Eq. tol_phi) */
    CH_K_ARNOLDI,       /* a whole Arnoldi iteration (Fig. 2) in one launch
                           (sequential passes; Gram-corrected on FP32 grids, j <= 31) */
    CH_K_COUNT
} ch_kernel_class;

/* Start timing every launch of one kernel class with CUDA events recorded on the grid's
 * stream immediately before and after it (kernel_class = -1 stops timing).  Resets the
 * accumulated time and the per-class launch counts.                                      */
ch_status ch_timing_start(ch_grid *g, int kernel_class);

/* Synchronise and report: total event time (ms) and number of timed launches of the timed
 * class, and per-class launch counts since ch_timing_start (counts may be NULL, else an
 * array of CH_K_COUNT entries).  Arnoldi iterations queued after their Krylov run ended
 * return at once; for CH_K_ARNOLDI those launches count neither time nor work.            */
ch_status ch_timing_read(ch_grid *g, double *total_ms, int64_t *timed_launches,
                         int64_t *counts);

/* Algorithmic work of the launches timed since ch_timing_start: floating-point operations
 * (an FMA counts 2) and the bytes the method must move, as each launch computes them from
 * its sizes.  Reported by the classes CH_K_ARNOLDI (Arnoldi iteration j on N points; FP64
 * sequential passes: (4 + 6d + 4j) N flops, (5 + j) N values moved; FP32 Gram-corrected
 * form: (4 + 6d + 6j) N flops, (6 + 2j) N values), CH_K_RESID1 ((2 + 3d) N flops, 32 N
 * bytes) and CH_K_LIM2 ((5 + 3d) N flops, 32 N bytes); 0 for the others.  Does not
 * synchronise; read it after ch_timing_read.                                            */
ch_status ch_timing_work(ch_grid *g, double *flops, double *bytes);

/* Time one kernel class in isolation on this grid's current workspace: R back-to-back
 * launches captured in a CUDA graph, CUDA events on the grid's stream around the graph.
 * Returns the mean duration of one launch and its algorithmic traffic and arithmetic per
 * launch (bytes the kernel must move, floating-point operations counting an FMA as 2, and
 * issued FP64-pipe instructions for FP64 grids).  Supported classes: CH_K_ARNOLDI (j = 10,
 * on grids that run fused Arnoldi iterations), CH_K_TSTAGE,
 * CH_K_WSTAGE, CH_K_MGS, CH_K_RESID1, CH_K_LIM2, CH_K_RHS1, CH_K_RHS2.  Call after an
 * integration so the workspace holds finite data.  Synchronises.                         */
ch_status ch_bench_kernel(ch_grid *g, int kernel_class, int reps, double *avg_us,
                          double *bytes_per_launch, double *flops_per_launch,
                          double *fp64_instr_per_launch);

/* ---- Energy and mass without any allocation ------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot let a library
 * allocate device memory: applications that hand out all device memory from their own pool
 * (a caching allocator or a fixed arena sized at start-up), and callers keeping work running
 * concurrently on several streams, where the device synchronisation that cudaMalloc / cudaFree
 * may cause would stall it.  It computes what ch_energy_mass computes (discrete energy and
 * mass of y on a periodic grid of dim 2 or 3 with n[a] >= 1 points per axis, at most
 * 2^31 - 1 points in all) without a grid object: the caller passes y (device, N doubles) and
 * out (device, 2 doubles: energy, mass), and the work is queued on cuda_stream without a
 * synchronisation.  Its reduction scratch is a fixed 16 KiB + 256 B array in the library's
 * device image (every GPU that loads the library holds it until the process exits); all
 * calls on a device share it, so calls whose work overlaps on the GPU (different streams, or
 * unordered host threads) race and must be serialised by the caller.  The first call on each
 * device does a one-time set-up (it looks up the array's device address with
 * cudaGetSymbolAddress); make that first call before any stream capture.  Grids beyond
 * 2^31 - 1 points are rejected with CH_EINVAL, and so are y or out that are not device (or
 * managed) memory of the current device, which is where the work runs; cuda_stream must
 * belong to that device too.                                                                */
ch_status ch_energy_mass_noalloc(int dim, const int64_t n[3], double eps, const double *y,
                                 double *out, void *cuda_stream);

/* Measured FP64 FMA rate of the current GPU in TFLOP/s (an FMA counts 2): independent FMA
 * chains from registers on a grid of all resident blocks, the best over a few shapes (4, 8
 * or 16 chains per thread, 256 or 1024 threads per block), each timed with CUDA events on
 * cuda_stream after a warm-up launch.  No counterpart in the paper: it is the roofline
 * denominator of the FP64 kernels, which are bound by FP64 issue on GB300.  Allocates and
 * frees a small output buffer; synchronises the stream.                                   */
ch_status ch_probe_fp64_peak(void *cuda_stream, double *tflops);

/* Message of the last error on the calling thread ("" when none). */
const char *ch_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CH_H_ */
