/*
 * tartarus.h -- C ABI of the GB300 geodesic ray tracer.
 *
 * Backward tracing of one null geodesic per image-plane pixel from a distant
 * observer through a Kerr metric (closed form) or a tabulated (r, theta)
 * metric, after TARTARUS (arXiv 2609.08989):
 *   - Hamiltonian flow H = 1/2 g^{mu nu} p_mu p_nu, H = 0            (Sec. 2.1)
 *   - initial momenta from the ZAMO tetrad at (r_obs, theta_obs)     (Sec. 2.2)
 *   - adaptive Dormand-Prince 5(4) with horizon / escape / disk events (Sec. 3.2)
 *   - Page-Thorne flux F(r), redshift g and I = g^4 F at crossings    (Sec. 2.3-2.4)
 *   - the constraint residual |H| monitored after every accepted step (Sec. 4.1)
 *
 * Conventions.  Geometric units G = c = 1, Boyer-Lindquist coordinates.
 * The state integrated is the time-reversed photon: p_mu -> -p_mu of the
 * physical, future-directed momentum, with the affine parameter increasing.
 * A pixel (i, j) of an nx x ny camera sits at the cell centre
 *   alpha = alpha_min + (i + 1/2) (alpha_max - alpha_min) / nx,
 *   beta  = beta_min  + (j + 1/2) (beta_max  - beta_min)  / ny,
 * and has the linear index p = j nx + i.
 *
 * Errors.  Every entry point returns 0 (TT_OK) or a negative TT_E* code; no
 * exception or abort crosses the ABI.  Invalid arguments are reported before
 * anything is launched.  Numerical failures of single rays are not call
 * errors: they are per-pixel termination codes (TT_CODE_*).
 *
 * Ownership.  The caller owns every output buffer and every descriptor.  The
 * library owns the device copies of metric tables (until
 * tartarus_table_destroy) and a small per-device work-queue buffer that lives
 * until the process exits.
 *
 * Streams.  Work is enqueued on the CUDA stream passed in (NULL = the legacy
 * default stream) and returns without synchronising, except the *_host entry
 * point, which synchronises its stream before returning.
 */
#ifndef TARTARUS_H
#define TARTARUS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define TT_OK            0
#define TT_EINVAL       -1   /* an argument is out of range; nothing launched   */
#define TT_ENOMEM       -2   /* a device or pinned allocation failed            */
#define TT_ECUDA        -3   /* a CUDA runtime call failed (see error string)   */
#define TT_EUNSUPPORTED -4   /* the request names a variant that is not built   */

/* ---- per-pixel termination codes (int8) ------------------------------- */
#define TT_CODE_ESCAPED   0  /* r > escape_factor * r_obs (paper Sec. 3.2, C_E)            */
#define TT_CODE_CAPTURED  1  /* r < r_h (1 + horizon_eps) (paper Sec. 3.2, C_H)            */
#define TT_CODE_MAXSTEPS  2  /* accepted + rejected steps reached max_steps                */
#define TT_CODE_UNDERFLOW 3  /* step size fell below h_min                                  */
#define TT_CODE_NONFINITE 4  /* a NaN or Inf appeared in the state or the error estimate    */
#define TT_CODE_BADPIXEL  5  /* alpha^2 + beta^2 >= r_obs^2, or a non-finite pixel position  */

#define TT_MAX_CROSSINGS 3   /* disk crossings stored per pixel */

/* ---- enumerations ---------------------------------------------------- */
#define TT_METRIC_KERR   0
#define TT_METRIC_TABLE  1
#define TT_DP54          0   /* Dormand-Prince 5(4) (paper Sec. 3.2)   */
#define TT_CK45          1   /* Cash-Karp 5(4) (paper Sec. 3.2), FP64 only */
#define TT_F45           2   /* Fehlberg 5(4) (paper Sec. 3.2), FP64 only  */
#define TT_GBS           3   /* Gragg-Bulirsch-Stoer extrapolation (Sec. 3.2), FP64 only */
#define TT_VERLET        4   /* Stormer-Verlet, fixed step h0 > 0 (Sec. 3.2), FP64 only  */
#define TT_FP64          0   /* all arithmetic in binary64             */
#define TT_MIXED         1   /* FP32 stages, FP64 state accumulation   */
#define TT_MIXED_PAIR    2   /* FP32 stages, compensated FP32-pair state accumulation (~48 bits) */
#define TT_DOUBLE_FLOAT  3   /* every stage in double-float (FP32 pairs, ~48 bits) on the FP32 pipe */
#define TT_MIXED_SPLIT   4   /* FP32 stages; FP64 state accumulation, error norm and step control,
                                FP64 steps near the horizon and FP64 crossing refinement */
#define TT_REFINE_HENON   0  /* exact step onto theta = pi/2 (default) */
#define TT_REFINE_HERMITE 1  /* paper's cubic-Hermite bisection        */
#define TT_REFINE_HENON64 2  /* Henon with FP64 stages on the mixed paths too (default there: FP32 stages) */

typedef struct tt_table tt_table;        /* opaque device copy of a metric table */

/* Spacetime.  kind TT_METRIC_KERR: mass M > 0, spin |a| < M.
 * kind TT_METRIC_TABLE: 'table' from tartarus_table_create; M and a are then
 * used only by the disk model (ISCO, Keplerian Omega, Page-Thorne flux). */
typedef struct {
    int kind;
    double M, a;
    const tt_table *table;
} tt_metric;

/* Observer at r_obs > 0 and inclination 0 < theta_obs < pi (radians). */
typedef struct {
    double r_obs, theta_obs;
} tt_observer;

/* Camera grid; pixels [pix_begin, pix_begin + pix_count) are traced and written
 * to outputs index 0 .. pix_count-1.  pix_count <= 0 means "to the end". */
typedef struct {
    int nx, ny;
    double alpha_min, alpha_max, beta_min, beta_max;
    long long pix_begin, pix_count;
} tt_camera;

/* Integrator (paper Sec. 3.2).  rtol, atol > 0.  h0 <= 0: automatic start step
 * (Hairer-Norsett-Wanner starting-step algorithm).  h_min <= 0: 1e-14 max(1, |lambda|).
 * max_steps >= 1 caps accepted + rejected steps.  Captured when
 * r < r_h (1 + horizon_eps), escaped when r > escape_factor * r_obs
 * (escape_factor > 1).  fp64_radius_factor (mixed paths, and the
 * double-float path on a table): steps that start at r < fp64_radius_factor *
 * r_h run in extended precision (0 selects 1.5 on the mixed paths and 2 on a
 * table; negative: none); so do steps that start within asin(fp64_pole_sin) of
 * the polar axis (0 or negative: none).  The FP32 stages of the mixed paths
 * take theta relative to the nearest axis crossing (theta - m pi), so that
 * sin(theta) keeps FP32's relative precision near both poles; with the
 * defaults every escaped ray keeps |H| <= 1e-6 at rtol 1e-8.  TT_MIXED and
 * TT_MIXED_PAIR run these extended-precision
 * steps in double-float (FP32-pair, ~48-bit) arithmetic on the FP32 pipe;
 * TT_MIXED_SPLIT runs them in FP64, forms the error norm and the step-size
 * control of its FP32 steps in FP64 from the FP32 error terms, and refines
 * crossings with FP64 stages (the precision split stated for the mixed path,
 * kept for comparison).
 * critical_band, critical_rtol (mixed paths): a photon whose radial potential
 * R(r) = r^4 + (a^2 - xi^2 - eta) r^2 + 2M (eta + (xi - a)^2) r - a^2 eta
 * (xi = L/E, eta = Q/E^2, from its initial data) has a near-double root
 * outside the horizon passes close to the unstable spherical photon orbits,
 * and each circuit around them multiplies any perturbation of the ray by
 * ~e^pi, so FP32 stage rounding (~1e-7) would reach its later crossings.
 * A ray whose distance from the critical curve, estimated as
 * R(r_m) / (2 r_m^2 b) at the local minimum r_m of R (b^2 = xi^2 + eta), is
 * below critical_band (in units of M) is traced entirely in double-float, as
 * TT_DOUBLE_FLOAT traces it, at rtol = atol = critical_rtol; these rays are
 * traced first, by whole warps, in the same launch.  critical_band 0 selects
 * 0.15 on TT_MIXED and TT_MIXED_PAIR and none on TT_MIXED_SPLIT, negative:
 * none; critical_rtol 0 selects 1e-10.  Other precisions ignore both.
 * TT_DOUBLE_FLOAT steps every ray in double-float: flow, stage points, stage
 * sums and error estimate (with double-float coefficients) and the state, with
 * an FP32 error norm and step control; crossings are refined and emission
 * evaluated in FP64.  On a table its zone steps run in FP64, where the
 * interpolated D = g_tt g_phiphi - g_tphi^2 goes to zero at the horizon.
 * TT_MIXED, TT_MIXED_PAIR and TT_MIXED_SPLIT are available for the
 * closed-form Kerr metric (with a table they return TT_EUNSUPPORTED);
 * TT_DOUBLE_FLOAT for either
 * kind, but a batch that mixes both kinds returns TT_EUNSUPPORTED for it.
 * h_max is the largest |H| seen: on the FP64 path at the start and after every
 * accepted step; on the double-float path at the start (FP64) and after every
 * accepted step (double-float); on the mixed paths after every double-float
 * or FP64 step, and in FP64 at the start of every step with a disk crossing,
 * every monitor_period warp iterations and at the end (rays of the critical
 * band as on the double-float path).
 * method: one of the five integrators of Sec. 3.2.  The embedded 5(4) pairs
 * (TT_DP54, TT_CK45, TT_F45) propagate their fifth-order solution and take the
 * difference to the fourth-order one as the error estimate.  TT_GBS: macro-
 * steps of Gragg's modified midpoint rule with 2, 4, ..., 12 sub-steps,
 * extrapolated in h^2 (Aitken-Neville, 6 columns); the error estimate is the
 * difference of the two highest-order entries, and the step adapts with the
 * factor 0.94 (0.65/err)^(1/11), clamped to [0.02, 4].  TT_VERLET: the
 * Stormer-Verlet scheme for the non-separable H (implicit half steps solved by
 * fixed-point iteration to 1e-15 relative, at most 50 iterations) with the
 * fixed step h0, which must be > 0 (TT_EINVAL otherwise); rtol/atol are unused
 * and rejects stay 0.  Every method other than TT_DP54 runs in FP64 only
 * (other precisions return TT_EUNSUPPORTED), for either metric kind, but a
 * batch that mixes closed-form Kerr and tabulated images returns
 * TT_EUNSUPPORTED for them, with nothing launched; other values of method give
 * TT_EINVAL.  With TT_REFINE_HENON, crossings of TT_GBS and TT_VERLET rays are
 * refined with Dormand-Prince sub-steps.  tt_tune.reg_variant applies to
 * TT_DP54 only. */
typedef struct {
    int method;                 /* TT_DP54, TT_CK45, TT_F45, TT_GBS or TT_VERLET */
    int precision;              /* TT_FP64, TT_MIXED, TT_MIXED_PAIR, TT_DOUBLE_FLOAT or TT_MIXED_SPLIT */
    double rtol, atol, h0, h_min;
    long long max_steps;
    double horizon_eps, escape_factor;
    int refine;                 /* TT_REFINE_HENON, TT_REFINE_HERMITE or TT_REFINE_HENON64 */
    double fp64_radius_factor;
    double fp64_pole_sin;
    double critical_band;
    double critical_rtol;
} tt_solver;

/* Thin disk in the equatorial plane (paper Sec. 2.3).  r_in <= 0 selects the
 * prograde ISCO (requires a >= 0).  max_crossings in 0..3 are stored; all
 * crossings with r_in <= r <= r_out are counted.  doppler = 0 drops the
 * Omega p_phi term of the redshift (paper Fig. 3b). */
typedef struct {
    int enabled;
    double r_in, r_out, mdot;
    int max_crossings;
    int doppler;
} tt_disk;

/* Outputs: caller-owned DEVICE buffers of pix_count elements, except the three
 * crossing arrays, which hold 3 * pix_count doubles, crossing-major (crossing k
 * of output pixel q at [k * pix_count + q]).  Unused crossing slots are 0.
 *   code       int8  termination code
 *   n_cross    int8  number of in-range crossings (saturates at 127)
 *   r_cross    f64   crossing radius
 *   g          f64   redshift factor nu_obs / nu_em
 *   I_cross    f64   g^4 F(r)
 *   intensity  f64   sum of I_cross over the stored crossings
 *   h_max      f64   max |H| over the initial state and every accepted step
 *   steps      int32 accepted steps
 *   rejects    int32 rejected steps                                      */
typedef struct {
    int8_t *code;
    int8_t *n_cross;
    double *r_cross;
    double *g;
    double *I_cross;
    double *intensity;
    double *h_max;
    int32_t *steps;
    int32_t *rejects;
} tt_outputs;

/* Launch shape of the persistent kernel; NULL or zero fields select defaults.
 *   block           threads per block, 0 (default), 128, 256 or 384.  Built:
 *                   FP64 Dormand-Prince on the closed-form metric 128 (default),
 *                   256 and 384; the other FP64 integrators 128 (default) and
 *                   256 (384 runs as 256); tables 128 (any size runs as 128);
 *                   mixed paths 256 (default; 384 runs as 256, 128 fails with
 *                   TT_ECUDA).  Other sizes: TT_EUNSUPPORTED.
 *   reg_variant     registers per thread of the FP64 closed-form Kerr kernel at
 *                   128 threads, single camera: 0 the compiler's choice, 1 at
 *                   most 168, 2 at most 128 (other kernels ignore it)
 *   refill          flush finished rays and refill lanes once at least this many
 *                   lanes of a warp are done or idle (1..32; default 32)
 *   blocks_per_sm   persistent blocks per SM (0: as many as fit)
 *   crossing_batch  refine disk crossings once this many lanes of a warp have
 *                   one pending (1..32; default 16 FP64, 32 otherwise)
 *   fp64_batch      mixed paths (and the double-float path on a table): run the
 *                   extended-precision zone steps once this many lanes need one
 *                   (1..32, default 32; 1 on the double-float path)
 *   monitor_period  mixed paths: evaluate |H| in FP64 every this many warp
 *                   iterations (default 32)
 *   fp64_wait       mixed paths: lanes waiting for a zone step get one after at
 *                   most this many warp iterations (default 64)
 *   crit_stride     mixed paths with a critical band: the warps of one SM in
 *                   crit_stride start by scanning for near-critical rays
 *                   (default 1: every SM)
 *   crit_refill     mixed paths: a warp tracing near-critical rays refills once
 *                   this many lanes are free (1..32, default 32) */
typedef struct {
    int block;
    int reg_variant;
    int refill;
    int blocks_per_sm;
    int crossing_batch;
    int fp64_batch;
    int monitor_period;
    int fp64_wait;
    int crit_stride;
    int crit_refill;
} tt_tune;

/* Trace one camera (paper Sec. 3.1 execution flow, steps 1-6): every pixel of
 * the range gets its initial data, is integrated to a terminal event, and has
 * its crossings refined and their emission evaluated.  Asynchronous on stream.
 * Returns TT_EINVAL for inconsistent arguments (nothing launched), TT_ECUDA if
 * the launch fails. */
int tartarus_trace(const tt_metric *metric, const tt_observer *obs, const tt_camera *cam,
                   const tt_solver *solver, const tt_disk *disk, const tt_outputs *out,
                   const tt_tune *tune, void *cuda_stream);

/* Same as tartarus_trace, but the outputs are HOST buffers (pinned memory is
 * fastest): the library traces into device buffers it owns and copies the
 * results back; it synchronises the stream before returning. */
int tartarus_trace_host(const tt_metric *metric, const tt_observer *obs, const tt_camera *cam,
                        const tt_solver *solver, const tt_disk *disk, const tt_outputs *host_out,
                        const tt_tune *tune, void *cuda_stream);

/* One image of a batch. */
typedef struct {
    tt_metric metric;
    tt_observer obs;
    tt_camera cam;
    tt_disk disk;
    tt_outputs out;
} tt_image;

/* Trace n images of uneven size, spin and inclination in ONE persistent launch
 * that pulls rays from a shared queue (replaces the paper's per-pixel thread
 * pool, Sec. 4.3).  All images share the solver settings.  An image whose
 * descriptor is invalid is skipped and reported in status[i] (TT_EINVAL) if
 * status is not NULL; the call then returns TT_EINVAL but still traces the
 * valid images.  Asynchronous on stream. */
int tartarus_trace_batch(const tt_image *images, int n, const tt_solver *solver,
                         const tt_tune *tune, int *status, void *cuda_stream);

/* tartarus_trace_batch without any allocation (the paper has no counterpart;
 * this is an interface for embedding).  For callers that must not allocate
 * device memory once they are running -- for example an application that
 * reserves its whole GPU memory budget at start-up and hands out all buffers
 * itself, where a CUDA allocation made by a library could exceed or fragment
 * that budget.  tartarus_trace and tartarus_trace_batch allocate a small
 * counter buffer on their first call on a device; this entry point instead
 * uses a fixed 4 KiB array of work-queue counters compiled into the library
 * (present on every device that loads it, until the process exits).
 * Arguments, outputs and results are those of tartarus_trace_batch; the
 * caller still owns every output buffer.  Limits and rules:
 *   - at most 1024 images per call (16 counters, one per launch of up to 64
 *     images); larger n returns TT_EINVAL before anything is launched;
 *   - the first call on a device looks up the array's device address (a
 *     runtime symbol query, no allocation) with that device current; make
 *     that first call before any stream capture;
 *   - every call shares the same counters and zeroes the ones it uses on its
 *     stream before each launch, so two calls whose work overlaps on the GPU
 *     (different streams, or different host threads) race on them: serialise
 *     such calls, e.g. by issuing them on one stream;
 *   - every image is validated, and status[] written, before the first launch;
 *     a TT_ECUDA return means that a launch failed after the earlier chunks of
 *     64 images were enqueued.
 * No cudaMalloc, cudaFree or other allocating routine is called. */
int tartarus_trace_batch_noalloc(const tt_image *images, int n, const tt_solver *solver,
                                 const tt_tune *tune, int *status, void *cuda_stream);

/* Copy a metric table to the device (paper: numerically generated metrics).
 * host_nodes holds nth * nr * 20 doubles: node (j, k) at [(j nr + k) 20], with
 * r_k = r_min (r_max / r_min)^(k/(nr-1)) and theta_j = pi j / (nth-1); for each
 * field F in (g_tt, g_tphi, g_thth, g_phiphi, g^rr) the four numbers
 * F, dF/dr, dF/dtheta, d2F/(dr dtheta).  r_min is taken as the horizon.
 * Interpolation is bicubic Hermite in (ln r, theta).  nr, nth >= 2,
 * 0 < r_min < r_max.  The host array may be freed after the call. */
int tartarus_table_create(const double *host_nodes, int nr, int nth, double r_min, double r_max,
                          tt_table **out);
int tartarus_table_destroy(tt_table *table);

/* Host only (no GPU, no CUDA call): the per-cell patch coefficients that
 * tartarus_table_create uploads, for the same arguments and with the same
 * validation (TT_EINVAL on null pointers, nr or nth < 2, bad radii or a
 * non-finite node value).  out (caller-owned) receives (nth - 1)(nr - 1) * 80
 * doubles: cell (j, k) -- theta interval j, radial interval k -- at offset
 * (j (nr - 1) + k) * 80, then per field f in the node order (g_tt, g_tphi,
 * g_thth, g_phiphi, g^rr) 16 numbers c[4 i + q], the coefficients of t^i w^q
 * in the field's bicubic Hermite patch, where t = (ln r - ln r_min)/du - k and
 * w = theta/dth - j are the cell's unit coordinates (du = ln(r_max/r_min)/(nr-1),
 * dth = pi/(nth-1)). */
int tartarus_table_coefficients(const double *host_nodes, int nr, int nth, double r_min, double r_max,
                                double *out);

/* Static description of a status code. */
const char *tartarus_error_string(int status);

/* Number of kernels this library has launched in this process. */
long long tartarus_launch_count(void);

/* Bounds-checking build only (the library compiled with TT_BOUNDS_CHECK, a
 * test artefact): every output store of the kernels is checked against its
 * buffer's length, and a store that would fall outside is skipped and counted
 * instead (no trap, no fault).  Synchronises the device, writes the number of
 * such stores since the last call to *count and resets it.  The ordinary
 * build writes 0 and returns TT_EUNSUPPORTED.  TT_EINVAL if count is NULL. */
int tartarus_debug_faults(long long *count);

/* Version string. */
const char *tartarus_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TARTARUS_H */
