// tt_internal.h -- descriptors passed from the host API to the tracing kernels.
//
// Everything a kernel needs about one image is resolved on the host once
// (thresholds, disk constants, camera spacing) and handed over as a flat,
// trivially copyable struct; a batch is an array of them in device memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tt {

constexpr int kMaxCross = 3;
constexpr int kTableNF = 20;         // doubles per table node (5 fields x value, 2 slopes, twist)
constexpr int kTableCoef = 80;       // doubles per table cell (5 fields x 16 patch coefficients)

struct ImageDesc {
    // camera
    int nx, ny;
    long long pix_begin, pix_count;
    double alpha_min, dalpha, beta_min, dbeta;
    // observer
    double r_obs, theta_obs;
    // the flags, packed (the batch of descriptors travels as kernel parameters):
    // metric kind (0 Kerr, 1 table), observer tetrad resolved (below), disk
    // enabled, crossings to record, Doppler factor in the redshift
    int kind;
    int8_t obs_ready, disk, max_cross, doppler;
    // ZAMO tetrad at the observer, resolved on the host for the closed-form
    // metric (obs_ready = 1): g_tt, g_tphi, g_rr, g_thth, g_phiphi, omega/N,
    // 1/N, 1/sqrt(g_rr), 1/sqrt(g_thth), 1/sqrt(g_phiphi)
    double obs_g[5];
    double obs_omN, obs_iN, obs_ir, obs_ith, obs_iph;
    // metric
    double M, a;
    const double* table;          // device patch coefficients, cell-major (see tt_capi.cu)
    const float2* table_df;       // the same as double-float (hi, lo) pairs
    int nr, nth;
    double u0, du, dth;           // ln r_min, ln-spacing, theta spacing
    float2 u0_df, idu_df, idth_df;          // u0, 1/du, 1/dth as double-float (hi, lo)
    // events
    double r_capture;             // r_h (1 + horizon_eps)
    double r_escape;              // escape_factor * r_obs
    double r_fp64;                // mixed paths: double-float steps below this radius
    double th_pole;               // mixed paths: double-float steps within this angle of the axis
    double r_plus, r_minus;       // Kerr horizons (mixed path: Delta = (r - r_+)(r - r_-))
    // disk
    double r_in, r_out, mdot;
    double fx0, fa;               // x0 = sqrt(r_isco / M), a / M
    double fxr[3], fcoef[3], flog0[3];   // roots x_i, their coefficients, log(x0 - x_i)
    double flux_scale;            // mdot / M^2
    double sqrtM;
    // outputs (device)
    int8_t* code;
    int8_t* n_cross;
    double* r_cross;
    double* g;
    double* I_cross;
    double* intensity;
    double* h_max;
    int32_t* steps;
    int32_t* rejects;
    // position of the image's first ray in the shared queue
    long long ray_begin;
};

struct SolverDesc {
    double rtol, atol, h0, h_min;
    long long max_steps;
    int refine;                   // 0 Henon, 1 Hermite, 2 Henon in FP64 on the mixed paths too
    int precision;                // 0 FP64, 1 mixed (FP64 state), 2 mixed (FP32-pair state),
                                  // 3 double-float, 4 mixed with the FP64 norm, zone steps and refinement
    int method;                   // 0 Dormand-Prince; FP64 only: 1 Cash-Karp, 2 Fehlberg, 3 GBS, 4 Verlet
    // mixed paths: rays within crit_band (units of M) of the critical curve are
    // traced in double-float at crit_rtol / crit_atol (0: none)
    double crit_band, crit_rtol, crit_atol;
    // bounds-checking build (TT_BOUNDS_CHECK): counter of output stores whose
    // index fell outside their buffer (skipped, never made); unused otherwise
    unsigned long long* faults;
};

struct LaunchShape {
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
};

// Warp-phase thresholds of the persistent loop (see tt_kernel.cu).
struct TuneParams {
    int refill;           // refill when at least this many lanes are done or idle
    int crossing_batch;   // refine crossings once this many lanes have one pending
    int fp64_batch;       // mixed: run the double-float zone steps once this many lanes need one
    int monitor_period;   // mixed: FP64 |H| check every this many iterations
    int fp64_wait;        // mixed: zone steps run after this many iterations of waiting
    int crit_stride;      // mixed: the warps of one SM in crit_stride start with the near-critical rays
    int crit_refill;      // mixed: refill threshold of a warp tracing near-critical rays
};

// Images handed to one launch by value (kernel parameters, no host-to-device
// copy and therefore no stream synchronisation).  Larger batches are split.
constexpr int kMaxImagesPerLaunch = 64;

template <int N>
struct LaunchParams {
    SolverDesc sol;
    SolverDesc solc;                 // mixed paths: the settings of the near-critical rays
    int n_desc;
    TuneParams tune;
    long long total;                 // rays over all images
    unsigned long long* queue;       // two zeroed 64-bit counters: [0] the ray queue, [1] the
                                     // mixed paths' scan for near-critical rays
    ImageDesc desc[N];
};

// Enqueue the persistent tracing kernel over n <= kMaxImagesPerLaunch images.
// FP64 kernels of the Cash-Karp (METHOD 1) and Fehlberg (2) pairs, the
// Gragg-Bulirsch-Stoer extrapolator (3) and Verlet (4) for metric_mode 0 or 1
// (one explicit instantiation per translation unit).
template <int METHOD>
cudaError_t launch_rk(const ImageDesc* descs, int n, long long total, int metric_mode, const SolverDesc& sol,
                      const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream);

// metric_mode: 0 closed-form Kerr only, 1 tables only, 2 both (per-ray dispatch).
cudaError_t launch_trace(const ImageDesc* descs, int n, long long total_rays, int metric_mode,
                         const SolverDesc& sol, const LaunchShape& shape,
                         unsigned long long* queue, cudaStream_t stream);

// Device properties needed for the persistent grid.
int sm_count();

}  // namespace tt
