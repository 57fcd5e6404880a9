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
constexpr int kTableNF = 20;

struct ImageDesc {
    // camera
    int nx, ny;
    long long pix_begin, pix_count;
    double alpha_min, dalpha, beta_min, dbeta;
    // observer
    double r_obs, theta_obs;
    // metric
    int kind;                     // 0 Kerr, 1 table
    double M, a;
    const double* table;          // device nodes in local-slope form (see tt_capi.cu)
    int nr, nth;
    double u0, du, dth;           // ln r_min, ln-spacing, theta spacing
    // events
    double r_capture;             // r_h (1 + horizon_eps)
    double r_escape;              // escape_factor * r_obs
    double r_fp64;                // mixed path: FP64 steps below this radius
    // disk
    int disk, max_cross, doppler;
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
    int refine;                   // 0 Henon, 1 Hermite
    int precision;                // 0 FP64, 1 mixed
};

struct LaunchShape {
    int block;
    int reg_variant;
    int refill;
    int blocks_per_sm;
};

// Images handed to one launch by value (kernel parameters, no host-to-device
// copy and therefore no stream synchronisation).  Larger batches are split.
constexpr int kMaxImagesPerLaunch = 64;

template <int N>
struct LaunchParams {
    SolverDesc sol;
    int n_desc;
    int refill;
    long long total;                 // rays over all images
    unsigned long long* queue;       // zeroed 64-bit counter
    ImageDesc desc[N];
};

// Enqueue the persistent tracing kernel over n <= kMaxImagesPerLaunch images.
// metric_mode: 0 closed-form Kerr only, 1 tables only, 2 both (per-ray dispatch).
cudaError_t launch_trace(const ImageDesc* descs, int n, long long total_rays, int metric_mode,
                         const SolverDesc& sol, const LaunchShape& shape,
                         unsigned long long* queue, cudaStream_t stream);

// Device properties needed for the persistent grid.
int sm_count();

}  // namespace tt
