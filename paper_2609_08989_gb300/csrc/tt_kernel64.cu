// tt_kernel64.cu -- FP64 persistent tracing kernels and the launch dispatch.
#include "tt_trace.cuh"

namespace tt {

template <int METRIC, int N>
__global__ void __launch_bounds__(128) trace_kernel64(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<METRIC, 0>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

template <int METRIC, int N>
__global__ void __launch_bounds__(256) trace_kernel64_b256(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<METRIC, 0>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

// 384 threads (12 warps per SM at 160 registers, against 8 for 256 threads).
template <int METRIC, int N>
__global__ void __launch_bounds__(384) trace_kernel64_b384(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<METRIC, 0>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

// Register-capped builds of the closed-form Kerr kernel (128 threads): at least
// MINB resident blocks per SM caps registers at 65536 / (128 MINB) per thread
// (MINB 3: 168, MINB 4: 128).
template <int MINB>
__global__ void __launch_bounds__(128, MINB) trace_kernel64_regcap(const __grid_constant__ LaunchParams<1> p) {
    trace_loop<0, 0>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Built variants: closed-form Kerr (128, 256 and 384 threads), tables (128),
// and batches that mix both kinds (128, batch width only); a block size
// without a build of its own runs at the kernel's built size.
template <int N>
static cudaError_t launch64(const ImageDesc* descs, int n, long long total, int metric_mode, const SolverDesc& sol,
                            const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    LaunchParams<N> p;
    fill_params<N>(p, descs, n, total, sol, shape, queue);
    const int bps = shape.blocks_per_sm;
    if (metric_mode == 0) {
        if (shape.block == 256) return launch_persistent<N>(trace_kernel64_b256<0, N>, 256, bps, p, stream);
        if (shape.block == 384) return launch_persistent<N>(trace_kernel64_b384<0, N>, 384, bps, p, stream);
        if constexpr (N == 1) {
            if (shape.reg_variant == 1) return launch_persistent<N>(trace_kernel64_regcap<3>, 128, bps, p, stream);
            if (shape.reg_variant == 2) return launch_persistent<N>(trace_kernel64_regcap<4>, 128, bps, p, stream);
        }
        return launch_persistent<N>(trace_kernel64<0, N>, 128, bps, p, stream);
    }
    if (metric_mode == 1) return launch_persistent<N>(trace_kernel64<1, N>, 128, bps, p, stream);
    return cudaErrorInvalidValue;
}

static cudaError_t launch64_mixed_kinds(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                                        const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    LaunchParams<kMaxImagesPerLaunch> p;
    fill_params<kMaxImagesPerLaunch>(p, descs, n, total, sol, shape, queue);
    return launch_persistent<kMaxImagesPerLaunch>(trace_kernel64<2, kMaxImagesPerLaunch>, 128, shape.blocks_per_sm,
                                                  p, stream);
}

cudaError_t launch_trace(const ImageDesc* descs, int n, long long total_rays, int metric_mode,
                         const SolverDesc& sol, const LaunchShape& shape, unsigned long long* queue,
                         cudaStream_t stream) {
    if (n < 1 || n > kMaxImagesPerLaunch) return cudaErrorInvalidValue;
    if (sol.method != 0) {
        if (sol.precision != 0 || metric_mode == 2) return cudaErrorInvalidValue;
        if (sol.method == 1) return launch_rk<1>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
        if (sol.method == 2) return launch_rk<2>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
        if (sol.method == 3) return launch_rk<3>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
        if (sol.method == 4) return launch_rk<4>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
        return cudaErrorInvalidValue;
    }
    if (sol.precision == 3) return launch_df(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
    if (sol.precision != 0) {
        if (metric_mode != 0) return cudaErrorInvalidValue;
        return launch_mixed(descs, n, total_rays, sol, shape, queue, stream);
    }
    if (metric_mode == 2) return launch64_mixed_kinds(descs, n, total_rays, sol, shape, queue, stream);
    if (n == 1) return launch64<1>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
    return launch64<kMaxImagesPerLaunch>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
}

}  // namespace tt
