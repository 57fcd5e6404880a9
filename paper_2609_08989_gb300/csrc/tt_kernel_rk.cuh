// tt_kernel_rk.cuh -- FP64 persistent tracing kernels for the integrators of
// paper Sec. 3.2 other than Dormand-Prince: the Cash-Karp (1) and Fehlberg (2)
// 5(4) pairs, the Gragg-Bulirsch-Stoer extrapolator (3) and Verlet (4), for
// closed-form Kerr (128 or 256 threads) and tabulated metrics (128 threads).
// Each integrator is built in a translation unit of its own, which defines
// TT_RK_METHOD and includes this file.
#pragma once

#include "tt_trace.cuh"

namespace tt {

template <int METHOD, int METRIC, int N, int BLOCK>
__global__ void __launch_bounds__(BLOCK) trace_kernel_rk(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<METRIC, 0, METHOD>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

template <int METHOD, int N>
static cudaError_t launch_rk_n(const ImageDesc* descs, int n, long long total, int metric_mode,
                               const SolverDesc& sol, const LaunchShape& shape, unsigned long long* queue,
                               cudaStream_t stream) {
    LaunchParams<N> p;
    fill_params<N>(p, descs, n, total, sol, shape, queue);
    const int bps = shape.blocks_per_sm;
    if (metric_mode == 0) {
        if (shape.block >= 256) return launch_persistent<N>(trace_kernel_rk<METHOD, 0, N, 256>, 256, bps, p, stream);
        return launch_persistent<N>(trace_kernel_rk<METHOD, 0, N, 128>, 128, bps, p, stream);
    }
    if (metric_mode == 1) return launch_persistent<N>(trace_kernel_rk<METHOD, 1, N, 128>, 128, bps, p, stream);
    return cudaErrorInvalidValue;
}

template <int METHOD>
cudaError_t launch_rk(const ImageDesc* descs, int n, long long total, int metric_mode, const SolverDesc& sol,
                      const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    if (n == 1) return launch_rk_n<METHOD, 1>(descs, n, total, metric_mode, sol, shape, queue, stream);
    return launch_rk_n<METHOD, kMaxImagesPerLaunch>(descs, n, total, metric_mode, sol, shape, queue, stream);
}

template cudaError_t launch_rk<TT_RK_METHOD>(const ImageDesc*, int, long long, int, const SolverDesc&,
                                             const LaunchShape&, unsigned long long*, cudaStream_t);

}  // namespace tt
