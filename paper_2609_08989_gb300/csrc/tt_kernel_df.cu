// tt_kernel_df.cu -- double-float persistent tracing kernels (closed-form Kerr
// and tabulated metrics): every Dormand-Prince step in double-float (~48 bits)
// on the FP32 pipe, the state an FP32 pair; crossings refined and emission
// evaluated in FP64.
#include "tt_trace.cuh"

namespace tt {

// 256-thread blocks, registers uncapped (~180: one block per SM; a cap at 128
// spills and measured 10 % slower).
template <int METRIC, int N>
__global__ void __launch_bounds__(256) trace_kernel_df(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<METRIC, 3>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

template <int METRIC, int N>
static cudaError_t launch_df_n(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                               const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    LaunchParams<N> p;
    fill_params<N>(p, descs, n, total, sol, shape, queue);
    return launch_persistent<N>(trace_kernel_df<METRIC, N>, 256, shape.blocks_per_sm, p, stream);
}

// metric_mode 0: closed-form Kerr only, 1: tables only (a batch of both kinds
// is refused by the C ABI)
cudaError_t launch_df(const ImageDesc* descs, int n, long long total, int metric_mode, const SolverDesc& sol,
                      const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    if (shape.block == 128) return cudaErrorInvalidValue;      // not built
    if (metric_mode == 0) {
        if (n == 1) return launch_df_n<0, 1>(descs, n, total, sol, shape, queue, stream);
        return launch_df_n<0, kMaxImagesPerLaunch>(descs, n, total, sol, shape, queue, stream);
    }
    if (metric_mode == 1) {
        if (n == 1) return launch_df_n<1, 1>(descs, n, total, sol, shape, queue, stream);
        return launch_df_n<1, kMaxImagesPerLaunch>(descs, n, total, sol, shape, queue, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace tt
