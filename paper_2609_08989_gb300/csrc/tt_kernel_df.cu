// tt_kernel_df.cu -- double-float persistent tracing kernels (closed-form Kerr):
// every Dormand-Prince step in double-float (~48 bits) on the FP32 pipe, the
// state an FP32 pair; crossings refined and emission evaluated in FP64.
#include "tt_trace.cuh"

namespace tt {

// 256-thread blocks, registers uncapped (~180: one block per SM; a cap at 128
// spills and measured 10 % slower).
template <int N>
__global__ void __launch_bounds__(256) trace_kernel_df(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<0, 3>(p.desc, p.n_desc, p.total, p.sol, p.tune, p.queue);
}

template <int N>
static cudaError_t launch_df_n(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                               const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    LaunchParams<N> p;
    fill_params<N>(p, descs, n, total, sol, shape, queue);
    return launch_persistent<N>(trace_kernel_df<N>, 256, shape.blocks_per_sm, p, stream);
}

cudaError_t launch_df(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                      const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    if (shape.block == 128) return cudaErrorInvalidValue;      // not built
    if (n == 1) return launch_df_n<1>(descs, n, total, sol, shape, queue, stream);
    return launch_df_n<kMaxImagesPerLaunch>(descs, n, total, sol, shape, queue, stream);
}

}  // namespace tt
