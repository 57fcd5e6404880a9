// tt_kernel_mixed.cu -- mixed-precision persistent tracing kernels
// (closed-form Kerr; PREC 1: FP64 state accumulation, PREC 2: FP32 pair).  Their
// steps near the horizon and the axis run in double-float; the prescribed split
// (PREC 4) is built in tt_kernel_split.cu.
#include "tt_trace.cuh"

namespace tt {

// 256-thread blocks, two per SM (128 registers: a few spills, but twice the
// warps of the uncapped 190-register build, measured 14 % faster).
template <int PREC, int N>
__global__ void __launch_bounds__(256, 2) trace_kernel_mixed(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<0, PREC>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

template <int N>
static cudaError_t launch_mixed_n(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                                  const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    LaunchParams<N> p;
    fill_params<N>(p, descs, n, total, sol, shape, queue);
    if (sol.precision == 2)
        return launch_persistent<N>(trace_kernel_mixed<2, N>, 256, shape.blocks_per_sm, p, stream);
    return launch_persistent<N>(trace_kernel_mixed<1, N>, 256, shape.blocks_per_sm, p, stream);
}

cudaError_t launch_mixed(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                         const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    if (shape.block == 128) return cudaErrorInvalidValue;      // spills: not built
    if (sol.precision == 4) return launch_split(descs, n, total, sol, shape, queue, stream);
    if (n == 1) return launch_mixed_n<1>(descs, n, total, sol, shape, queue, stream);
    return launch_mixed_n<kMaxImagesPerLaunch>(descs, n, total, sol, shape, queue, stream);
}

}  // namespace tt
