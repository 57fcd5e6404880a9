// tt_kernel_split.cu -- the mixed-precision kernel with the prescribed split
// (closed-form Kerr, PREC 4): FP32 stages; FP64 state accumulation, error norm
// and step control; FP64 steps near the horizon; FP64 crossing refinement.
#include "tt_trace.cuh"

namespace tt {

// The shape of the other mixed kernels: 256-thread blocks, two per SM.
template <int N>
__global__ void __launch_bounds__(256, 2) trace_kernel_split(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<0, 4>(p.desc, p.n_desc, p.total, p.sol, p.solc, p.tune, p.queue);
}

template <int N>
static cudaError_t launch_split_n(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                                  const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    LaunchParams<N> p;
    fill_params<N>(p, descs, n, total, sol, shape, queue);
    return launch_persistent<N>(trace_kernel_split<N>, 256, shape.blocks_per_sm, p, stream);
}

cudaError_t launch_split(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                         const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    if (n == 1) return launch_split_n<1>(descs, n, total, sol, shape, queue, stream);
    return launch_split_n<kMaxImagesPerLaunch>(descs, n, total, sol, shape, queue, stream);
}

}  // namespace tt
