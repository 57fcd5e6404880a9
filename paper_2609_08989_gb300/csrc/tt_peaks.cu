// tt_peaks.cu -- FMA-chain probe of the FP64 and FP32 pipes (libtt_peaks.so).
//
// The tracer is bound by arithmetic, not by memory: its roofline denominators
// are the chip's FP64 and FP32 fused multiply-add rates.  This probe measures
// them: every thread runs kChains independent chains x <- x * b + c (enough
// independent work per warp to hide the pipe latency), the grid fills every SM
// several times over, and the kernel's CUDA-event time gives the rate
// (2 flops per FMA).  The chains converge to c / (1 - b) = 1, so no value
// overflows or goes subnormal; the sums are stored so nothing is optimised away.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_chain(T* out, int iters, T b, T c) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int blocks_per_sm, int iters, double* tflops, double* ms_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -3;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -3;
    const int grid = sms * blocks_per_sm, block = 256;
    T* out = nullptr;
    if (cudaMalloc((void**)&out, (size_t)grid * block * sizeof(T)) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T b = (T)0.999999, c = (T)1e-6;
    fma_chain<T><<<grid, block>>>(out, iters / 10 + 1, b, c);       // warm-up
    cudaEventRecord(e0);
    fma_chain<T><<<grid, block>>>(out, iters, b, c);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.0f) return -3;
    const double fmas = (double)grid * block * (double)iters * 16.0 * kChains;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    *ms_out = ms;
    return 0;
}

}  // namespace

extern "C" {

// Measured FMA rate of the FP64 (fp64 != 0) or FP32 pipe in TFLOP/s over one
// launch of blocks_per_sm x (SM count) blocks of 256 threads, each thread
// iters x 16 x 8 FMAs; also the launch's duration in ms.  Returns 0, or -2
// (allocation) / -3 (CUDA error).
int tt_fma_peak(int fp64, int blocks_per_sm, int iters, double* tflops, double* ms) {
    if (!tflops || !ms || blocks_per_sm < 1 || iters < 1) return -1;
    return fp64 ? run<double>(blocks_per_sm, iters, tflops, ms) : run<float>(blocks_per_sm, iters, tflops, ms);
}

}  // extern "C"
