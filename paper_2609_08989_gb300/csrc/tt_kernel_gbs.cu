// tt_kernel_gbs.cu -- FP64 tracing kernels with the Gragg-Bulirsch-Stoer extrapolator.
#define TT_RK_METHOD 3
#include "tt_kernel_rk.cuh"
