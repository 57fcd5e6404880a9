// tt_kernel_verlet.cu -- FP64 tracing kernels with the Stormer-Verlet scheme.
#define TT_RK_METHOD 4
#include "tt_kernel_rk.cuh"
