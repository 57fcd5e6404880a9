// tt_kernel_ck.cu -- FP64 tracing kernels with the Cash-Karp 5(4) pair.
#define TT_RK_METHOD 1
#include "tt_kernel_rk.cuh"
