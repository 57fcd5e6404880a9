// tt_kernel_f.cu -- FP64 tracing kernels with the Fehlberg 5(4) pair.
#define TT_RK_METHOD 2
#include "tt_kernel_rk.cuh"
