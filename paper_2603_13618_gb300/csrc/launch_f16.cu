// launch_f16.cu -- FP16-deviation storage instantiation of the kernels and launchers
// (populations stored as __half deviation codes, FP32 arithmetic).
#define KSS_T __half
#define KSS_STORAGE_HALF 1
#include "launch_impl.cuh"
