// launch_f32.cu -- FP32-storage instantiation of the kernels and launchers.
#define KSS_T float
#include "launch_impl.cuh"
