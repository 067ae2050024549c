// launch_f64.cu -- FP64-storage instantiation of the kernels and launchers.
#define KSS_T double
#include "launch_impl.cuh"
