// launch.h -- host-side launchers of the kernels in step_kernel.cuh, one explicit
// instantiation set per storage precision (launch_f32.cu, launch_f64.cu).
#pragma once

#include <cuda_runtime.h>

#include "step_kernel.cuh"

namespace kss {

// Grid of the fused step for an nx x ny lattice with tagging tile `tile`.
template <class T>
inline dim3 step_grid(int nx, int ny, int tile) {
  const int cols = 32 * Vec<T>::N;
  return dim3((unsigned)((nx + cols - 1) / cols), (unsigned)((ny + tile - 1) / tile), 1u);
}

// mode: MODE_PLAIN / MODE_STD / MODE_FULL; pull: stream first; store: collide + write.
// Valid combinations: (any mode, pull, store) for steps; (STD/FULL, pull or not, no store)
// for evaluation passes.
template <class T>
cudaError_t launch_step(const StepParams<T>& p, int mode, bool pull, bool store,
                        cudaStream_t stream);

template <class T>
cudaError_t launch_init_equilibrium(const double* rho, const double* ux, const double* uy,
                                    T* f, long long plane, int pitch, int nx, int ny,
                                    cudaStream_t stream);

template <class T>
cudaError_t launch_moments(const T* f, long long plane, int pitch, int nx, int ny, double* rho,
                           double* ux, double* uy, cudaStream_t stream);

template <class T>
cudaError_t launch_pitched_to_dense(const T* src, long long plane, int pitch, int nx, int ny,
                                    int nplanes, double* dst, cudaStream_t stream);

template <class T>
cudaError_t launch_dense_to_pitched(const double* src, long long plane, int pitch, int nx,
                                    int ny, int nplanes, T* dst, cudaStream_t stream);

}  // namespace kss
