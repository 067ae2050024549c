// launch_impl.cuh -- bodies of the launchers declared in launch.h; included once per
// storage precision by launch_f32.cu / launch_f64.cu with KSS_T defined.
#pragma once

#include "launch.h"

namespace kss {

// (column blocks of 256) x (rows, strided beyond 65535) for the auxiliary kernels.
inline dim3 helper_grid(int nx, long long rows) {
  return dim3((unsigned)((nx + 255) / 256), (unsigned)(rows < 65535 ? rows : 65535));
}

template <>
cudaError_t launch_step<KSS_T>(const StepParams<KSS_T>& p, int mode, bool pull, bool store,
                               cudaStream_t stream) {
  const dim3 grid = step_grid<KSS_T>(p.nx, p.ny, p.tile);
  const dim3 block(kThreads);
  if (store && pull) {
    switch (mode) {
      case MODE_PLAIN: step_kernel<KSS_T, MODE_PLAIN, true, true><<<grid, block, 0, stream>>>(p); break;
      case MODE_STD: step_kernel<KSS_T, MODE_STD, true, true><<<grid, block, 0, stream>>>(p); break;
      case MODE_FULL: step_kernel<KSS_T, MODE_FULL, true, true><<<grid, block, 0, stream>>>(p); break;
      default: return cudaErrorInvalidValue;
    }
  } else if (!store) {
    if (mode == MODE_STD && pull) step_kernel<KSS_T, MODE_STD, true, false><<<grid, block, 0, stream>>>(p);
    else if (mode == MODE_STD) step_kernel<KSS_T, MODE_STD, false, false><<<grid, block, 0, stream>>>(p);
    else if (mode == MODE_FULL && pull) step_kernel<KSS_T, MODE_FULL, true, false><<<grid, block, 0, stream>>>(p);
    else if (mode == MODE_FULL) step_kernel<KSS_T, MODE_FULL, false, false><<<grid, block, 0, stream>>>(p);
    else return cudaErrorInvalidValue;
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <>
cudaError_t launch_batch_step<KSS_T>(const StepParams<KSS_T>* table, const BatchItem* items,
                                     int nitems, int ctas, int mode, cudaStream_t stream) {
  if (nitems < 1 || ctas < 1) return cudaErrorInvalidValue;
  const dim3 grid(unsigned(ctas < nitems ? ctas : nitems)), block(kThreads);
  switch (mode) {
    case MODE_PLAIN: batch_step_kernel<KSS_T, MODE_PLAIN><<<grid, block, 0, stream>>>(table, items, nitems); break;
    case MODE_STD: batch_step_kernel<KSS_T, MODE_STD><<<grid, block, 0, stream>>>(table, items, nitems); break;
    case MODE_FULL: batch_step_kernel<KSS_T, MODE_FULL><<<grid, block, 0, stream>>>(table, items, nitems); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#ifndef KSS_STORAGE_HALF
template <>
cudaError_t launch_adj_objective<KSS_T>(const AdjParams<KSS_T>& p, cudaStream_t stream) {
  adj_objective_kernel<KSS_T><<<adj_grid(p.nx, p.ny), kThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <>
cudaError_t launch_adj_step<KSS_T>(const AdjParams<KSS_T>& p, cudaStream_t stream) {
  adj_step_kernel<KSS_T><<<adj_grid(p.nx, p.ny), kThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <>
cudaError_t launch_adj_final<KSS_T>(const AdjParams<KSS_T>& p, cudaStream_t stream) {
  adj_final_kernel<KSS_T><<<adj_grid(p.nx, p.ny), kThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_tma_mode(const StepParams<KSS_T>& p, TmaPlan plan, int ctas,
                            cudaStream_t stream) {
  static bool configured = false;  // the dynamic shared-memory opt-in, once per process
  if (!configured) {
    const cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<KSS_T, MODE>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(kTmaSmemBytes));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  step_tma_kernel<KSS_T, MODE><<<ctas, kTmaThreads, kTmaSmemBytes, stream>>>(p, plan);
  return cudaGetLastError();
}

template <>
cudaError_t launch_step_tma<KSS_T>(const StepParams<KSS_T>& p, int mode, TmaPlan plan, int ctas,
                                   cudaStream_t stream) {
  switch (mode) {
    case MODE_PLAIN: return launch_tma_mode<MODE_PLAIN>(p, plan, ctas, stream);
    case MODE_STD: return launch_tma_mode<MODE_STD>(p, plan, ctas, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_fixup<KSS_T>(const StepParams<KSS_T>& p, bool pull, int ctas,
                                cudaStream_t stream) {
  if (pull)
    fixup_kernel<KSS_T, true><<<ctas, 256, 0, stream>>>(p);
  else
    fixup_kernel<KSS_T, false><<<ctas, 256, 0, stream>>>(p);
  return cudaGetLastError();
}

#endif  // KSS_STORAGE_HALF

template <>
cudaError_t launch_init_equilibrium<KSS_T>(const double* rho, const double* ux, const double* uy,
                                           KSS_T* f, long long plane, int pitch, int nx, int ny,
                                           const codec_t<KSS_T>& codec, cudaStream_t stream) {
  init_equilibrium_kernel<KSS_T><<<helper_grid(nx, ny), 256, 0, stream>>>(
      rho, ux, uy, f, plane, pitch, nx, ny, codec);
  return cudaGetLastError();
}

template <>
cudaError_t launch_moments<KSS_T>(const KSS_T* f, long long plane, int pitch, int nx, int ny,
                                  double* rho, double* ux, double* uy,
                                  const codec_t<KSS_T>& codec, cudaStream_t stream) {
  moments_kernel<KSS_T><<<helper_grid(nx, ny), 256, 0, stream>>>(
      f, plane, pitch, nx, ny, rho, ux, uy, codec);
  return cudaGetLastError();
}

template <>
cudaError_t launch_pops_to_dense<KSS_T>(const KSS_T* src, long long plane, int pitch, int nx,
                                        int ny, double* dst, const codec_t<KSS_T>& codec,
                                        cudaStream_t stream) {
  pops_to_dense_kernel<KSS_T><<<helper_grid(nx, ny), 256, 0, stream>>>(
      src, plane, pitch, nx, ny, dst, codec);
  return cudaGetLastError();
}

template <>
cudaError_t launch_dense_to_pops<KSS_T>(const double* src, long long plane, int pitch, int nx,
                                        int ny, KSS_T* dst, const codec_t<KSS_T>& codec,
                                        cudaStream_t stream) {
  dense_to_pops_kernel<KSS_T><<<helper_grid(nx, ny), 256, 0, stream>>>(
      src, plane, pitch, nx, ny, dst, codec);
  return cudaGetLastError();
}

#ifndef KSS_STORAGE_HALF
template <>
cudaError_t launch_pitched_to_dense<KSS_T>(const KSS_T* src, long long plane, int pitch, int nx,
                                           int ny, int nplanes, double* dst, cudaStream_t stream) {
  pitched_to_dense_kernel<KSS_T><<<helper_grid(nx, ny), 256, 0, stream>>>(
      src, plane, pitch, nx, ny, nplanes, dst);
  return cudaGetLastError();
}

template <>
cudaError_t launch_dense_to_pitched<KSS_T>(const double* src, long long plane, int pitch, int nx,
                                           int ny, int nplanes, KSS_T* dst, cudaStream_t stream) {
  dense_to_pitched_kernel<KSS_T><<<helper_grid(nx, ny), 256, 0, stream>>>(
      src, plane, pitch, nx, ny, nplanes, dst);
  return cudaGetLastError();
}
#endif  // KSS_STORAGE_HALF

}  // namespace kss
