// launch_impl.cuh -- bodies of the launchers declared in launch.h; included once per
// storage precision by launch_f32.cu / launch_f64.cu with KSS_T defined.
#pragma once

#include <atomic>

#include "launch.h"

namespace kss {

// (column blocks of 256) x (rows, strided beyond 65535) for the auxiliary kernels.
inline dim3 helper_grid(int nx, long long rows) {
  return dim3((unsigned)((nx + 255) / 256), (unsigned)(rows < 65535 ? rows : 65535));
}

// Let `kernel` take DYN bytes of dynamic shared memory on the current device (beyond the
// default 48 KB of static plus dynamic memory an opt-in is needed), once per device.
// Threads that race here at most repeat the (idempotent) attribute call.
template <auto kernel, int DYN>
cudaError_t allow_dynamic_smem() {
  if constexpr (DYN == 0) {
    return cudaSuccess;
  } else {
    constexpr int kMaxDev = 64;
    static std::atomic<bool> done[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (!done[dev].load(std::memory_order_acquire)) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DYN);
      if (e != cudaSuccess) return e;
      done[dev].store(true, std::memory_order_release);
    }
    return cudaSuccess;
  }
}

// CTAs of `kernel` (with DYN bytes of dynamic shared memory) resident on the current
// device at once (its occupancy times the SM count), looked up once per device (racing
// threads at most repeat the query).
template <auto kernel, int DYN = 0>
int resident_ctas() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev] = {};  // one per kernel: a template argument
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 0;
  int n = cache[dev].load(std::memory_order_acquire);
  if (!n) {
    int nsm = 0, per = 0;
    if (allow_dynamic_smem<kernel, DYN>() != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, DYN) != cudaSuccess)
      return 0;
    n = nsm * per;
    cache[dev].store(n, std::memory_order_release);
  }
  return n;
}

// Persistent steps: when the step grid exceeds one wave of resident CTAs, one wave that
// strides over the blocks (step_kernel_persistent).  Measured on GB300 (4096^2 / 8192^2):
// slower than one CTA per block for FP32 (fused 0.257 vs 0.243 ms, plain 0.199 vs 0.179 ms)
// and for fused FP16 deviations, faster only for plain FP16-deviation steps (0.113 vs
// 0.123 ms), so that is the one case that takes it (KSS_PERSISTENT=1 forces it everywhere).
#ifndef KSS_PERSISTENT
#define KSS_PERSISTENT 0
#endif
// Eight cells per lane for the FP16 {Kn, KL, neq} step (step_block<..., VC = 8>); 0 keeps
// four.
#ifndef KSS_F16_CELLS8
#define KSS_F16_CELLS8 1
#endif

template <int MODE>
cudaError_t launch_step_mode(const StepParams<KSS_T>& p, dim3 grid, cudaStream_t stream) {
  const int nblocks = int(grid.x * grid.y);
  constexpr bool kHalfPlain = std::is_same<KSS_T, __half>::value && MODE == MODE_PLAIN;
  if (KSS_PERSISTENT || kHalfPlain) {
    const int wave = resident_ctas<step_kernel_persistent<KSS_T, MODE, true, true>>();
    if (wave > 0 && nblocks > wave) {
      step_kernel_persistent<KSS_T, MODE, true, true><<<wave, kThreads, 0, stream>>>(
          p, int(grid.x), nblocks);
      return cudaGetLastError();
    }
  }
  if constexpr (std::is_same<KSS_T, float>::value &&
                step_prefetch_smem<KSS_T, MODE, true>() > 0) {
    // FP32 {Kn, KL, neq} with the row prefetch (KSS_F32_ONESTEP_PREFETCH)
    constexpr int dyn = step_prefetch_smem<KSS_T, MODE, true>();
    const cudaError_t e = allow_dynamic_smem<step_kernel<KSS_T, MODE, true, true, false, true>, dyn>();
    if (e != cudaSuccess) return e;
    step_kernel<KSS_T, MODE, true, true, false, true><<<grid, kThreads, dyn, stream>>>(p);
    return cudaGetLastError();
  }
  if constexpr (std::is_same<KSS_T, __half>::value && KSS_F16_PREFETCH &&
                step_prefetch_smem<KSS_T, MODE, true>() > 0) {
    // FP16 deviations, {Kn, KL, neq}: the row prefetch, with its dynamic shared memory.
    // Eight cells per lane: CTA blocks of 256 columns and at most 8 rows per warp, where
    // that grid has no more blocks than the four-cell one (whose count sized the partial
    // sums)
    if constexpr (KSS_F16_CELLS8) {
      constexpr int NW = KSS_H8_WARPS;
      dim3 g8;
      int bands8 = 0;
      if (step_grid8(p.nx, p.ny, p.tile, p.bands, NW, g8, bands8)) {
        StepParams<KSS_T> q = p;
        q.bands = bands8;
        constexpr auto kern = step_kernel<KSS_T, MODE, true, true, false, true, 8, NW>;
        constexpr int dyn8 = step_prefetch_smem<KSS_T, MODE, true, 8, NW>();
        const cudaError_t e = allow_dynamic_smem<kern, dyn8>();
        if (e != cudaSuccess) return e;
        kern<<<g8, 32 * NW, dyn8, stream>>>(q);
        return cudaGetLastError();
      }
    }
    constexpr int dyn = step_prefetch_smem<KSS_T, MODE, true>();
    const cudaError_t e = allow_dynamic_smem<step_kernel<KSS_T, MODE, true, true, false, true>, dyn>();
    if (e != cudaSuccess) return e;
    step_kernel<KSS_T, MODE, true, true, false, true><<<grid, kThreads, dyn, stream>>>(p);
    return cudaGetLastError();
  }
  step_kernel<KSS_T, MODE, true, true><<<grid, kThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <>
cudaError_t launch_step<KSS_T>(const StepParams<KSS_T>& p, int mode, bool pull, bool store,
                               cudaStream_t stream) {
  const dim3 grid = step_grid<KSS_T>(p.nx, p.ny, p.tile, p.bands);
  const dim3 block(kThreads);
  if (store && pull) {
    switch (mode) {
      case MODE_PLAIN: return launch_step_mode<MODE_PLAIN>(p, grid, stream);
      case MODE_STD: return launch_step_mode<MODE_STD>(p, grid, stream);
      case MODE_FULL: return launch_step_mode<MODE_FULL>(p, grid, stream);
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
cudaError_t launch_step_aar<KSS_T>(const StepParams<KSS_T>& p, int mode, cudaStream_t stream) {
  const dim3 grid = step_grid<KSS_T>(p.nx, p.ny, p.tile, p.bands);
  switch (mode) {
    case MODE_PLAIN: step_kernel<KSS_T, MODE_PLAIN, true, true, true><<<grid, kThreads, 0, stream>>>(p); break;
    case MODE_STD: step_kernel<KSS_T, MODE_STD, true, true, true><<<grid, kThreads, 0, stream>>>(p); break;
    case MODE_FULL: step_kernel<KSS_T, MODE_FULL, true, true, true><<<grid, kThreads, 0, stream>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <>
int multi_resident_ctas<KSS_T>(int mode, bool aar) {
  if (mode != MODE_STD) return 0;
  return aar ? resident_ctas<step_kernel_multi<KSS_T, MODE_STD, true>,
                             multi_prefetch_smem<KSS_T, MODE_STD, true>()>()
             : resident_ctas<step_kernel_multi<KSS_T, MODE_STD>,
                             multi_prefetch_smem<KSS_T, MODE_STD, false>()>();
}

template <>
cudaError_t launch_step_multi<KSS_T>(const StepParams<KSS_T>& pa, const StepParams<KSS_T>& pb,
                                     const MultiState& m, int mode, int ctas,
                                     cudaStream_t stream, bool aar) {
  StepParams<KSS_T> a = pa, b = pb;
  MultiState ms = m;
  void* args[] = {&a, &b, &ms};
  if (mode != MODE_STD) return cudaErrorInvalidValue;
  constexpr int dyn_aar = multi_prefetch_smem<KSS_T, MODE_STD, true>();
  constexpr int dyn_bgk = multi_prefetch_smem<KSS_T, MODE_STD, false>();
  const int dyn = aar ? dyn_aar : dyn_bgk;
  const cudaError_t e =
      aar ? allow_dynamic_smem<step_kernel_multi<KSS_T, MODE_STD, true>, dyn_aar>()
          : allow_dynamic_smem<step_kernel_multi<KSS_T, MODE_STD>, dyn_bgk>();
  if (e != cudaSuccess) return e;
  const void* fn = aar ? reinterpret_cast<const void*>(step_kernel_multi<KSS_T, MODE_STD, true>)
                       : reinterpret_cast<const void*>(step_kernel_multi<KSS_T, MODE_STD>);
  return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kThreads), args, dyn, stream);
}

template <>
int batch_multi_resident_ctas<KSS_T>(int mode) {
  return mode == MODE_STD ? resident_ctas<batch_kernel_multi<KSS_T, MODE_STD>,
                                         multi_prefetch_smem<KSS_T, MODE_STD, false>()>()
                          : 0;
}

template <>
cudaError_t launch_batch_multi<KSS_T>(const StepParams<KSS_T>* ta, const StepParams<KSS_T>* tb,
                                      const MultiState* mtab, const BatchItem* items,
                                      int nitems, int nsteps, uint32_t* work, int mode,
                                      int ctas, cudaStream_t stream) {
  if (mode != MODE_STD || nitems < 1 || nsteps < 1 || ctas < 1) return cudaErrorInvalidValue;
  const StepParams<KSS_T>* a = ta;
  const StepParams<KSS_T>* b = tb;
  const MultiState* m = mtab;
  const BatchItem* it = items;
  int ni = nitems, ns = nsteps;
  uint32_t* w = work;
  void* args[] = {&a, &b, &m, &it, &ni, &ns, &w};
  constexpr int dyn = multi_prefetch_smem<KSS_T, MODE_STD, false>();
  const cudaError_t e = allow_dynamic_smem<batch_kernel_multi<KSS_T, MODE_STD>, dyn>();
  if (e != cudaSuccess) return e;
  const void* fn = reinterpret_cast<const void*>(batch_kernel_multi<KSS_T, MODE_STD>);
  return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kThreads), args, dyn, stream);
}

template <>
cudaError_t launch_batch_step<KSS_T>(const StepParams<KSS_T>* table, const BatchItem* items,
                                     int nitems, int ctas, int mode, cudaStream_t stream,
                                     bool aar) {
  if (nitems < 1 || ctas < 1) return cudaErrorInvalidValue;
  const dim3 grid(unsigned(ctas < nitems ? ctas : nitems)), block(kThreads);
  if (aar) {
    switch (mode) {
      case MODE_PLAIN: batch_step_kernel<KSS_T, MODE_PLAIN, true><<<grid, block, 0, stream>>>(table, items, nitems); break;
      case MODE_STD: batch_step_kernel<KSS_T, MODE_STD, true><<<grid, block, 0, stream>>>(table, items, nitems); break;
      case MODE_FULL: batch_step_kernel<KSS_T, MODE_FULL, true><<<grid, block, 0, stream>>>(table, items, nitems); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
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
  adj_objective_kernel<KSS_T><<<adj_grid(p.nx, p.ny, p.rows), kThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <>
cudaError_t launch_adj_step<KSS_T>(const AdjParams<KSS_T>& p, cudaStream_t stream) {
  adj_step_kernel<KSS_T><<<adj_grid(p.nx, p.ny, p.rows), kThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <>
cudaError_t launch_adj_final<KSS_T>(const AdjParams<KSS_T>& p, cudaStream_t stream) {
  adj_final_kernel<KSS_T><<<adj_grid(p.nx, p.ny, p.rows), kThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <>
int adj_multi_resident_ctas<KSS_T>() {
  return resident_ctas<adj_multi_kernel<KSS_T>>();
}

template <>
cudaError_t launch_adj_multi<KSS_T>(const AdjParams<KSS_T>& base, const AdjMulti<KSS_T>& m,
                                    int ctas, double* acc, cudaStream_t stream) {
  if (ctas < 1) return cudaErrorInvalidValue;
  // a cooperative launch (all CTAs resident: the waits need it), recorded as such when the
  // stream is being captured into a graph
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, adj_multi_kernel<KSS_T>, base, m);
  if (e != cudaSuccess) return e;
  const int nit = m.last - m.s0 + 1;
  adj_iteration_totals<KSS_T><<<nit, kThreads, 0, stream>>>(m.part, m.nblocks, nit, m.totals,
                                                             m.ticket, acc);
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
  init_equilibrium_kernel<KSS_T, double><<<helper_grid(nx, ny), 256, 0, stream>>>(
      rho, ux, uy, f, plane, pitch, nx, ny, codec);
  return cudaGetLastError();
}

template <>
cudaError_t launch_init_equilibrium_f32<KSS_T>(const float* rho, const float* ux,
                                               const float* uy, KSS_T* f, long long plane,
                                               int pitch, int nx, int ny,
                                               const codec_t<KSS_T>& codec, cudaStream_t stream) {
  init_equilibrium_kernel<KSS_T, float><<<helper_grid(nx, ny), 256, 0, stream>>>(
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
