// launch.h -- host-side launchers of the kernels in step_kernel.cuh, one explicit
// instantiation set per storage type (launch_f32.cu, launch_f64.cu, launch_f16.cu; the
// TMA, fixup, adjoint and plain-plane launchers exist for float and double only).
#pragma once

#include <cuda_runtime.h>

#include "adjoint_kernel.cuh"
#include "step_tma.cuh"

namespace kss {

// Grid of the fused step for an nx x ny lattice with tagging tile `tile` and
// `bands` tile bands per CTA (0: the default, step_bands(tile)).
template <class T>
inline dim3 step_grid(int nx, int ny, int tile, int bands = 0) {
  const int cols = 32 * Vec<T>::N;
  const int rows = tile * (bands > 0 ? bands : step_bands(tile));
  return dim3((unsigned)((nx + cols - 1) / cols), (unsigned)((ny + rows - 1) / rows), 1u);
}

// Grid g of the FP16 {Kn, KL, neq} step with eight cells per lane (CTA blocks of 256
// columns and at most 8 rows per warp of nw warps) for a lattice whose four-cell grid has
// `bands` tile bands per CTA, and its bands per CTA; false where its rows are not whole
// tiles or it would have more blocks than the four-cell grid (whose count sized the
// partial sums).
inline bool step_grid8(int nx, int ny, int tile, int bands, int nw, dim3& g, int& bands8) {
  const int rows = tile * bands, rows8 = rows < 8 * nw ? rows : 8 * nw;
  const dim3 g4 = step_grid<__half>(nx, ny, tile, bands);
  g = dim3(unsigned((nx + 255) / 256), unsigned((ny + rows8 - 1) / rows8), 1u);
  bands8 = rows8 / tile;
  return rows8 % tile == 0 && (long long)g.x * g.y <= (long long)g4.x * g4.y;
}

// mode: MODE_PLAIN / MODE_STD / MODE_FULL; pull: stream first; store: collide + write.
// Valid combinations: (any mode, pull, store) for steps; (STD/FULL, pull or not, no store)
// for evaluation passes.
template <class T>
cudaError_t launch_step(const StepParams<T>& p, int mode, bool pull, bool store,
                        cudaStream_t stream);

// One step with adaptive algorithm refinement: the two-relaxation collision in the
// region p.region (output steps rewrite it); mode as launch_step, always pull + store.
template <class T>
cudaError_t launch_step_aar(const StepParams<T>& p, int mode, cudaStream_t stream);

// One batched step (batch_step_kernel): `table` holds one StepParams per lattice
// (grid_x, nblocks and bands set), `items` the nitems CTA blocks; `ctas` CTAs (<= nitems)
// stride over the items.  mode MODE_PLAIN / MODE_STD / MODE_FULL; always pull + store.
template <class T>
cudaError_t launch_batch_step(const StepParams<T>* table, const BatchItem* items, int nitems,
                              int ctas, int mode, cudaStream_t stream, bool aar = false);

// nsteps batched steps in one cooperative launch (batch_kernel_multi): ta / tb are the
// parameter tables of even / odd steps, mtab each lattice's MultiState, work the shared
// work counter (0 at launch); mode MODE_STD; ctas <= batch_multi_resident_ctas.
template <class T>
cudaError_t launch_batch_multi(const StepParams<T>* ta, const StepParams<T>* tb,
                               const MultiState* mtab, const BatchItem* items, int nitems,
                               int nsteps, uint32_t* work, int mode, int ctas,
                               cudaStream_t stream);
template <class T>
int batch_multi_resident_ctas(int mode);

// nsteps fused steps in one cooperative launch (step_kernel_multi): pa reads buffer A and
// writes B, pb the reverse; mode MODE_STD (the {Kn, KL, neq} set every step);
// ctas <= multi_resident_ctas.
template <class T>
cudaError_t launch_step_multi(const StepParams<T>& pa, const StepParams<T>& pb,
                              const MultiState& m, int mode, int ctas, cudaStream_t stream,
                              bool aar = false);
// CTAs of the multi-step kernel resident on the current device at once (0 on error).
template <class T>
int multi_resident_ctas(int mode, bool aar = false);

// The TMA-staged step (step_tma.cuh): mode MODE_PLAIN or MODE_STD, always pull + store;
// `ctas` persistent CTAs (one per SM).
template <class T>
cudaError_t launch_step_tma(const StepParams<T>& p, int mode, TmaPlan plan, int ctas,
                            cudaStream_t stream);

// fixup_kernel after a MODE_STD pass (step or evaluation; `pull` as that pass), with
// `ctas` CTAs of 256 threads striding over the tiles.
template <class T>
cudaError_t launch_fixup(const StepParams<T>& p, bool pull, int ctas, cudaStream_t stream);

// Rows per CTA (32, 16 or 8) for CTAs `cols` columns wide: the tallest that still gives
// at least two CTAs per SM, else 8.  Steps without outputs and the adjoint kernels use it
// (their results do not depend on the CTA shape, or are reduced in a fixed order).
inline int fill_rows(int nx, int ny, int cols, int nsm) {
  const long long gx = (nx + cols - 1) / cols;
  for (int r = 32; r >= 16; r /= 2)
    if (gx * ((ny + r - 1) / r) >= 2LL * nsm) return r;
  return 8;
}

// Adjoint kernels (adjoint_kernel.cuh) on the grid adj_grid(nx, ny, rows).
inline dim3 adj_grid(int nx, int ny, int rows = kAdjRows) {
  return dim3((unsigned)((nx + 32 * kAdjV - 1) / (32 * kAdjV)),
              (unsigned)((ny + rows - 1) / rows), 1u);
}
template <class T>
cudaError_t launch_adj_objective(const AdjParams<T>& p, cudaStream_t stream);
template <class T>
cudaError_t launch_adj_step(const AdjParams<T>& p, cudaStream_t stream);
template <class T>
cudaError_t launch_adj_final(const AdjParams<T>& p, cudaStream_t stream);
// The reverse sweep of one segment in one cooperative launch of `ctas` persistent CTAs
// (adj_multi_kernel), then its iteration totals added to *acc in order; and the CTAs of
// that kernel the device holds at once.
template <class T>
cudaError_t launch_adj_multi(const AdjParams<T>& base, const AdjMulti<T>& m, int ctas,
                             double* acc, cudaStream_t stream);
template <class T>
int adj_multi_resident_ctas();

// Population conversions for any storage S (float, double, __half deviations); the
// codec is that of the lattice (empty for float and double).
template <class S>
cudaError_t launch_init_equilibrium(const double* rho, const double* ux, const double* uy,
                                    S* f, long long plane, int pitch, int nx, int ny,
                                    const codec_t<S>& codec, cudaStream_t stream);
template <class S>
cudaError_t launch_init_equilibrium_f32(const float* rho, const float* ux, const float* uy,
                                        S* f, long long plane, int pitch, int nx, int ny,
                                        const codec_t<S>& codec, cudaStream_t stream);

template <class S>
cudaError_t launch_moments(const S* f, long long plane, int pitch, int nx, int ny, double* rho,
                           double* ux, double* uy, const codec_t<S>& codec, cudaStream_t stream);

template <class S>
cudaError_t launch_pops_to_dense(const S* src, long long plane, int pitch, int nx, int ny,
                                 double* dst, const codec_t<S>& codec, cudaStream_t stream);

template <class S>
cudaError_t launch_dense_to_pops(const double* src, long long plane, int pitch, int nx, int ny,
                                 S* dst, const codec_t<S>& codec, cudaStream_t stream);

// Plain pitched planes of an arithmetic type T (float, double): sensor fields, weights.
template <class T>
cudaError_t launch_pitched_to_dense(const T* src, long long plane, int pitch, int nx, int ny,
                                    int nplanes, double* dst, cudaStream_t stream);

template <class T>
cudaError_t launch_dense_to_pitched(const double* src, long long plane, int pitch, int nx,
                                    int ny, int nplanes, T* dst, cudaStream_t stream);

}  // namespace kss
