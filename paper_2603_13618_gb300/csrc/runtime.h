// runtime.h -- internal declarations shared by the host runtime's translation units
// (kss_runtime.cu: single lattices; kss_batch.cu: batches of lattices).  Not part of
// the C ABI.
#pragma once

#include <cmath>
#include <cstdint>
#include <limits>
#include <string>
#include <type_traits>

#include "../../include/kss.h"
#include "launch.h"

// NVTX ranges around the compute entry points (kss_step, kss_batch_step, the adjoint's
// forward and backward passes, kss_regrid), named as the calls: a profiler's timeline then
// shows which call launched which kernels.  The header-only NVTX v3 API costs nothing when
// no tool is attached.  -DKSS_NVTX=0 builds without it.
#ifndef KSS_NVTX
#define KSS_NVTX 1
#endif
#if KSS_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace kss_rt {
struct NvtxRange {
#if KSS_NVTX
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
#else
  explicit NvtxRange(const char*) {}
#endif
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace kss_rt

namespace kss_rt {

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

}  // namespace kss_rt

struct kss_batch;

struct kss_lattice {
  kss_config cfg{};
  int device = 0;
  size_t esz = 0;           // bytes per stored population element
  size_t tsz = 0;           // bytes per arithmetic element (sensor planes)
  kss::codec_t<__half> codec16{};  // FP16 deviation codec (KSS_FP16DEV)
  int pitch = 0;            // row pitch in elements (multiple of 128 bytes)
  long long plane = 0;      // elements per plane
  int ntx = 0, nty = 0, nblocks = 0;
  int bands = 0;            // tile bands per CTA of the vector step (CTA height bands * tile)
  int rows_plain = 0;       // CTA height of steps without outputs (any multiple of 8)
  int nsm = 0;              // SMs of the device (persistent grid of the TMA kernel)
  void* f[2] = {nullptr, nullptr};
  void* f_alloc[2] = {nullptr, nullptr};  // the allocations behind f (a slab's start one
                                          // halo row before f)
  bool slab = false;        // a y-slab of a decomposed lattice (kss_slab_create): halo rows
                            // -1 and ny next to its own rows, no periodic wrap in y
  int cur = 0;              // f[cur] holds the stored state
  void* rec = nullptr;      // recorded sensor planes
  int rec_slot[KSS_S_COUNT];
  void* evalplane = nullptr;
  uint8_t* flags = nullptr;
  int32_t* tiles = nullptr;
  double* part_sum = nullptr;
  uint32_t* part_cnt = nullptr;
  unsigned char* small = nullptr;  // done counter + final sums + final counts
  uint32_t* done = nullptr;
  double* stat_sums = nullptr;
  unsigned long long* stat_counts = nullptr;
  uint32_t* err_word = nullptr;    // device error word (bounded waits)
  uint32_t* defer_list = nullptr;  // cells deferred by the fused pass to its fixup
  uint32_t defer_cap = 0;
  double* staging = nullptr;
  size_t staging_elems = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t step = 0;         // steps since the last set
  int64_t out_step = -1;    // step whose flags / tiles / sums are stored
  int64_t rec_step = -1;    // step whose recorded sensor planes are stored
  int64_t eval_step = -1;   // step whose evalplane holds eval_sensor
  int eval_sensor = -1;
  int err = KSS_OK;
  std::string msg;
  kss_batch* owner = nullptr;  // the batch that created this lattice, if any
  void* regrid = nullptr;      // regridding workspace (kss_regrid.cu), made on first use
  void* multi = nullptr;       // multi-step kernel bookkeeping, made on first use
  uint8_t* region = nullptr;   // two-relaxation region [ny][pitch] (cfg.tau2 > 0 only)
  void* eval_out = nullptr;    // flags, tiles, sums and counts of on-demand evaluations
                               // while the step's own outputs are current, made on first use
  // runs of single-step launches replayed as CUDA graphs (kss_runtime.cu), keyed by the
  // step count, the buffer holding the state and the phase of the output steps; recorded
  // on a stream of their own
  static constexpr int kPlainGraphs = 8;
  struct PlainGraph {
    int nsteps = 0, cur = 0;
    int64_t phase = 0;
    cudaGraphExec_t exec = nullptr;
  } plain_graphs[kPlainGraphs];
  int plain_graph_next = 0;
  cudaStream_t cap = nullptr;
};

namespace kss_rt {

inline int fail(kss_lattice* L, int code, const std::string& m) {
  if (L) {
    if (code == KSS_ERR_CUDA) L->err = code;  // sticky
    L->msg = m;
  }
  return code;
}

#define KSS_CUDA(L, call)                                                             \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail((L), KSS_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

// Largest T value <= t, so that (T)eps > result  <=>  eps > t exactly.
template <class T>
inline T round_down(double t) {
  T r = static_cast<T>(t);
  if (static_cast<double>(r) > t) r = std::nextafter(r, -std::numeric_limits<T>::infinity());
  return r;
}

inline uint32_t needed_mask(const kss_lattice* L, uint32_t extra) {
  uint32_t m = extra | (1u << L->cfg.refine_sensor);
  if (L->cfg.switch_threshold >= 0.0) m |= 1u << L->cfg.switch_sensor;
  return m;
}

// The kernel of an output step computing the sensors in mask: {Kn, KL, neq} (and qe on the
// steps of a lattice with adaptive algorithm refinement, qe_std) in the fused pair loop,
// anything else in the all-sensor kernel.
inline int mode_for(uint32_t mask, bool qe_std = false) {
  const uint32_t fused = kss::kStdMask | (qe_std ? 1u << KSS_S_QE : 0u);
  return (mask & ~fused) ? kss::MODE_FULL : kss::MODE_STD;
}

// Codec of a lattice's storage type S (empty unless S is the FP16 deviation storage).
template <class S>
inline kss::codec_t<S> codec_of(const kss_lattice* L) {
  if constexpr (std::is_same<S, __half>::value) {
    return L->codec16;
  } else {
    (void)L;
    return kss::codec_t<S>{};
  }
}

template <class S>
kss::StepParams<S> make_params(const kss_lattice* L, const void* src, void* dst) {
  using T = kss::arith_t<S>;
  kss::StepParams<S> p{};
  p.src = static_cast<const S*>(src);
  p.dst = static_cast<S*>(dst);
  p.rec = static_cast<T*>(L->rec);
  p.flags = L->flags;
  p.tiles = L->tiles;
  p.tiles_def = L->tiles + 2 * size_t(L->ntx) * L->nty;
  p.defer_list = L->defer_list;
  p.defer_count = reinterpret_cast<uint32_t*>(L->small + 208);
  p.defer_ticket = reinterpret_cast<uint32_t*>(L->small + 212);
  p.defer_cap = L->defer_cap;
  p.part_sum = L->part_sum;
  p.part_cnt = L->part_cnt;
  p.done = L->done;
  p.stat_sums = L->stat_sums;
  p.stat_counts = L->stat_counts;
  p.err = L->err_word;
  p.slab = L->slab ? 1 : 0;
  p.plane = L->plane;
  p.pitch = L->pitch;
  p.nx = L->cfg.nx;
  p.ny = L->cfg.ny;
  p.tile = L->cfg.tile;
  p.bands = L->bands;
  p.ntx = L->ntx;
  p.nty = L->nty;
  p.omega = T(1.0 / L->cfg.tau);
  p.tau = T(L->cfg.tau);
  p.thr_r = round_down<T>(L->cfg.refine_threshold);
  p.switch_on = L->cfg.switch_threshold >= 0.0;
  p.thr_s = p.switch_on ? round_down<T>(L->cfg.switch_threshold) : T(0);
  p.refine_s = L->cfg.refine_sensor;
  p.switch_s = L->cfg.switch_sensor;
  for (int s = 0; s < KSS_S_COUNT; ++s) p.rec_slot[s] = L->rec_slot[s];
  p.codec = codec_of<S>(L);
  p.region = L->region;
  if (L->cfg.tau2 > 0.0) {
    const double w1 = 1.0 / L->cfg.tau, w2 = 1.0 / L->cfg.tau2;
    p.trt.a = T(0.5 * (w1 + w2));
    p.trt.b = T(0.5 * (w1 - w2));
    p.trt.qe = true;
  }
  return p;
}

// Storage type of a precision, as a tag for generic lambdas: with_storage(prec, f) calls
// f(Tag<S>{}) with S = float, double or __half.
template <class S>
struct Tag {
  using type = S;
};
template <class F>
inline auto with_storage(int precision, F&& f) {
  if (precision == KSS_FP64) return f(Tag<double>{});
  if (precision == KSS_FP16DEV) return f(Tag<__half>{});
  return f(Tag<float>{});
}

// Device allocations of the library's host runtimes go through these two calls: they
// count the live allocations and, for tests, can be made to fail (kss_testing_fail_after:
// the n-th allocation or launch from now reports an error without touching the GPU).
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}
cudaError_t dev_free(void* p);
// Launch injection point: cudaErrorLaunchFailure when an armed launch failure is due.
cudaError_t injected_launch_error();

// Sticky error of a lattice, if any (KSS_ERR_ARG for NULL).
inline int enter(kss_lattice* L) {
  if (!L) return KSS_ERR_ARG;
  if (L->err) return L->err;
  return KSS_OK;
}

// Free a lattice's device buffers and stream after its stream drains (kss_runtime.cu).
void release(kss_lattice* L);

// After a stream synchronisation: did a bounded device wait run out?  (sticky)
int device_error(kss_lattice* L);

// Free a lattice's regridding workspace, if any (kss_regrid.cu).
void regrid_release(kss_lattice* L);

}  // namespace kss_rt
