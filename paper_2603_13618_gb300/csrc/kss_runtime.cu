// kss_runtime.cu -- host runtime behind the C ABI of include/kss.h: owns each
// lattice's device buffers and stream, sequences the fused-step launches, keeps
// track of which outputs describe which step, and moves data across the boundary.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <numeric>
#include <string>

#include <atomic>
#include <mutex>

#include "runtime.h"
#include "step_tma.cuh"

using namespace kss_rt;

namespace {

using kss::MODE_FULL;
using kss::MODE_PLAIN;
using kss::MODE_STD;

constexpr int kVersion = 100;  // 0.1.0

bool valid_sensor(int s) { return s >= 0 && s < KSS_S_COUNT; }

int check_config(const kss_config* c) {
  if (!c) return KSS_ERR_ARG;
  if (c->nx < 1 || c->ny < 1) return KSS_ERR_ARG;
  if ((long long)c->nx * c->ny > std::numeric_limits<int>::max()) return KSS_ERR_ARG;
  if (c->precision != KSS_FP64 && c->precision != KSS_FP32 && c->precision != KSS_FP16DEV)
    return KSS_ERR_UNSUPPORTED;
  if (c->precision == KSS_FP16DEV) {
    if (!(c->rho0 > 0.0) || !std::isfinite(c->rho0)) return KSS_ERR_ARG;
    if (c->dev_exp < -24 || c->dev_exp > 40) return KSS_ERR_ARG;
    if (c->dev_unscaled != 0 && c->dev_unscaled != 1) return KSS_ERR_ARG;
  }
  if (!(c->tau > 0.5) || !std::isfinite(c->tau)) return KSS_ERR_ARG;
  if (c->tau2 != 0.0 && (!(c->tau2 > 0.5) || !std::isfinite(c->tau2))) return KSS_ERR_ARG;
  if (!valid_sensor(c->refine_sensor) || !valid_sensor(c->switch_sensor)) return KSS_ERR_ARG;
  if (std::isnan(c->refine_threshold) || std::isnan(c->switch_threshold)) return KSS_ERR_ARG;
  if (c->record_mask >> KSS_S_COUNT) return KSS_ERR_ARG;
  if (c->output_every < 0) return KSS_ERR_ARG;
  if (c->tile != 8 && c->tile != 16 && c->tile != 32 && c->tile != 64) return KSS_ERR_ARG;
  if (c->own_stream != 0 && c->own_stream != 1) return KSS_ERR_ARG;
  if (c->kernel < KSS_KERNEL_AUTO || c->kernel > KSS_KERNEL_TMA) return KSS_ERR_ARG;
  return KSS_OK;
}

// The automatic choice is the vector kernel: on GB300 it is faster than the TMA-staged
// one at every size measured (plain steps 0.179 vs 0.209 ms, sensor steps 0.25 vs
// 0.28 ms at 4096^2 FP32); the TMA kernel is used only when asked for.
bool use_tma(const kss_lattice* L, int mode) {
  return mode != MODE_FULL && L->cfg.kernel == KSS_KERNEL_TMA && !L->slab;
}

// CTAs of the fixup pass (2 per SM, grid-striding over the deferred cells).
int fixup_ctas(const kss_lattice* L) { return 2 * L->nsm; }

template <class S>
cudaError_t launch_one_step(kss_lattice* L, bool out) {
  kss::StepParams<S> p = make_params<S>(L, L->f[L->cur], L->f[L->cur ^ 1]);
  const int mode = out ? mode_for(needed_mask(L, L->cfg.record_mask), L->region != nullptr)
                       : MODE_PLAIN;
  if (mode == MODE_PLAIN) {  // the tile only shapes the grid of a step without outputs
    p.tile = 8;
    p.bands = L->rows_plain / 8;
  }
  if (L->region) return kss::launch_step_aar<S>(p, mode, L->stream);
  // (the vector kernel recomputes its deferred cells itself, at the end of each CTA; FP16
  // deviation storage has the vector kernel only)
  if constexpr (std::is_same<S, __half>::value) {
    return kss::launch_step<S>(p, mode, true, true, L->stream);
  } else {
    if (!use_tma(L, mode)) return kss::launch_step<S>(p, mode, true, true, L->stream);
  // persistent grid: one CTA (two warp groups) per SM; the groups on a strip split
  // its rows evenly, at least 4 rows per run
  kss::TmaPlan plan;
  const int width = kss::kGroupWarps * 32 * kss::Vec<S>::N;
  plan.strips = (L->cfg.nx + width - 1) / width;
  const int groups = L->nsm * kss::kTmaGroups;
  const int by_groups = groups / plan.strips;
  const int by_rows = (L->cfg.ny + 3) / 4;
  plan.chunks = std::max(1, std::min(by_groups, by_rows));
  if (out) {
    // the TMA kernel adds tile counts with atomics
    const cudaError_t e = cudaMemsetAsync(L->tiles, 0, sizeof(int32_t) * 3 * size_t(L->ntx) * L->nty,
                                          L->stream);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = kss::launch_step_tma<S>(p, mode, plan, L->nsm, L->stream);
  if (e != cudaSuccess || mode != MODE_STD) return e;
  return kss::launch_fixup<S>(p, true, fixup_ctas(L), L->stream);
  }
}

// Multi-step launches (KSS_MULTISTEP, default on): kss_step(n >= 2) with every step an
// output step of the {Kn, KL, neq} set runs as one cooperative launch of
// step_kernel_multi (the kernel also takes plain steps).
#ifndef KSS_MULTISTEP
#define KSS_MULTISTEP 1
#endif

// FP16-deviation lattices in multi-step launches too (KSS_MULTISTEP_F16).
#ifndef KSS_MULTISTEP_F16
#define KSS_MULTISTEP_F16 0
#endif

constexpr int kMultiRing = 8;  // partial-sum slots of the multi-step kernel

// Runs of single-step launches as replayed CUDA graphs (KSS_STEP_GRAPHS, default on), of
// at most kGraphChunk steps each.
#ifndef KSS_STEP_GRAPHS
#define KSS_STEP_GRAPHS 1
#endif
constexpr int32_t kGraphChunk = 512;

int multi_workspace(kss_lattice* L) {
  if (L->multi) return KSS_OK;
  const size_t nb = size_t(L->nblocks), R = kMultiRing;
  const size_t bytes = sizeof(uint32_t) * (nb + 2 * R + 1) + 256 +  // done, ticket, fin, work
                       sizeof(double) * R * nb * 3 + sizeof(uint32_t) * R * nb * 4 +  // partials
                       (sizeof(double) + sizeof(unsigned long long)) * R * 3;        // step sums
  if (kss_rt::dev_malloc(&L->multi, bytes) != cudaSuccess) {
    cudaGetLastError();
    L->multi = nullptr;
    return fail(L, KSS_ERR_OOM, "multi-step workspace");
  }
  return KSS_OK;
}

template <class S>
cudaError_t launch_multi(kss_lattice* L, int mode, int nsteps) {
  if (multi_workspace(L)) return cudaErrorMemoryAllocation;
  const int nb = L->nblocks, R = kMultiRing;
  unsigned char* w = static_cast<unsigned char*>(L->multi);
  kss::MultiState m{};
  m.done = reinterpret_cast<uint32_t*>(w);
  m.ticket = m.done + nb;
  m.fin = m.ticket + R;
  m.work = m.fin + R;
  const size_t head = sizeof(uint32_t) * (size_t(nb) + 2 * R + 1);
  unsigned char* q = w + (head + 255) / 256 * 256;
  m.part_sum = reinterpret_cast<double*>(q);
  m.part_cnt = reinterpret_cast<uint32_t*>(q + sizeof(double) * size_t(R) * nb * 3);
  m.ring_sums = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(m.part_cnt) +
                                          sizeof(uint32_t) * size_t(R) * nb * 4);
  m.ring_counts = reinterpret_cast<unsigned long long*>(m.ring_sums + 3 * R);
  m.err = L->err_word;
  m.deadline = 4000000000LL;  // clock64 cycles, about 2 s at 2 GHz
  m.ring = R;
  m.nsteps = nsteps;
  const dim3 g = kss::step_grid<S>(L->cfg.nx, L->cfg.ny, L->cfg.tile, L->bands);
  m.gx = int(g.x);
  m.gy = int(g.y);
  m.nblocks = nb;
  const bool aar = L->region != nullptr;
  const int resident = kss::multi_resident_ctas<S>(mode, aar);
  if (resident < 1) return cudaErrorInvalidConfiguration;
  // as many CTAs as keep the blocks per CTA even
  const int per = (nb + resident - 1) / resident;
  const int ctas = (nb + per - 1) / per;
  cudaError_t e = cudaMemsetAsync(w, 0, head, L->stream);
  if (e != cudaSuccess) return e;
  const kss::StepParams<S> pa = make_params<S>(L, L->f[L->cur], L->f[L->cur ^ 1]);
  const kss::StepParams<S> pb = make_params<S>(L, L->f[L->cur ^ 1], L->f[L->cur]);
  return kss::launch_step_multi<S>(pa, pb, m, mode, ctas, L->stream, aar);
}

// Scratch outputs of an evaluation that only a sensor field is wanted from: flags
// [ny][pitch], tile counts [3][nty][ntx], then sums and counts.
size_t eval_out_tiles(const kss_lattice* L) { return (size_t(L->pitch) * L->cfg.ny + 255) / 256 * 256; }
size_t eval_out_small(const kss_lattice* L) {
  return eval_out_tiles(L) + (sizeof(int32_t) * 3 * size_t(L->ntx) * L->nty + 255) / 256 * 256;
}

int ensure_eval_out(kss_lattice* L) {
  if (L->eval_out) return KSS_OK;
  if (kss_rt::dev_malloc(&L->eval_out, eval_out_small(L) + 256) != cudaSuccess) {
    cudaGetLastError();
    L->eval_out = nullptr;
    return fail(L, KSS_ERR_OOM, "evaluation scratch allocation failed");
  }
  return KSS_OK;
}

// Evaluate sensors / flags / tiles / sums of the state of the most recent step
// (its pre-collision populations: the other buffer, streamed) or of the stored
// state when no step was taken since the last set.  sensor >= 0 also writes
// that sensor's field into evalplane.  keep: the lattice's flags, tiles, sums and counts
// already describe that state, so the pass writes its own into scratch (an all-sensor
// pass sums in another order than the step did, and its KL series is another one).
template <class S>
cudaError_t launch_eval(kss_lattice* L, int sensor, bool keep) {
  const bool pull = L->step > 0;
  const void* src = pull ? L->f[L->cur ^ 1] : L->f[L->cur];
  kss::StepParams<S> p = make_params<S>(L, src, nullptr);
  if (keep) {
    unsigned char* o = static_cast<unsigned char*>(L->eval_out);
    p.flags = o;
    p.tiles = reinterpret_cast<int32_t*>(o + eval_out_tiles(L));
    p.tiles_def = p.tiles + 2 * size_t(L->ntx) * L->nty;
    p.stat_sums = reinterpret_cast<double*>(o + eval_out_small(L));
    p.stat_counts = reinterpret_cast<unsigned long long*>(o + eval_out_small(L) + 64);
  }
  for (int s = 0; s < KSS_S_COUNT; ++s) p.rec_slot[s] = -1;
  uint32_t extra = 0;
  if (sensor >= 0) {
    p.rec = static_cast<kss::arith_t<S>*>(L->evalplane);
    p.rec_slot[sensor] = 0;
    extra = 1u << sensor;
  }
  return kss::launch_step<S>(p, mode_for(needed_mask(L, extra)), pull, false, L->stream);
}

// A device word that nothing ever writes: the bounded wait of kss_testing_expire_wait
// waits on it.
__device__ uint32_t g_never_set = 0u;

// One thread waits, with the multi-step kernels' own bounded wait, for g_never_set to reach
// 1; after `deadline` cycles the wait gives up and sets bit 1 of the lattice's error word.
__global__ void expire_wait_kernel(uint32_t* err, long long deadline) {
  kss::MultiState m{};
  m.err = err;
  m.deadline = deadline;
  kss::wait_at_least(m, &g_never_set, 1u);
}

// The TMA kernel's bounded mbarrier wait, on a barrier whose phase never completes (two
// arrivals expected, one made; no copy is ever issued to it): after `deadline` cycles the
// wait gives up and sets bit 0 of the error word, as the TMA kernel does.
__global__ void expire_mbarrier_kernel(uint32_t* err, long long deadline) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    kss::mbar_init(&bar, 2);
    kss::fence_mbarrier_init();
    kss::mbar_arrive(&bar);
    if (!kss::mbar_wait_bounded(&bar, 0u, deadline)) atomicOr(err, 1u);
  }
}

// Region bytes as the kernels write them: 1 for a switched cell, 0 otherwise.
__global__ void region_to_01_kernel(uint8_t* r, int pitch, int nx, int ny) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < ny; j += gridDim.y) {
    if (i < nx) {
      uint8_t* c = r + (long long)j * pitch + i;
      *c = *c != 0;
    }
  }
}

// The device address of page-locked host memory (cudaHostAlloc / cudaHostRegister), which
// kernels read directly over the host link, or nullptr for pageable memory.  Reading pinned
// inputs in the consuming kernel skips the staging copy's round trip through HBM (4096^2
// fields: 1.91 instead of 2.08 ms, both bound by the ~210 GB/s host link).
template <class E>
const E* pinned_device_view(const E* host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<const E*>(a.devicePointer);
}

// Is step n (counted from the last set) an output step?
bool is_output_step(const kss_lattice* L, int64_t n) {
  return L->cfg.output_every > 0 && n % L->cfg.output_every == 0;
}

// The next nsteps >= 2 steps from buffer L->cur, one launch each, as one replayed CUDA
// graph: a small lattice's steps are a few microseconds each, about the launch overhead.
// The graph is recorded on the lattice's capture stream the first time a (step count,
// buffer, output phase) triple comes up and replayed on its stream afterwards.
int steps_graph(kss_lattice* L, int nsteps) {
  const int64_t phase = L->cfg.output_every > 0 ? L->step % L->cfg.output_every : 0;
  for (const auto& g : L->plain_graphs) {
    if (g.exec && g.nsteps == nsteps && g.cur == L->cur && g.phase == phase) {
      KSS_CUDA(L, cudaGraphLaunch(g.exec, L->stream));
      return KSS_OK;
    }
  }
  if (!L->cap) KSS_CUDA(L, cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking));
  KSS_CUDA(L, cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal));
  const cudaStream_t keep = L->stream;
  const int cur0 = L->cur;
  L->stream = L->cap;
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < nsteps && le == cudaSuccess; ++s) {
    const bool out = is_output_step(L, L->step + s + 1);
    le = with_storage(L->cfg.precision, [&](auto tag) {
      return launch_one_step<typename decltype(tag)::type>(L, out);
    });
    L->cur ^= 1;
  }
  L->stream = keep;
  L->cur = cur0;
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(L->cap, &graph);
  if (le != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return fail(L, KSS_ERR_CUDA, std::string("graph capture: ") +
                                     cudaGetErrorString(le != cudaSuccess ? le : ee));
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  KSS_CUDA(L, ie);
  auto& slot = L->plain_graphs[L->plain_graph_next];
  L->plain_graph_next = (L->plain_graph_next + 1) % kss_lattice::kPlainGraphs;
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot.nsteps = nsteps;
  slot.cur = L->cur;
  slot.phase = phase;
  slot.exec = exec;
  KSS_CUDA(L, cudaGraphLaunch(exec, L->stream));
  return KSS_OK;
}

int ensure_staging(kss_lattice* L, size_t elems) {
  if (L->staging_elems >= elems) return KSS_OK;
  if (L->staging) {
    KSS_CUDA(L, cudaStreamSynchronize(L->stream));
    kss_rt::dev_free(L->staging);
    L->staging = nullptr;
    L->staging_elems = 0;
  }
  void* p = nullptr;
  if (kss_rt::dev_malloc(&p, elems * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(L, KSS_ERR_OOM, "staging allocation failed");
  }
  L->staging = static_cast<double*>(p);
  L->staging_elems = elems;
  return KSS_OK;
}

// Make flags / tiles / sums (and, if sensor >= 0, that sensor's field) describe
// the current step.  Returns where the sensor field is (rec slot or evalplane).
int ensure_outputs(kss_lattice* L, int sensor, const void** field) {
  const bool have_out = L->out_step == L->step;
  const void* where = nullptr;
  if (sensor >= 0) {
    if (L->rec_step == L->step && L->rec_slot[sensor] >= 0)
      where = static_cast<const char*>(L->rec) + L->tsz * L->plane * L->rec_slot[sensor];
    else if (L->eval_step == L->step && L->eval_sensor == sensor)
      where = L->evalplane;
  }
  if (have_out && (sensor < 0 || where)) {
    if (field) *field = where;
    return KSS_OK;
  }
  const int s = (sensor >= 0 && !where) ? sensor : -1;
  int rc = KSS_OK;
  if (have_out && (rc = ensure_eval_out(L))) return rc;
  KSS_CUDA(L, with_storage(L->cfg.precision, [&](auto tag) {
             return launch_eval<typename decltype(tag)::type>(L, s, have_out);
           }));
  L->out_step = L->step;
  if (s >= 0) {
    L->eval_step = L->step;
    L->eval_sensor = s;
    where = L->evalplane;
  }
  if (field) *field = where;
  return KSS_OK;
}

int nonpos_status(kss_lattice* L) {
  unsigned long long c[3];
  KSS_CUDA(L, cudaMemcpyAsync(c, L->stat_counts, sizeof(c), cudaMemcpyDeviceToHost, L->stream));
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  const int rc = device_error(L);
  if (rc) return rc;
  return c[2] > 0 ? KSS_WARN_NONPOSITIVE : KSS_OK;
}

}  // namespace

namespace kss_rt {

// After a stream synchronisation: did a bounded device wait run out?  (sticky)
int device_error(kss_lattice* L) {
  uint32_t w = 0;
  KSS_CUDA(L, cudaMemcpyAsync(&w, L->err_word, sizeof(w), cudaMemcpyDeviceToHost, L->stream));
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  if (w & kss::kErrBounds) {
    L->err = KSS_ERR_BOUNDS;
    L->msg = "a device bounds check failed (debug build)";
    return KSS_ERR_BOUNDS;
  }
  if (w) {
    L->err = KSS_ERR_TIMEOUT;
    L->msg = "a bounded device wait ran out (bulk copy did not complete)";
    return KSS_ERR_TIMEOUT;
  }
  return KSS_OK;
}

// ---- counted device allocations and host-side fault injection (test support) ----
namespace inject {
std::atomic<long long> g_live_allocs{0};
std::mutex g_inject_mutex;
long long g_fail_alloc = -1;   // allocations to pass before one fails (-1: disarmed)
long long g_fail_launch = -1;  // kss_step calls to pass before one fails (-1: disarmed)

// Is the armed event of this counter due now?  (then it disarms)
bool injection_due(long long& counter) {
  std::lock_guard<std::mutex> lock(g_inject_mutex);
  if (counter < 0) return false;
  if (counter-- == 0) {
    counter = -1;
    return true;
  }
  return false;
}
}  // namespace inject
using inject::g_fail_alloc;
using inject::g_fail_launch;
using inject::g_inject_mutex;
using inject::g_live_allocs;
using inject::injection_due;

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  if (injection_due(g_fail_alloc)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) ++g_live_allocs;
  return e;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  const cudaError_t e = cudaFree(p);
  if (e == cudaSuccess) --g_live_allocs;
  return e;
}

cudaError_t injected_launch_error() {
  return injection_due(g_fail_launch) ? cudaErrorLaunchFailure : cudaSuccess;
}

void release(kss_lattice* L) {
  if (!L) return;
  cudaStreamSynchronize(L->stream);
  regrid_release(L);
  if (L->multi) kss_rt::dev_free(L->multi);
  if (L->region) kss_rt::dev_free(L->region);
  if (L->eval_out) kss_rt::dev_free(L->eval_out);
  for (auto& g : L->plain_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (L->cap) cudaStreamDestroy(L->cap);
  void* bufs[] = {L->f_alloc[0], L->f_alloc[1], L->rec, L->evalplane, L->flags, L->tiles, L->part_sum,
                  L->part_cnt, L->small, L->staging, L->defer_list};
  for (void* b : bufs)
    if (b) kss_rt::dev_free(b);
  if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
  delete L;
}

}  // namespace kss_rt

extern "C" {

int kss_version(void) { return kVersion; }

const char* kss_strerror(int code) {
  switch (code) {
    case KSS_OK: return "ok";
    case KSS_ERR_ARG: return "invalid argument";
    case KSS_ERR_OOM: return "out of memory";
    case KSS_ERR_CUDA: return "CUDA error";
    case KSS_ERR_TIMEOUT: return "device wait timed out";
    case KSS_ERR_BOUNDS: return "device bounds check failed";
    case KSS_ERR_STATE: return "invalid state";
    case KSS_ERR_UNSUPPORTED: return "unsupported option";
    case KSS_WARN_NONPOSITIVE: return "non-positive populations present";
    default: return "unknown error code";
  }
}

const char* kss_last_error(const kss_lattice* L) { return L ? L->msg.c_str() : "null lattice"; }

int kss_config_default(kss_config* c, int32_t nx, int32_t ny, int32_t precision) {
  if (!c) return KSS_ERR_ARG;
  std::memset(c, 0, sizeof(*c));
  c->nx = nx;
  c->ny = ny;
  c->precision = precision;
  c->tau = 0.8;
  c->refine_sensor = KSS_S_KN;
  c->refine_threshold = 1e-3;
  c->switch_sensor = KSS_S_NEQ;
  c->switch_threshold = 1e-4;
  c->record_mask = 1u << KSS_S_KL;
  c->output_every = 1;
  c->tile = 16;
  c->stream = nullptr;
  c->own_stream = 0;
  c->kernel = KSS_KERNEL_AUTO;
  c->rho0 = 1.0;
  c->dev_exp = 12;
  c->dev_unscaled = 0;
  c->tau2 = 0.0;
  return KSS_OK;
}

static int create_lattice(const kss_config* cfg, bool slab, kss_lattice** out) {
  if (!out) return KSS_ERR_ARG;
  *out = nullptr;
  const int rc = check_config(cfg);
  if (rc) return rc;
  kss_lattice* L = new (std::nothrow) kss_lattice();
  if (!L) return KSS_ERR_OOM;
  L->cfg = *cfg;
  L->slab = slab;
  if (cudaGetDevice(&L->device) != cudaSuccess) {
    cudaGetLastError();
    delete L;
    return KSS_ERR_CUDA;
  }
  L->esz = cfg->precision == KSS_FP64 ? 8 : (cfg->precision == KSS_FP32 ? 4 : 2);
  L->tsz = cfg->precision == KSS_FP64 ? 8 : 4;
  if (cfg->precision == KSS_FP16DEV) {
    // b_q = RN_fp32(w_q rho0); s_q = 2^(k_q + K), k_q = 1, 3, 5 (w_q = 4/9, 1/9, 1/36)
    static const double w[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    static const int k[9] = {1, 3, 3, 3, 3, 5, 5, 5, 5};
    for (int q = 0; q < 9; ++q) {
      L->codec16.base[q] = static_cast<float>(w[q] * cfg->rho0);
      const int e = cfg->dev_unscaled ? 0 : k[q] + cfg->dev_exp;
      L->codec16.scale[q] = std::ldexp(1.0f, e);
      L->codec16.inv[q] = std::ldexp(1.0f, -e);
    }
  }
  const int align = int(128 / L->esz);
  L->pitch = (cfg->nx + align - 1) / align * align;
  // a slab's planes hold its two halo rows too (row -1 before its rows, row ny after)
  L->plane = (long long)L->pitch * (cfg->ny + (slab ? 2 : 0));
  L->ntx = (cfg->nx + cfg->tile - 1) / cfg->tile;
  L->nty = (cfg->ny + cfg->tile - 1) / cfg->tile;
  if (cudaDeviceGetAttribute(&L->nsm, cudaDevAttrMultiProcessorCount, L->device) != cudaSuccess ||
      L->nsm < 1) {
    cudaGetLastError();
    delete L;
    return KSS_ERR_CUDA;
  }
  // CTA height: 32 rows; 64 rows when even 64-row CTAs make at least 4 waves of the 3
  // resident CTAs per SM (the per-CTA epilogue and, in multi-step launches, the per-block
  // dependency waits then cost more than the longer tail: fused 4096^2 FP32 multi-step
  // 0.2282 vs 0.2306 ms per step, single launches 0.2415 vs 0.2437 ms)
  auto grid_for = [&](int bands) {
    return with_storage(cfg->precision, [&](auto tag) {
      return kss::step_grid<typename decltype(tag)::type>(cfg->nx, cfg->ny, cfg->tile, bands);
    });
  };
  // Steps without outputs have no epilogue to amortise and no tile counts: 64 rows from 8
  // waves of such CTAs up (4096^2 FP32 plain step 0.181 vs 0.185 ms with 64 rows), else the
  // tallest CTA of 32, 16 or 8 rows that gives two CTAs per SM (small lattices fill the GPU).
  L->bands = kss::step_bands(cfg->tile);
  const int cols = with_storage(cfg->precision, [](auto tag) {
    return 32 * kss::Vec<typename decltype(tag)::type>::N;
  });
  L->rows_plain = kss::fill_rows(cfg->nx, cfg->ny, cols, L->nsm);
  if (cfg->tile <= 64 && 64 % cfg->tile == 0 && 64 / cfg->tile <= kss::kMaxBands) {
    const dim3 g64 = grid_for(64 / cfg->tile);
    if ((long long)g64.x * g64.y >= 4LL * 3 * L->nsm) L->bands = 64 / cfg->tile;
    if ((long long)g64.x * g64.y >= 8LL * 3 * L->nsm) L->rows_plain = 64;
  }
  const dim3 g = grid_for(L->bands);
  L->nblocks = int(g.x * g.y);
  const int npart = std::max(L->nblocks, L->nsm);  // partials of either step kernel
  // list of deferred cells: 1/8 of the lattice (a full scan takes over beyond that)
  L->defer_cap = uint32_t(std::max<long long>(4096, (long long)cfg->nx * cfg->ny / 8));
  int nrec = 0;
  for (int s = 0; s < KSS_S_COUNT; ++s)
    L->rec_slot[s] = ((cfg->record_mask >> s) & 1u) ? nrec++ : -1;

  if (!cfg->own_stream) {
    L->stream = static_cast<cudaStream_t>(cfg->stream);
  } else {
    if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete L;
      return KSS_ERR_CUDA;
    }
    L->own_stream = true;
  }
  const size_t pop_bytes = 9 * size_t(L->plane) * L->esz;
  const size_t plane_bytes = size_t(L->plane) * L->tsz;  // sensor planes
  struct {
    void** p;
    size_t bytes;
  } allocs[] = {
      {&L->f_alloc[0], pop_bytes},
      {&L->f_alloc[1], pop_bytes},
      {&L->rec, plane_bytes * (nrec > 0 ? nrec : 1)},
      {&L->evalplane, plane_bytes},
      {reinterpret_cast<void**>(&L->flags), size_t(L->pitch) * cfg->ny},
      {reinterpret_cast<void**>(&L->tiles), sizeof(int32_t) * 3 * size_t(L->ntx) * L->nty},
      {reinterpret_cast<void**>(&L->part_sum), sizeof(double) * 3 * size_t(npart)},
      {reinterpret_cast<void**>(&L->part_cnt), sizeof(uint32_t) * 4 * size_t(npart)},
      {reinterpret_cast<void**>(&L->small), 256},
      {reinterpret_cast<void**>(&L->defer_list), sizeof(uint32_t) * size_t(L->defer_cap)},
  };
  for (auto& a : allocs) {
    if (kss_rt::dev_malloc(a.p, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      release(L);
      return KSS_ERR_OOM;
    }
    if (cudaMemsetAsync(*a.p, 0, a.bytes, L->stream) != cudaSuccess) {
      cudaGetLastError();
      release(L);
      return KSS_ERR_CUDA;
    }
  }
  if (cfg->tau2 > 0.0) {
    const size_t bytes = size_t(L->pitch) * cfg->ny;
    if (kss_rt::dev_malloc(&L->region, bytes) != cudaSuccess) {
      cudaGetLastError();
      L->region = nullptr;
      release(L);
      return KSS_ERR_OOM;
    }
    if (cudaMemsetAsync(L->region, 0, bytes, L->stream) != cudaSuccess) {
      cudaGetLastError();
      release(L);
      return KSS_ERR_CUDA;
    }
  }
  for (int b = 0; b < 2; ++b)  // row 0 of plane 0 (a slab's halo row -1 precedes it)
    L->f[b] = static_cast<unsigned char*>(L->f_alloc[b]) + (slab ? size_t(L->pitch) * L->esz : 0);
  L->done = reinterpret_cast<uint32_t*>(L->small);
  L->stat_sums = reinterpret_cast<double*>(L->small + 64);
  L->stat_counts = reinterpret_cast<unsigned long long*>(L->small + 128);
  L->err_word = reinterpret_cast<uint32_t*>(L->small + 192);
  if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
    cudaGetLastError();
    release(L);
    return KSS_ERR_CUDA;
  }
  *out = L;
  return KSS_OK;
}

int kss_create(const kss_config* cfg, kss_lattice** out) {
  return create_lattice(cfg, false, out);
}

int kss_slab_create(const kss_config* cfg, kss_lattice** out) {
  return create_lattice(cfg, true, out);
}

void kss_destroy(kss_lattice* L) {
  if (!L || L->owner) return;  // members of a batch are freed with the batch
  DeviceGuard g(L->device);
  release(L);
}

// A new state: step 0, no outputs yet, an empty two-relaxation region.
static int reset_after_set(kss_lattice* L) {
  L->step = 0;
  L->out_step = L->rec_step = L->eval_step = -1;
  L->eval_sensor = -1;
  if (L->region)
    KSS_CUDA(L, cudaMemsetAsync(L->region, 0, size_t(L->pitch) * L->cfg.ny, L->stream));
  return KSS_OK;
}

}  // extern "C"

// kss_set_fields and kss_set_fields_f32: fields of element type E (double or float), read
// in place from device or page-locked host memory, else through the staging buffer.
namespace {
template <class E>
int set_fields_of(kss_lattice* L, const E* rho, const E* ux, const E* uy, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!rho || !ux || !uy) return fail(L, KSS_ERR_ARG, "null field pointer");
  DeviceGuard g(L->device);
  const size_t n = size_t(L->cfg.nx) * L->cfg.ny;
  const E *r = rho, *u = ux, *v = uy;
  if (!on_device) {
    r = pinned_device_view(rho);
    u = pinned_device_view(ux);
    v = pinned_device_view(uy);
  }
  if (!on_device && !(r && u && v)) {
    // (the staging buffer holds 3 n doubles: enough for 3 n elements of either type)
    if ((rc = ensure_staging(L, 3 * n))) return rc;
    E* st = reinterpret_cast<E*>(L->staging);
    KSS_CUDA(L, cudaMemcpyAsync(st, rho, n * sizeof(E), cudaMemcpyHostToDevice, L->stream));
    KSS_CUDA(L, cudaMemcpyAsync(st + n, ux, n * sizeof(E), cudaMemcpyHostToDevice, L->stream));
    KSS_CUDA(L, cudaMemcpyAsync(st + 2 * n, uy, n * sizeof(E), cudaMemcpyHostToDevice, L->stream));
    r = st;
    u = st + n;
    v = st + 2 * n;
  }
  const int nx = L->cfg.nx, ny = L->cfg.ny;
  KSS_CUDA(L, with_storage(L->cfg.precision, [&](auto tag) {
             using S = typename decltype(tag)::type;
             S* const f = static_cast<S*>(L->f[L->cur]);
             if constexpr (std::is_same<E, float>::value)
               return kss::launch_init_equilibrium_f32<S>(r, u, v, f, L->plane, L->pitch, nx,
                                                          ny, codec_of<S>(L), L->stream);
             else
               return kss::launch_init_equilibrium<S>(r, u, v, f, L->plane, L->pitch, nx, ny,
                                                      codec_of<S>(L), L->stream);
           }));
  if (!on_device) KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return reset_after_set(L);
}
}  // namespace

extern "C" {

int kss_set_fields(kss_lattice* L, const double* rho, const double* ux, const double* uy,
                   int on_device) {
  return set_fields_of<double>(L, rho, ux, uy, on_device);
}

int kss_set_fields_f32(kss_lattice* L, const float* rho, const float* ux, const float* uy,
                       int on_device) {
  return set_fields_of<float>(L, rho, ux, uy, on_device);
}

int kss_set_populations(kss_lattice* L, const double* f, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!f) return fail(L, KSS_ERR_ARG, "null population pointer");
  DeviceGuard g(L->device);
  const size_t n = 9 * size_t(L->cfg.nx) * L->cfg.ny;
  const double* src = on_device ? f : pinned_device_view(f);
  if (!src) {
    if ((rc = ensure_staging(L, n))) return rc;
    KSS_CUDA(L, cudaMemcpyAsync(L->staging, f, n * 8, cudaMemcpyHostToDevice, L->stream));
    src = L->staging;
  }
  const int nx = L->cfg.nx, ny = L->cfg.ny;
  KSS_CUDA(L, with_storage(L->cfg.precision, [&](auto tag) {
             using S = typename decltype(tag)::type;
             return kss::launch_dense_to_pops<S>(src, L->plane, L->pitch, nx, ny,
                                                 static_cast<S*>(L->f[L->cur]), codec_of<S>(L),
                                                 L->stream);
           }));
  if (!on_device) KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return reset_after_set(L);
}

int kss_get_populations(kss_lattice* L, double* f, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!f) return fail(L, KSS_ERR_ARG, "null population pointer");
  DeviceGuard g(L->device);
  const size_t n = 9 * size_t(L->cfg.nx) * L->cfg.ny;
  double* dst = f;
  if (!on_device) {
    if ((rc = ensure_staging(L, n))) return rc;
    dst = L->staging;
  }
  const int nx = L->cfg.nx, ny = L->cfg.ny;
  KSS_CUDA(L, with_storage(L->cfg.precision, [&](auto tag) {
             using S = typename decltype(tag)::type;
             return kss::launch_pops_to_dense<S>(static_cast<const S*>(L->f[L->cur]), L->plane,
                                                 L->pitch, nx, ny, dst, codec_of<S>(L), L->stream);
           }));
  if (!on_device)
    KSS_CUDA(L, cudaMemcpyAsync(f, L->staging, n * 8, cudaMemcpyDeviceToHost, L->stream));
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return device_error(L);
}

int kss_step(kss_lattice* L, int32_t nsteps) {
  const kss_rt::NvtxRange nvtx_range("kss_step");
  int rc = enter(L);
  if (rc) return rc;
  if (nsteps < 0) return fail(L, KSS_ERR_ARG, "negative step count");
  if (L->slab && nsteps > 1)
    return fail(L, KSS_ERR_ARG, "a slab steps once per call: its halo rows change every step");
  if (injected_launch_error() != cudaSuccess)
    return fail(L, KSS_ERR_CUDA, "injected launch failure (kss_testing_fail_after)");
  DeviceGuard g(L->device);
  // several output steps of the {Kn, KL, neq} set on FP32 or FP64 storage: one multi-step
  // launch (measured on GB300 at 4096^2 FP32: 0.232 vs 0.244 ms per step; plain steps and
  // FP16-deviation storage gain nothing from it: 0.179 vs 0.179, 0.224 vs 0.221 ms)
  const int every = L->cfg.output_every;
  const int mode =
      every == 1 ? mode_for(needed_mask(L, L->cfg.record_mask), L->region != nullptr) : MODE_PLAIN;
  if (KSS_MULTISTEP && nsteps >= 2 && every == 1 && mode == MODE_STD &&
      (KSS_MULTISTEP_F16 || L->cfg.precision != KSS_FP16DEV) &&
      (L->region || !use_tma(L, mode)) &&
      (long long)nsteps * L->nblocks < (1LL << 30)) {
    KSS_CUDA(L, with_storage(L->cfg.precision, [&](auto tag) {
               return launch_multi<typename decltype(tag)::type>(L, mode, nsteps);
             }));
    L->cur ^= nsteps & 1;
    L->step += nsteps;
    if (every == 1) L->out_step = L->rec_step = L->step;
    return KSS_OK;
  }
  // any other run of steps: one launch each, replayed as graphs of at most kGraphChunk
  // steps; longer runs go in chunks of whole output periods and an even step count, so that
  // every chunk has the same (count, buffer, phase) key and replays the same graph
  int32_t left = nsteps;
  while (left > 0) {
    int32_t c = 1;
    if (KSS_STEP_GRAPHS && left >= 2) {
      c = std::min<int32_t>(left, kGraphChunk);
      const int64_t period = every > 0 ? std::lcm<int64_t>(2, every) : 2;
      if (c < left && period <= kGraphChunk) c = int32_t(c / period * period);
    }
    if (c >= 2) {
      if ((rc = steps_graph(L, c))) return rc;
    } else {
      const bool out = is_output_step(L, L->step + 1);
      KSS_CUDA(L, with_storage(L->cfg.precision, [&](auto tag) {
                 return launch_one_step<typename decltype(tag)::type>(L, out);
               }));
    }
    for (int32_t s = 0; s < c; ++s)
      if (is_output_step(L, L->step + s + 1)) L->out_step = L->rec_step = L->step + s + 1;
    L->cur ^= c & 1;
    L->step += c;
    left -= c;
  }
  return KSS_OK;
}

int kss_read_moments(kss_lattice* L, double* rho, double* ux, double* uy, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!rho || !ux || !uy) return fail(L, KSS_ERR_ARG, "null field pointer");
  DeviceGuard g(L->device);
  const size_t n = size_t(L->cfg.nx) * L->cfg.ny;
  double *r = rho, *u = ux, *v = uy;
  if (!on_device) {
    if ((rc = ensure_staging(L, 3 * n))) return rc;
    r = L->staging;
    u = L->staging + n;
    v = L->staging + 2 * n;
  }
  const int nx = L->cfg.nx, ny = L->cfg.ny;
  KSS_CUDA(L, with_storage(L->cfg.precision, [&](auto tag) {
             using S = typename decltype(tag)::type;
             return kss::launch_moments<S>(static_cast<const S*>(L->f[L->cur]), L->plane,
                                           L->pitch, nx, ny, r, u, v, codec_of<S>(L), L->stream);
           }));
  if (!on_device) {
    KSS_CUDA(L, cudaMemcpyAsync(rho, r, n * 8, cudaMemcpyDeviceToHost, L->stream));
    KSS_CUDA(L, cudaMemcpyAsync(ux, u, n * 8, cudaMemcpyDeviceToHost, L->stream));
    KSS_CUDA(L, cudaMemcpyAsync(uy, v, n * 8, cudaMemcpyDeviceToHost, L->stream));
  }
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return device_error(L);
}

int kss_read_sensor(kss_lattice* L, int32_t sensor, double* out, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!valid_sensor(sensor)) return fail(L, KSS_ERR_ARG, "invalid sensor id");
  if (!out) return fail(L, KSS_ERR_ARG, "null output pointer");
  DeviceGuard g(L->device);
  const void* field = nullptr;
  if ((rc = ensure_outputs(L, sensor, &field))) return rc;
  const size_t n = size_t(L->cfg.nx) * L->cfg.ny;
  double* dst = out;
  if (!on_device) {
    if ((rc = ensure_staging(L, n))) return rc;
    dst = L->staging;
  }
  const int nx = L->cfg.nx, ny = L->cfg.ny;
  if (L->cfg.precision != KSS_FP64)  // FP32 and FP16-deviation lattices: FP32 sensor planes
    KSS_CUDA(L, kss::launch_pitched_to_dense<float>(static_cast<const float*>(field), L->plane,
                                                    L->pitch, nx, ny, 1, dst, L->stream));
  else
    KSS_CUDA(L, kss::launch_pitched_to_dense<double>(static_cast<const double*>(field), L->plane,
                                                     L->pitch, nx, ny, 1, dst, L->stream));
  if (!on_device)
    KSS_CUDA(L, cudaMemcpyAsync(out, L->staging, n * 8, cudaMemcpyDeviceToHost, L->stream));
  return nonpos_status(L);
}

int kss_read_flags(kss_lattice* L, uint8_t* flags, int32_t* tile_counts, int64_t counts[3],
                   int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  DeviceGuard g(L->device);
  if ((rc = ensure_outputs(L, -1, nullptr))) return rc;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (flags)
    KSS_CUDA(L, cudaMemcpy2DAsync(flags, size_t(L->cfg.nx), L->flags, size_t(L->pitch),
                                  size_t(L->cfg.nx), size_t(L->cfg.ny), kind, L->stream));
  if (tile_counts)
    KSS_CUDA(L, cudaMemcpyAsync(tile_counts, L->tiles,
                                sizeof(int32_t) * 2 * size_t(L->ntx) * L->nty, kind, L->stream));
  unsigned long long c[3];
  KSS_CUDA(L, cudaMemcpyAsync(c, L->stat_counts, sizeof(c), cudaMemcpyDeviceToHost, L->stream));
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  if ((rc = device_error(L))) return rc;
  if (counts)
    for (int k = 0; k < 3; ++k) counts[k] = int64_t(c[k]);
  return c[2] > 0 ? KSS_WARN_NONPOSITIVE : KSS_OK;
}

int kss_read_stats(kss_lattice* L, double sums[3], int64_t counts[3], int64_t* step) {
  int rc = enter(L);
  if (rc) return rc;
  DeviceGuard g(L->device);
  if ((rc = ensure_outputs(L, -1, nullptr))) return rc;
  double s[3];
  unsigned long long c[3];
  KSS_CUDA(L, cudaMemcpyAsync(s, L->stat_sums, sizeof(s), cudaMemcpyDeviceToHost, L->stream));
  KSS_CUDA(L, cudaMemcpyAsync(c, L->stat_counts, sizeof(c), cudaMemcpyDeviceToHost, L->stream));
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  if ((rc = device_error(L))) return rc;
  if (sums)
    for (int k = 0; k < 3; ++k) sums[k] = s[k];
  if (counts)
    for (int k = 0; k < 3; ++k) counts[k] = int64_t(c[k]);
  if (step) *step = L->out_step;
  return c[2] > 0 ? KSS_WARN_NONPOSITIVE : KSS_OK;
}

int kss_set_aar_region(kss_lattice* L, const uint8_t* region, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!L->region) return fail(L, KSS_ERR_STATE, "the lattice has no two-relaxation model (tau2 = 0)");
  if (!region) return fail(L, KSS_ERR_ARG, "null region pointer");
  DeviceGuard g(L->device);
  KSS_CUDA(L, cudaMemcpy2DAsync(L->region, size_t(L->pitch), region, size_t(L->cfg.nx),
                                size_t(L->cfg.nx), size_t(L->cfg.ny),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                L->stream));
  const int ny = L->cfg.ny;
  region_to_01_kernel<<<dim3((L->cfg.nx + 255) / 256, ny < 65535 ? ny : 65535), 256, 0,
                        L->stream>>>(L->region, L->pitch, L->cfg.nx, ny);
  KSS_CUDA(L, cudaGetLastError());
  if (!on_device) KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return KSS_OK;
}

int kss_get_aar_region(kss_lattice* L, uint8_t* region, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!L->region) return fail(L, KSS_ERR_STATE, "the lattice has no two-relaxation model (tau2 = 0)");
  if (!region) return fail(L, KSS_ERR_ARG, "null region pointer");
  DeviceGuard g(L->device);
  KSS_CUDA(L, cudaMemcpy2DAsync(region, size_t(L->cfg.nx), L->region, size_t(L->pitch),
                                size_t(L->cfg.nx), size_t(L->cfg.ny),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                L->stream));
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return device_error(L);
}

int kss_testing_expire_wait(kss_lattice* L, int64_t deadline_cycles) {
  int rc = enter(L);
  if (rc) return rc;
  if (deadline_cycles < 1 || deadline_cycles > 1000000000LL)
    return fail(L, KSS_ERR_ARG, "deadline must be 1 .. 1e9 cycles");
  DeviceGuard g(L->device);
  expire_wait_kernel<<<1, 1, 0, L->stream>>>(L->err_word, (long long)deadline_cycles);
  KSS_CUDA(L, cudaGetLastError());
  return KSS_OK;
}

// ---- y-slab decomposition: the rows that cross a slab's faces ----
// Pull streaming moves population q from row j - cy_q to row j: a slab's row 0 takes the
// c_y = +1 populations (q = 2, 5, 6) of the row below it, its row ny - 1 the c_y = -1
// populations (q = 4, 7, 8) of the row above it.  Each is a row of nx elements of one
// plane, contiguous in memory; a buffer of the exchange holds three such rows.
static const int kUpQ[3] = {2, 5, 6};    // cross the face above a slab, upwards
static const int kDownQ[3] = {4, 7, 8};  // cross the face below a slab, downwards

static int slab_rows(kss_lattice* L, const int* qs, int row, void* buf, bool to_buf) {
  const size_t row_bytes = size_t(L->cfg.nx) * L->esz;
  unsigned char* base = static_cast<unsigned char*>(L->f[L->cur]);
  for (int k = 0; k < 3; ++k) {
    unsigned char* r =
        base + (size_t(qs[k]) * size_t(L->plane) + (long long)row * L->pitch) * L->esz;
    unsigned char* b = static_cast<unsigned char*>(buf) + size_t(k) * row_bytes;
    KSS_CUDA(L, cudaMemcpyAsync(to_buf ? b : r, to_buf ? r : b, row_bytes, cudaMemcpyDefault,
                                L->stream));
  }
  return KSS_OK;
}

int kss_slab_edges(kss_lattice* L, void* to_below, void* to_above, int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!L->slab) return fail(L, KSS_ERR_ARG, "not a slab lattice (kss_slab_create)");
  if (!to_below || !to_above) return fail(L, KSS_ERR_ARG, "null buffer");
  DeviceGuard g(L->device);
  rc = slab_rows(L, kDownQ, 0, to_below, true);
  if (rc) return rc;
  rc = slab_rows(L, kUpQ, L->cfg.ny - 1, to_above, true);
  if (rc) return rc;
  if (!on_device) KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return KSS_OK;
}

int kss_slab_set_halos(kss_lattice* L, const void* from_below, const void* from_above,
                       int on_device) {
  int rc = enter(L);
  if (rc) return rc;
  if (!L->slab) return fail(L, KSS_ERR_ARG, "not a slab lattice (kss_slab_create)");
  if (!from_below || !from_above) return fail(L, KSS_ERR_ARG, "null buffer");
  DeviceGuard g(L->device);
  rc = slab_rows(L, kUpQ, -1, const_cast<void*>(from_below), false);
  if (rc) return rc;
  rc = slab_rows(L, kDownQ, L->cfg.ny, const_cast<void*>(from_above), false);
  if (rc) return rc;
  if (!on_device) KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return KSS_OK;
}

int kss_testing_expire_mbarrier(kss_lattice* L, int64_t deadline_cycles) {
  int rc = enter(L);
  if (rc) return rc;
  if (deadline_cycles < 1 || deadline_cycles > 1000000000LL)
    return fail(L, KSS_ERR_ARG, "deadline must be 1 .. 1e9 cycles");
  DeviceGuard g(L->device);
  expire_mbarrier_kernel<<<1, 32, 0, L->stream>>>(L->err_word, (long long)deadline_cycles);
  KSS_CUDA(L, cudaGetLastError());
  return KSS_OK;
}

int kss_testing_fail_after(int32_t kind, int64_t n) {
  if (kind != 0 && kind != 1) return KSS_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_inject_mutex);
  (kind == 0 ? g_fail_alloc : g_fail_launch) = n < 0 ? -1 : (long long)n;
  return KSS_OK;
}

int64_t kss_testing_live_allocations(void) { return g_live_allocs.load(); }

int kss_get_step(const kss_lattice* L, int64_t* step) {
  if (!L || !step) return KSS_ERR_ARG;
  *step = L->step;
  return KSS_OK;
}

int kss_sync(kss_lattice* L) {
  int rc = enter(L);
  if (rc) return rc;
  DeviceGuard g(L->device);
  KSS_CUDA(L, cudaStreamSynchronize(L->stream));
  return device_error(L);
}

}  // extern "C"
