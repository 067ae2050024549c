// kss_adjoint.cu -- host side of the adjoint entry points (include/kss.h): the forward
// pass with checkpoints, the segment-wise recomputation and the reverse sweep of the
// adjoint kernels (adjoint_kernel.cuh).
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "runtime.h"

using namespace kss_rt;

// Rows per CTA of the adjoint kernels: 0 takes fill_rows (the tallest of 32, 16, 8 that
// still gives two CTAs per SM); 8, 16 or 32 fix it (a build-time tuning knob).
#ifndef KSS_ADJ_ROWS
#define KSS_ADJ_ROWS 0
#endif

struct kss_adjoint {
  kss_adjoint_config cfg{};
  int device = 0;
  bool fp32 = true;
  size_t esz = 4;
  int pitch = 0;
  long long plane = 0;
  size_t state_bytes = 0;  // one population buffer (9 planes)
  int nck = 0;             // checkpoints kept: f^0, f^E, f^2E, ... (E = checkpoint_every)
  int adj_rows = 32;       // rows per CTA of the adjoint kernels (fill_rows)
  int step_rows = 32;      // rows per CTA of the forward steps (fill_rows)
  unsigned char* ck = nullptr;   // nck states
  // two buffers of checkpoint_every states: a segment's states (slot k - s0 for step k,
  // slot 0 unused: that state is the checkpoint), the last segment's written by the
  // forward pass, the others recomputed; segment i (counted from the last) uses seg[i & 1]
  unsigned char* seg = nullptr;
  unsigned char* seg2 = nullptr;
  unsigned char* work[2] = {nullptr, nullptr};  // forward ping-pong
  unsigned char* lam[2] = {nullptr, nullptr};   // adjoint ping-pong
  void* wplane = nullptr;    // weights, one pitched plane of T
  double* fields = nullptr;  // staging: rho0, ux0, uy0 (dense)
  double* grad = nullptr;    // dense dJ/drho0
  double* part = nullptr;    // per-CTA partials
  unsigned char* small = nullptr;  // done counter @0, acc[2] @64, error word @128
  // the reverse sweep of a segment in one cooperative launch (adj_multi_kernel): its
  // counters (block progress, iteration tickets, work counter: zeroed before each launch),
  // the per-block partials and the iteration totals
  bool multi = true;
  int multi_ctas = 0;
  uint32_t* mcount = nullptr;  // [nblocks] done, [E] tickets, [1] work, [fnblocks] fdone
  double* mpart = nullptr;     // [E][nblocks]
  double* mtot = nullptr;      // [E]
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double tau = 0;
  int lam_cur = 0;         // lam[lam_cur] holds lt^{N-1} after the forward pass
  bool have_forward = false;
  bool have_weight = false;
  // the forward and the backward launch sequences replayed as CUDA graphs, recorded on a
  // stream of their own for the (tau, weight) they were taken with
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_fwd = nullptr, g_bwd = nullptr;
  double g_tau = 0;
  int g_weight = -1;
  std::string msg;
};

namespace {

int afail(kss_adjoint* A, int code, const std::string& m) {
  if (A) A->msg = m;
  return code;
}

#define KSS_ACUDA(A, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return afail((A), KSS_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

void free_all(kss_adjoint* A) {
  if (!A) return;
  DeviceGuard g(A->device);
  cudaStreamSynchronize(A->stream);
  void* bufs[] = {A->ck,     A->seg,    A->seg2,  A->work[0], A->work[1],
                  A->lam[0], A->lam[1], A->wplane, A->fields, A->grad,
                  A->part,   A->small,  A->mcount, A->mpart,  A->mtot};
  for (void* b : bufs)
    if (b) kss_rt::dev_free(b);
  if (A->g_fwd) cudaGraphExecDestroy(A->g_fwd);
  if (A->g_bwd) cudaGraphExecDestroy(A->g_bwd);
  if (A->cap) cudaStreamDestroy(A->cap);
  if (A->own_stream && A->stream) cudaStreamDestroy(A->stream);
  delete A;
}

unsigned char* state_at(kss_adjoint* A, unsigned char* base, long long k) {
  return base + size_t(k) * A->state_bytes;
}

// Parameters of a plain forward step (stream + collide, no outputs) from src to dst.
template <class T>
kss::StepParams<T> plain_params(const kss_adjoint* A, const void* src, void* dst) {
  kss::StepParams<T> p{};
  p.src = static_cast<const T*>(src);
  p.dst = static_cast<T*>(dst);
  p.plane = A->plane;
  p.pitch = A->pitch;
  p.nx = A->cfg.nx;
  p.ny = A->cfg.ny;
  p.tile = 8;  // no outputs: the tile only shapes the grid, step_rows rows per CTA
  p.bands = A->step_rows / 8;
  p.ntx = (A->cfg.nx + 7) / 8;
  p.nty = (A->cfg.ny + 7) / 8;
  p.omega = T(1.0 / A->tau);
  p.tau = T(A->tau);
  for (int s = 0; s < KSS_S_COUNT; ++s) p.rec_slot[s] = -1;
  return p;
}

// One plain forward step from src to dst.
template <class T>
cudaError_t plain_step(const kss_adjoint* A, const void* src, void* dst, cudaStream_t s) {
  return kss::launch_step<T>(plain_params<T>(A, src, dst), kss::MODE_PLAIN, true, true, s);
}

// The forward step grid of the plain steps (plain_params: tile 8, step_rows rows).
template <class T>
dim3 plain_grid(const kss_adjoint* A) {
  return kss::step_grid<T>(A->cfg.nx, A->cfg.ny, 8, A->step_rows / 8);
}

// First step of the last segment of states f^0 .. f^{N-2} that the reverse sweep needs.
int last_segment(const kss_adjoint* A) {
  const int N = A->cfg.nsteps, E = A->cfg.checkpoint_every;
  return N >= 2 ? ((N - 2) / E) * E : -1;
}

template <class T>
kss::AdjParams<T> adj_params(kss_adjoint* A) {
  kss::AdjParams<T> p{};
  p.part = A->part;
  p.done = reinterpret_cast<uint32_t*>(A->small);
  p.plane = A->plane;
  p.pitch = A->pitch;
  p.nx = A->cfg.nx;
  p.ny = A->cfg.ny;
  p.rows = A->adj_rows;
  p.omega = T(1.0 / A->tau);
  p.err = reinterpret_cast<uint32_t*>(A->small + 128);
  return p;
}

double* acc_at(kss_adjoint* A, int k) { return reinterpret_cast<double*>(A->small + 64) + k; }

// The launches of the forward pass on stream s: f^0, f^1 .. f^{N-1} (checkpoints in their
// slots) and the objective with its seed lt^{N-1}.
template <class T>
cudaError_t forward_launches(kss_adjoint* A, cudaStream_t s) {
  const int N = A->cfg.nsteps, E = A->cfg.checkpoint_every;
  const size_t n = size_t(A->cfg.nx) * A->cfg.ny;
  cudaError_t e = kss::launch_init_equilibrium<T>(A->fields, A->fields + n, A->fields + 2 * n,
                                                  reinterpret_cast<T*>(A->ck), A->plane,
                                                  A->pitch, A->cfg.nx, A->cfg.ny,
                                                  kss::codec_t<T>{}, s);
  // f^k for k = 1 .. N-1: checkpoints land in their slot, the last segment's states in
  // seg[0] (the reverse sweep reads them without recomputing), the others alternate in
  // work[]
  const int sl = last_segment(A);
  const void* cur = A->ck;
  for (int k = 1; k < N && e == cudaSuccess; ++k) {
    void* dst = (k % E == 0)         ? state_at(A, A->ck, k / E)
                : (sl >= 0 && k > sl && k <= N - 2) ? state_at(A, A->seg, k - sl)
                                                    : A->work[k & 1];
    e = plain_step<T>(A, cur, dst, s);
    cur = dst;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(A->small + 64, 0, 2 * sizeof(double), s);
  kss::AdjParams<T> p = adj_params<T>(A);
  p.f = static_cast<const T*>(cur);
  p.lam_out = reinterpret_cast<T*>(A->lam[0]);
  p.weight = A->have_weight ? static_cast<const T*>(A->wplane) : nullptr;
  p.acc = acc_at(A, 0);
  if (e == cudaSuccess) e = kss::launch_adj_objective<T>(p, s);
  return e;
}

// The launches of the reverse sweep on stream s (from the seed lam[0] the forward pass
// leaves), ending with the projection on rho0 and the tau accumulator.
template <class T>
cudaError_t backward_launches(kss_adjoint* A, cudaStream_t s) {
  const int N = A->cfg.nsteps, E = A->cfg.checkpoint_every;
  int lc = 0;
  kss::AdjParams<T> p = adj_params<T>(A);
  p.acc = acc_at(A, 1);
  cudaError_t e = cudaSuccess;
  // segments [s0, last] of the states f^0 .. f^{N-2} that the reverse sweep needs,
  // last segment first (i = 0, 1, ...); slot 0 of a segment is its checkpoint, its other
  // states are in seg[i & 1]: the last segment's from the forward pass, each other one
  // recomputed -- by the previous segment's cooperative launch (fused), or by plain steps
  // before its own reverse steps
  const bool fused = A->multi && A->multi_ctas > 0;
  const dim3 g = kss::adj_grid(A->cfg.nx, A->cfg.ny, A->adj_rows);
  const dim3 fg = plain_grid<T>(A);
  const int nblocks = int(g.x * g.y), fnblocks = int(fg.x * fg.y);
  auto segbuf = [&](int i) { return (i & 1) ? A->seg2 : A->seg; };
  int i = 0;
  for (int s0 = last_segment(A); s0 >= 0 && e == cudaSuccess; s0 -= E, ++i) {
    const int last = std::min(s0 + E - 1, N - 2);
    unsigned char* sb = segbuf(i);
    auto state = [&](int k) -> const void* {
      return k == s0 ? static_cast<const void*>(state_at(A, A->ck, s0 / E))
                     : static_cast<const void*>(state_at(A, sb, k - s0));
    };
    if (i > 0 && !fused)
      for (int k = s0 + 1; k <= last && e == cudaSuccess; ++k)
        e = plain_step<T>(A, state(k - 1), const_cast<void*>(state(k)), s);
    if (fused && e == cudaSuccess) {
      // the segment's reverse steps in one cooperative launch (adj_multi_kernel), which
      // also recomputes the previous segment [s0 - E, s0 - 1] into seg[(i + 1) & 1]
      const int nit = last - s0 + 1;
      kss::AdjMulti<T> m{};
      m.ck = static_cast<const T*>(state(s0));
      m.seg = reinterpret_cast<const T*>(sb);
      m.state_elems = (long long)(A->state_bytes / A->esz);
      m.lam0 = reinterpret_cast<const T*>(A->lam[0]);
      m.lam1 = reinterpret_cast<const T*>(A->lam[1]);
      m.done = A->mcount;
      m.ticket = A->mcount + nblocks;
      m.work = A->mcount + nblocks + A->cfg.checkpoint_every;
      m.fdone = m.work + 1;
      m.part = A->mpart;
      m.totals = A->mtot;
      m.err = reinterpret_cast<uint32_t*>(A->small + 128);
      m.deadline = 2000000000LL;  // about a second at 2 GHz
      m.s0 = s0;
      m.last = last;
      m.lc = lc;
      m.gx = int(g.x);
      m.gy = int(g.y);
      m.nblocks = nblocks;
      if (s0 > 0) {
        unsigned char* nb = segbuf(i + 1);
        m.fp = plain_params<T>(A, nullptr, nullptr);
        m.fck = reinterpret_cast<const T*>(state_at(A, A->ck, s0 / E - 1));
        m.fseg = reinterpret_cast<T*>(nb);
        m.fsteps = E - 1;
        m.fgx = int(fg.x);
        m.fgy = int(fg.y);
        m.fnblocks = fnblocks;
      }
      e = cudaMemsetAsync(A->mcount, 0,
                          sizeof(uint32_t) * (size_t(nblocks) + A->cfg.checkpoint_every + 1 +
                                              size_t(fnblocks)),
                          s);
      const int items = nit * nblocks + m.fsteps * m.fnblocks;
      const int ctas = std::min(A->multi_ctas, items);
      if (e == cudaSuccess) e = kss::launch_adj_multi<T>(p, m, ctas, p.acc, s);
      lc ^= nit & 1;
      continue;
    }
    for (int k = last; k >= s0 && e == cudaSuccess; --k) {
      p.f = static_cast<const T*>(state(k));
      p.lam_in = reinterpret_cast<const T*>(A->lam[lc]);
      p.lam_out = reinterpret_cast<T*>(A->lam[lc ^ 1]);
      e = kss::launch_adj_step<T>(p, s);
      lc ^= 1;
    }
  }
  const size_t n = size_t(A->cfg.nx) * A->cfg.ny;
  p.lam_in = reinterpret_cast<const T*>(A->lam[lc]);
  p.ux0 = A->fields + n;
  p.uy0 = A->fields + 2 * n;
  p.grad = A->grad;
  if (e == cudaSuccess) e = kss::launch_adj_final<T>(p, s);
  return e;
}

// Replay the graph of fn's launches (recorded when tau or the weight option changed).
template <class F>
int run_graph(kss_adjoint* A, cudaGraphExec_t* exec, F&& fn) {
  if (A->g_tau != A->tau || A->g_weight != int(A->have_weight)) {
    for (cudaGraphExec_t* g : {&A->g_fwd, &A->g_bwd})
      if (*g) {
        cudaGraphExecDestroy(*g);
        *g = nullptr;
      }
    A->g_tau = A->tau;
    A->g_weight = int(A->have_weight);
  }
  if (!*exec) {
    if (!A->cap) KSS_ACUDA(A, cudaStreamCreateWithFlags(&A->cap, cudaStreamNonBlocking));
    KSS_ACUDA(A, cudaStreamBeginCapture(A->cap, cudaStreamCaptureModeThreadLocal));
    const cudaError_t le = fn(A->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(A->cap, &graph);
    if (le != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return afail(A, KSS_ERR_CUDA, std::string("graph capture: ") +
                                        cudaGetErrorString(le != cudaSuccess ? le : ee));
    }
    const cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    KSS_ACUDA(A, ie);
  }
  KSS_ACUDA(A, cudaGraphLaunch(*exec, A->stream));
  return KSS_OK;
}

template <class T>
int forward_impl(kss_adjoint* A, double* J) {
  int rc = run_graph(A, &A->g_fwd, [&](cudaStream_t s) { return forward_launches<T>(A, s); });
  if (rc) return rc;
  KSS_ACUDA(A, cudaMemcpyAsync(J, acc_at(A, 0), sizeof(double), cudaMemcpyDeviceToHost, A->stream));
  KSS_ACUDA(A, cudaStreamSynchronize(A->stream));
  A->lam_cur = 0;
  return KSS_OK;
}

template <class T>
int backward_impl(kss_adjoint* A, double* grad_tau) {
  int rc = run_graph(A, &A->g_bwd, [&](cudaStream_t s) { return backward_launches<T>(A, s); });
  if (rc) return rc;
  double s = 0;
  uint32_t err = 0;
  KSS_ACUDA(A, cudaMemcpyAsync(&s, acc_at(A, 1), sizeof(double), cudaMemcpyDeviceToHost, A->stream));
  KSS_ACUDA(A, cudaMemcpyAsync(&err, A->small + 128, sizeof(err), cudaMemcpyDeviceToHost, A->stream));
  KSS_ACUDA(A, cudaStreamSynchronize(A->stream));
  if (err & kss::kErrBounds)
    return afail(A, KSS_ERR_BOUNDS, "a device bounds check failed (debug build)");
  if (err) return afail(A, KSS_ERR_TIMEOUT, "a bounded wait of the reverse sweep ran out");
  if (grad_tau) *grad_tau = s / (A->tau * A->tau);
  return KSS_OK;
}

}  // namespace

extern "C" {

int kss_adjoint_create(const kss_adjoint_config* cfg, kss_adjoint** out) {
  if (!out) return KSS_ERR_ARG;
  *out = nullptr;
  if (!cfg || cfg->nx < 1 || cfg->ny < 1 || cfg->nsteps < 1 || cfg->checkpoint_every < 1)
    return KSS_ERR_ARG;
  if ((long long)cfg->nx * cfg->ny > 0x7fffffffLL) return KSS_ERR_ARG;
  if (cfg->precision != KSS_FP32 && cfg->precision != KSS_FP64) return KSS_ERR_UNSUPPORTED;
  if (cfg->own_stream != 0 && cfg->own_stream != 1) return KSS_ERR_ARG;
  kss_adjoint* A = new (std::nothrow) kss_adjoint();
  if (!A) return KSS_ERR_OOM;
  A->cfg = *cfg;
  A->cfg.checkpoint_every = std::min(cfg->checkpoint_every, cfg->nsteps);
  if (cudaGetDevice(&A->device) != cudaSuccess) {
    cudaGetLastError();
    delete A;
    return KSS_ERR_CUDA;
  }
  A->fp32 = cfg->precision == KSS_FP32;
  A->esz = A->fp32 ? 4 : 8;
  const int align = int(128 / A->esz);
  A->pitch = (cfg->nx + align - 1) / align * align;
  A->plane = (long long)A->pitch * cfg->ny;
  A->state_bytes = 9 * size_t(A->plane) * A->esz;
  A->nck = (cfg->nsteps - 1) / A->cfg.checkpoint_every + 1;
  if (cfg->own_stream) {
    if (cudaStreamCreateWithFlags(&A->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete A;
      return KSS_ERR_CUDA;
    }
    A->own_stream = true;
  } else {
    A->stream = static_cast<cudaStream_t>(cfg->stream);
  }
  const size_t n = size_t(cfg->nx) * cfg->ny;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device) != cudaSuccess) {
    cudaGetLastError();
    nsm = 1;
  }
  A->adj_rows = KSS_ADJ_ROWS ? KSS_ADJ_ROWS : kss::fill_rows(cfg->nx, cfg->ny, 32 * kss::kAdjV, nsm);
  A->step_rows = kss::fill_rows(cfg->nx, cfg->ny, 32 * (A->fp32 ? kss::Vec<float>::N : kss::Vec<double>::N), nsm);
  const dim3 g = kss::adj_grid(cfg->nx, cfg->ny, A->adj_rows);
  const dim3 fg = A->fp32 ? plain_grid<float>(A) : plain_grid<double>(A);
  struct {
    void** p;
    size_t bytes;
  } allocs[] = {
      {reinterpret_cast<void**>(&A->ck), A->state_bytes * size_t(A->nck)},
      {reinterpret_cast<void**>(&A->seg), A->state_bytes * size_t(A->cfg.checkpoint_every)},
      {reinterpret_cast<void**>(&A->seg2), A->state_bytes * size_t(A->cfg.checkpoint_every)},
      {reinterpret_cast<void**>(&A->work[0]), A->state_bytes},
      {reinterpret_cast<void**>(&A->work[1]), A->state_bytes},
      {reinterpret_cast<void**>(&A->lam[0]), A->state_bytes},
      {reinterpret_cast<void**>(&A->lam[1]), A->state_bytes},
      {&A->wplane, size_t(A->plane) * A->esz},
      {reinterpret_cast<void**>(&A->fields), 3 * n * sizeof(double)},
      {reinterpret_cast<void**>(&A->grad), n * sizeof(double)},
      {reinterpret_cast<void**>(&A->part), size_t(g.x) * g.y * sizeof(double)},
      {reinterpret_cast<void**>(&A->small), 256},
      {reinterpret_cast<void**>(&A->mcount),
       sizeof(uint32_t) * (size_t(g.x) * g.y + A->cfg.checkpoint_every + 1 + size_t(fg.x) * fg.y)},
      {reinterpret_cast<void**>(&A->mpart),
       sizeof(double) * size_t(g.x) * g.y * A->cfg.checkpoint_every},
      {reinterpret_cast<void**>(&A->mtot), sizeof(double) * size_t(A->cfg.checkpoint_every)},
  };
  for (auto& a : allocs) {
    if (kss_rt::dev_malloc(a.p, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      free_all(A);
      return KSS_ERR_OOM;
    }
  }
  // zero everything once: the padding of every state stays finite
  for (auto& a : allocs) {
    if (cudaMemsetAsync(*a.p, 0, a.bytes, A->stream) != cudaSuccess) {
      cudaGetLastError();
      free_all(A);
      return KSS_ERR_CUDA;
    }
  }
  if (cudaStreamSynchronize(A->stream) != cudaSuccess) {
    cudaGetLastError();
    free_all(A);
    return KSS_ERR_CUDA;
  }
  A->multi_ctas = A->fp32 ? kss::adj_multi_resident_ctas<float>()
                          : kss::adj_multi_resident_ctas<double>();
  *out = A;
  return KSS_OK;
}

void kss_adjoint_destroy(kss_adjoint* A) { free_all(A); }

int kss_adjoint_set_multistep(kss_adjoint* A, int on) {
  if (!A || (on != 0 && on != 1)) return KSS_ERR_ARG;
  if (A->multi != (on != 0) && A->g_bwd) {  // the recorded reverse sweep is the other form
    cudaGraphExecDestroy(A->g_bwd);
    A->g_bwd = nullptr;
  }
  A->multi = on != 0;
  return KSS_OK;
}

const char* kss_adjoint_last_error(const kss_adjoint* A) { return A ? A->msg.c_str() : "null adjoint"; }

int kss_adjoint_forward(kss_adjoint* A, const double* rho0, const double* ux0, const double* uy0,
                        const double* weight, double tau, int on_device, double* J) {
  const kss_rt::NvtxRange nvtx_range("kss_adjoint_forward");
  if (!A) return KSS_ERR_ARG;
  if (!rho0 || !ux0 || !uy0 || !J) return afail(A, KSS_ERR_ARG, "null pointer");
  if (!(tau > 0.5) || !std::isfinite(tau)) return afail(A, KSS_ERR_ARG, "tau must be > 0.5");
  DeviceGuard g(A->device);
  const size_t n = size_t(A->cfg.nx) * A->cfg.ny;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  KSS_ACUDA(A, cudaMemcpyAsync(A->fields, rho0, n * 8, kind, A->stream));
  KSS_ACUDA(A, cudaMemcpyAsync(A->fields + n, ux0, n * 8, kind, A->stream));
  KSS_ACUDA(A, cudaMemcpyAsync(A->fields + 2 * n, uy0, n * 8, kind, A->stream));
  A->have_weight = weight != nullptr;
  if (weight) {
    // the weights go through the gradient staging buffer into one pitched plane
    KSS_ACUDA(A, cudaMemcpyAsync(A->grad, weight, n * 8, kind, A->stream));
    if (A->fp32)
      KSS_ACUDA(A, kss::launch_dense_to_pitched<float>(A->grad, A->plane, A->pitch, A->cfg.nx,
                                                       A->cfg.ny, 1, static_cast<float*>(A->wplane),
                                                       A->stream));
    else
      KSS_ACUDA(A, kss::launch_dense_to_pitched<double>(A->grad, A->plane, A->pitch, A->cfg.nx,
                                                        A->cfg.ny, 1, static_cast<double*>(A->wplane),
                                                        A->stream));
  }
  A->tau = tau;
  A->have_forward = false;
  const int rc = A->fp32 ? forward_impl<float>(A, J) : forward_impl<double>(A, J);
  if (rc) return rc;
  A->have_forward = true;
  return KSS_OK;
}

int kss_adjoint_backward(kss_adjoint* A, double* grad_rho0, double* grad_tau, int on_device) {
  const kss_rt::NvtxRange nvtx_range("kss_adjoint_backward");
  if (!A) return KSS_ERR_ARG;
  if (!A->have_forward) return afail(A, KSS_ERR_STATE, "backward needs a forward pass");
  DeviceGuard g(A->device);
  // the sweep consumes the seed lt^{N-1}: one backward pass per forward pass
  A->have_forward = false;
  const int rc = A->fp32 ? backward_impl<float>(A, grad_tau) : backward_impl<double>(A, grad_tau);
  if (rc) return rc;
  if (grad_rho0) {
    const size_t n = size_t(A->cfg.nx) * A->cfg.ny;
    KSS_ACUDA(A, cudaMemcpyAsync(grad_rho0, A->grad, n * 8,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 A->stream));
    KSS_ACUDA(A, cudaStreamSynchronize(A->stream));
  }
  return KSS_OK;
}

}  // extern "C"
