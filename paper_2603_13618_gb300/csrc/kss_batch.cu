// kss_batch.cu -- batches of lattices (include/kss.h): one launch of the batched fused
// step per time step over the CTA blocks of every member, CUDA-graph replay of
// multi-step calls, and the autotuner of the work decomposition with its cache file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "runtime.h"

using namespace kss_rt;

namespace {

constexpr int kMaxGraphs = 8;  // cached graph executables per batch

struct Graph {
  int nsteps = 0, par = 0;
  std::string modes;  // mode of each step, one character per step
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct kss_batch {
  int n = 0;
  int device = 0;
  int prec = KSS_FP32;  // every member's precision
  int nsm = 0;
  std::vector<kss_lattice*> mem;
  cudaStream_t stream = nullptr;  // every member's stream
  bool own_stream = false;
  cudaStream_t cap = nullptr;     // graphs are recorded on this stream, replayed on `stream`
  kss_batch_tuning tun{};
  int rows_min = 16;              // smallest valid CTA height: the partials are sized for it
  int max_tile = 8;
  int mode_out = kss::MODE_STD;   // kernel of output steps: MODE_FULL if a member needs all
                                  // sensors (each member then runs its own set)
  bool aar = false;               // some member has the two-relaxation model (AAR kernels,
                                  // one launch per step)
  // device data
  void* table[2] = {nullptr, nullptr};  // StepParams<T>[n]; table[par] reads the stored states
  kss::BatchItem* items = nullptr;
  int nitems = 0;
  size_t items_cap = 0;
  double* part_sum = nullptr;     // per member [nblocks][3] from off[k]
  uint32_t* part_cnt = nullptr;   // per member [nblocks][4] from off[k]
  std::vector<int> base_cur;      // members' cur when the tables were written (par = 0)
  std::vector<long long> off;     // first partial of each member
  std::vector<dim3> grids;        // each member's step grid at the current CTA height
  int par = 0;
  bool tables_valid = false;
  std::vector<Graph> graphs;
  // multi-step launches: workspace sized for the smallest CTA height (a header of counters
  // zeroed before every launch, then the rings of partial sums) and each member's
  // MultiState at the current layout
  void* multi = nullptr;
  size_t multi_head = 0;          // header bytes at the current layout
  kss::MultiState* mtab = nullptr;
  std::string msg;
};

namespace {

int bfail(kss_batch* B, int code, const std::string& m) {
  if (B) B->msg = m;
  return code;
}

#define KSS_BCUDA(B, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return bfail((B), KSS_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

size_t param_bytes(const kss_batch* B) {
  return with_storage(B->prec, [](auto tag) {
    return sizeof(kss::StepParams<typename decltype(tag)::type>);
  });
}

int default_rows(const kss_batch* B) { return std::max(32, B->max_tile); }

constexpr int kMultiRing = 8;                   // partial-sum slots per member
constexpr long long kMultiDeadline = 4000000000LL;  // clock64 cycles per wait, about 2 s

// Bytes of the multi-step workspace for members with nb[k] blocks each: the header
// (work counter; per member its blocks' step counters, ring tickets and slot counters),
// then per member the ring of partial sums and counts and the ring of step sums.
size_t multi_bytes(const std::vector<long long>& nb, size_t* head) {
  long long h = 1, parts = 0;
  for (long long b : nb) {
    h += b + 2 * kMultiRing;
    parts += b;
  }
  const size_t hb = (sizeof(uint32_t) * size_t(h) + 255) / 256 * 256;
  if (head) *head = sizeof(uint32_t) * size_t(h);
  return hb + size_t(kMultiRing) * size_t(parts) * (3 * sizeof(double) + 4 * sizeof(uint32_t)) +
         nb.size() * size_t(kMultiRing) * 3 * (sizeof(double) + sizeof(unsigned long long));
}

// Each member's MultiState at the current layout (its blocks in the workspace).
int write_multi_table(kss_batch* B) {
  std::vector<long long> nb(B->n);
  for (int k = 0; k < B->n; ++k) nb[k] = (long long)B->grids[k].x * B->grids[k].y;
  const size_t total = multi_bytes(nb, &B->multi_head);
  (void)total;
  const int R = kMultiRing;
  unsigned char* w = static_cast<unsigned char*>(B->multi);
  uint32_t* hdr = reinterpret_cast<uint32_t*>(w);
  unsigned char* q = w + (B->multi_head + 255) / 256 * 256;
  long long parts = 0;
  for (long long b : nb) parts += b;
  double* psum = reinterpret_cast<double*>(q);
  uint32_t* pcnt = reinterpret_cast<uint32_t*>(q + sizeof(double) * 3 * size_t(R) * size_t(parts));
  double* rsum = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(pcnt) +
                                           sizeof(uint32_t) * 4 * size_t(R) * size_t(parts));
  unsigned long long* rcnt = reinterpret_cast<unsigned long long*>(rsum + 3 * size_t(R) * B->n);
  std::vector<kss::MultiState> tab(B->n);
  uint32_t* next = hdr + 1;
  long long poff = 0;
  for (int k = 0; k < B->n; ++k) {
    kss::MultiState& m = tab[k];
    m.work = hdr;
    m.done = next;
    m.ticket = next + nb[k];
    m.fin = m.ticket + R;
    next = m.fin + R;
    m.part_sum = psum + 3 * size_t(R) * size_t(poff);
    m.part_cnt = pcnt + 4 * size_t(R) * size_t(poff);
    poff += nb[k];
    m.ring_sums = rsum + 3 * size_t(R) * k;
    m.ring_counts = rcnt + 3 * size_t(R) * k;
    m.err = B->mem[k]->err_word;
    m.deadline = kMultiDeadline;
    m.ring = R;
    m.nsteps = 0;  // set by the kernel from its argument
    m.gx = int(B->grids[k].x);
    m.gy = int(B->grids[k].y);
    m.nblocks = int(nb[k]);
  }
  KSS_BCUDA(B, cudaMemcpy(B->mtab, tab.data(), sizeof(kss::MultiState) * B->n,
                          cudaMemcpyHostToDevice));
  return KSS_OK;
}

bool valid_rows(const kss_batch* B, int rows) {
  if (rows != 16 && rows != 32 && rows != 64) return false;
  for (const kss_lattice* L : B->mem)
    if (rows % L->cfg.tile != 0) return false;
  return true;
}

dim3 member_grid(const kss_batch* B, const kss_lattice* L, int rows) {
  const int bands = rows / L->cfg.tile;
  return with_storage(B->prec, [&](auto tag) {
    return kss::step_grid<typename decltype(tag)::type>(L->cfg.nx, L->cfg.ny, L->cfg.tile, bands);
  });
}

void drop_graphs(kss_batch* B) {
  for (Graph& g : B->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  B->graphs.clear();
}

// Work list at the current CTA height: members by decreasing size (the largest lists
// first, so that the small ones fill the last wave), each member's blocks in its own
// block order (by, bx).
int write_items(kss_batch* B) {
  const int rows = B->tun.rows;
  std::vector<int> order(B->n);
  for (int k = 0; k < B->n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const kss_lattice* A = B->mem[a];
    const kss_lattice* C = B->mem[b];
    return (long long)A->cfg.nx * A->cfg.ny > (long long)C->cfg.nx * C->cfg.ny;
  });
  B->grids.assign(B->n, dim3());
  B->off.assign(B->n, 0);
  long long total = 0;
  for (int k = 0; k < B->n; ++k) {
    B->grids[k] = member_grid(B, B->mem[k], rows);
    B->off[k] = total;
    total += (long long)B->grids[k].x * B->grids[k].y;
  }
  if (total > 0x7fffffffLL) return bfail(B, KSS_ERR_ARG, "batch work list too long");
  std::vector<kss::BatchItem> host;
  host.reserve(size_t(total));
  for (int k : order)
    for (unsigned by = 0; by < B->grids[k].y; ++by)
      for (unsigned bx = 0; bx < B->grids[k].x; ++bx) host.push_back({uint32_t(k), bx, by, 0u});
  if (host.size() > B->items_cap) {
    drop_graphs(B);  // graphs hold the old list's address
    KSS_BCUDA(B, cudaStreamSynchronize(B->stream));
    if (B->items) kss_rt::dev_free(B->items);
    B->items = nullptr;
    B->items_cap = 0;
    if (kss_rt::dev_malloc(&B->items, host.size() * sizeof(kss::BatchItem)) != cudaSuccess) {
      cudaGetLastError();
      return bfail(B, KSS_ERR_OOM, "work list allocation failed");
    }
    B->items_cap = host.size();
  }
  // pageable source: the copy completes before the call returns
  KSS_BCUDA(B, cudaMemcpy(B->items, host.data(), host.size() * sizeof(kss::BatchItem),
                          cudaMemcpyHostToDevice));
  B->nitems = int(host.size());
  return KSS_OK;
}

template <class S>
void fill_params(const kss_batch* B, std::vector<kss::StepParams<S>>& t0,
                 std::vector<kss::StepParams<S>>& t1) {
  t0.resize(B->n);
  t1.resize(B->n);
  for (int k = 0; k < B->n; ++k) {
    const kss_lattice* L = B->mem[k];
    const int c = L->cur;
    for (int o = 0; o < 2; ++o) {
      kss::StepParams<S> p = make_params<S>(L, L->f[c ^ o], L->f[c ^ o ^ 1]);
      p.bands = B->tun.rows / L->cfg.tile;
      p.grid_x = int(B->grids[k].x);
      p.nblocks = int(B->grids[k].x * B->grids[k].y);
      p.part_sum = B->part_sum + 3 * B->off[k];
      p.part_cnt = B->part_cnt + 4 * B->off[k];
      p.mode = mode_for(needed_mask(L, L->cfg.record_mask));
      (o == 0 ? t0 : t1)[k] = p;
    }
  }
}

// Both orientations of every member's parameters: table[0] reads each member's stored
// state, table[1] the other buffer.
int write_tables(kss_batch* B) {
  const size_t bytes = param_bytes(B) * B->n;
  const cudaError_t e = with_storage(B->prec, [&](auto tag) {
    using S = typename decltype(tag)::type;
    std::vector<kss::StepParams<S>> t0, t1;
    fill_params<S>(B, t0, t1);
    cudaError_t r = cudaMemcpy(B->table[0], t0.data(), bytes, cudaMemcpyHostToDevice);
    if (r == cudaSuccess) r = cudaMemcpy(B->table[1], t1.data(), bytes, cudaMemcpyHostToDevice);
    return r;
  });
  KSS_BCUDA(B, e);
  for (int k = 0; k < B->n; ++k) B->base_cur[k] = B->mem[k]->cur;
  B->par = 0;
  B->tables_valid = true;
  return KSS_OK;
}

// Re-derive the work list and tables after a tuning change.
int relayout(kss_batch* B) {
  // the tables and work list are read by launches still in flight
  KSS_BCUDA(B, cudaStreamSynchronize(B->stream));
  drop_graphs(B);
  int rc = write_items(B);
  if (rc) return rc;
  if ((rc = write_multi_table(B))) return rc;
  return write_tables(B);
}

// Tables still describe the members (a member stepped on its own flips its buffers)?
int check_tables(kss_batch* B) {
  bool ok = B->tables_valid;
  for (int k = 0; ok && k < B->n; ++k) ok = B->mem[k]->cur == (B->base_cur[k] ^ B->par);
  if (ok) return KSS_OK;
  KSS_BCUDA(B, cudaStreamSynchronize(B->stream));
  return write_tables(B);
}

int launch_ctas(const kss_batch* B) {
  if (B->tun.ctas_per_sm <= 0) return B->nitems;
  return std::min<long long>(B->nitems, (long long)B->tun.ctas_per_sm * B->nsm);
}

// All nsteps {Kn, KL, neq} steps of the batch in one cooperative launch.
cudaError_t launch_multi(kss_batch* B, int nsteps) {
  cudaError_t e = cudaMemsetAsync(B->multi, 0, B->multi_head, B->stream);
  if (e != cudaSuccess) return e;
  return with_storage(B->prec, [&](auto tag) {
    using S = typename decltype(tag)::type;
    const int resident = kss::batch_multi_resident_ctas<S>(kss::MODE_STD);
    if (resident < 1) return cudaErrorInvalidConfiguration;
    const long long work = (long long)nsteps * B->nitems;
    const int ctas = int(std::min<long long>(resident, work));
    const auto* t = static_cast<const kss::StepParams<S>*>(B->table[B->par]);
    const auto* u = static_cast<const kss::StepParams<S>*>(B->table[B->par ^ 1]);
    return kss::launch_batch_multi<S>(t, u, B->mtab, B->items, B->nitems, nsteps,
                                      static_cast<uint32_t*>(B->multi), kss::MODE_STD, ctas,
                                      B->stream);
  });
}

cudaError_t launch_one(kss_batch* B, int tbl, int mode, cudaStream_t s) {
  const int ctas = launch_ctas(B);
  return with_storage(B->prec, [&](auto tag) {
    using S = typename decltype(tag)::type;
    return kss::launch_batch_step<S>(static_cast<const kss::StepParams<S>*>(B->table[tbl]),
                                     B->items, B->nitems, ctas, mode, s, B->aar);
  });
}

char mode_char(int mode) { return mode == kss::MODE_PLAIN ? 'P' : (mode == kss::MODE_STD ? 'S' : 'F'); }
int char_mode(char c) { return c == 'P' ? kss::MODE_PLAIN : (c == 'S' ? kss::MODE_STD : kss::MODE_FULL); }

int graph_for(kss_batch* B, int nsteps, const std::string& modes, cudaGraphExec_t* out) {
  for (Graph& g : B->graphs) {
    if (g.nsteps == nsteps && g.par == B->par && g.modes == modes) {
      *out = g.exec;
      return KSS_OK;
    }
  }
  KSS_BCUDA(B, cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < nsteps && le == cudaSuccess; ++s)
    le = launch_one(B, B->par ^ (s & 1), char_mode(modes[s]), B->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(B->cap, &graph);
  if (le != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return bfail(B, KSS_ERR_CUDA, std::string("graph capture: ") +
                                      cudaGetErrorString(le != cudaSuccess ? le : ee));
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    return bfail(B, KSS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
  }
  if ((int)B->graphs.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(B->graphs.front().exec);
    B->graphs.erase(B->graphs.begin());
  }
  Graph g;
  g.nsteps = nsteps;
  g.par = B->par;
  g.modes = modes;
  g.exec = exec;
  B->graphs.push_back(g);
  *out = exec;
  return KSS_OK;
}

void destroy_batch(kss_batch* B) {
  if (!B) return;
  DeviceGuard g(B->device);
  cudaStreamSynchronize(B->stream);
  drop_graphs(B);
  for (kss_lattice* L : B->mem) {
    if (!L) continue;
    L->owner = nullptr;
    L->own_stream = false;  // the batch owns the shared stream
    release(L);
  }
  void* bufs[] = {B->table[0], B->table[1], B->items, B->part_sum, B->part_cnt, B->multi,
                  B->mtab};
  for (void* b : bufs)
    if (b) kss_rt::dev_free(b);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

// ---- autotuner cache: "key<TAB>rows<TAB>ctas_per_sm<TAB>ms<TAB>multi_step" lines (a
// line without the last field is a per-step choice).  The key ends with a hash of the
// CUDA sources and build flags of this library, so entries measured on other kernels
// are never reused. ----
#ifndef KSS_SOURCE_HASH
#define KSS_SOURCE_HASH "unhashed"
#endif
constexpr const char* kSourceHash = KSS_SOURCE_HASH;
std::string tune_key(const kss_batch* B) {
  cudaDeviceProp prop{};
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, B->device) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == '\t' || c == '\n' || c == '|') c = ' ';
  long long cells = 0;
  for (const kss_lattice* L : B->mem) cells += (long long)L->cfg.nx * L->cfg.ny;
  const int lc = int(std::lround(std::log2(double(std::max(1LL, cells)))));
  const int ln = int(std::lround(std::log2(double(B->n))));
  return name + "|" + std::to_string(B->nsm) + "|" + (B->prec == KSS_FP64 ? "fp64" : (B->prec == KSS_FP32 ? "fp32" : "fp16dev")) + "|" +
         std::to_string(lc) + "|" + std::to_string(ln) + "|" + kSourceHash;
}

bool cache_lookup(const char* path, const std::string& key, kss_batch_tuning* t) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    char* tab = std::strchr(line, '\t');
    if (!tab) continue;
    if (std::string(line, tab - line) != key) continue;
    int rows = 0, cps = 0, multi = 0;
    double ms = 0;
    const int got = std::sscanf(tab + 1, "%d\t%d\t%lf\t%d", &rows, &cps, &ms, &multi);
    if (got >= 3) {
      t->rows = rows;
      t->ctas_per_sm = cps;
      t->ms_per_step = ms;
      t->multi_step = got == 4 ? (multi != 0) : 0;
      found = true;  // the last entry for a key wins
    }
  }
  std::fclose(f);
  return found;
}

void cache_append(const char* path, const std::string& key, const kss_batch_tuning& t) {
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s\t%d\t%d\t%.9g\t%d\n", key.c_str(), t.rows, t.ctas_per_sm, t.ms_per_step,
               t.multi_step);
  std::fclose(f);
}

}  // namespace

extern "C" {

int kss_batch_create(int32_t n, const kss_config* cfgs, kss_batch** out) {
  if (!out) return KSS_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !cfgs) return KSS_ERR_ARG;
  for (int k = 1; k < n; ++k)
    if (cfgs[k].precision != cfgs[0].precision) return KSS_ERR_ARG;
  // a batched step is an output step for every member when it is one for any, and an
  // AAR member's output steps rewrite its region: with AAR members, one shared cadence
  bool any_aar = false;
  for (int k = 0; k < n; ++k) any_aar = any_aar || cfgs[k].tau2 != 0.0;
  for (int k = 1; any_aar && k < n; ++k)
    if (cfgs[k].output_every != cfgs[0].output_every) return KSS_ERR_UNSUPPORTED;
  kss_batch* B = new (std::nothrow) kss_batch();
  if (!B) return KSS_ERR_OOM;
  B->n = n;
  B->prec = cfgs[0].precision;
  if (cudaGetDevice(&B->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess) {
    cudaGetLastError();
    delete B;
    return KSS_ERR_CUDA;
  }
  if (cfgs[0].own_stream) {
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete B;
      return KSS_ERR_CUDA;
    }
    B->own_stream = true;
  } else {
    B->stream = static_cast<cudaStream_t>(cfgs[0].stream);
  }
  if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    destroy_batch(B);
    return KSS_ERR_CUDA;
  }
  B->mem.assign(n, nullptr);
  for (int k = 0; k < n; ++k) {
    kss_config c = cfgs[k];
    c.stream = B->stream;
    c.own_stream = 0;
    const int rc = kss_create(&c, &B->mem[k]);
    if (rc) {
      destroy_batch(B);
      return rc;
    }
    B->mem[k]->owner = B;
    if (c.tau2 > 0.0) B->aar = true;
    B->max_tile = std::max(B->max_tile, c.tile);
    if (mode_for(needed_mask(B->mem[k], c.record_mask)) == kss::MODE_FULL) B->mode_out = kss::MODE_FULL;
  }
  B->rows_min = std::max(16, B->max_tile);
  B->tun.rows = default_rows(B);
  B->tun.ctas_per_sm = 0;
  B->tun.graph = 1;
  B->tun.ms_per_step = 0;
  B->tun.multi_step = 1;
  B->base_cur.assign(n, 0);
  // partials for the smallest CTA height any tuning may choose
  long long parts = 0;
  std::vector<long long> nb_max;
  for (const kss_lattice* L : B->mem) {
    const dim3 g = member_grid(B, L, B->rows_min);
    parts += (long long)g.x * g.y;
    nb_max.push_back((long long)g.x * g.y);
  }
  const size_t pb = param_bytes(B) * size_t(n);
  struct {
    void** p;
    size_t bytes;
  } allocs[] = {
      {&B->table[0], pb},
      {&B->table[1], pb},
      {reinterpret_cast<void**>(&B->part_sum), sizeof(double) * 3 * size_t(parts)},
      {reinterpret_cast<void**>(&B->part_cnt), sizeof(uint32_t) * 4 * size_t(parts)},
      {&B->multi, multi_bytes(nb_max, nullptr)},
      {reinterpret_cast<void**>(&B->mtab), sizeof(kss::MultiState) * size_t(n)},
  };
  for (auto& a : allocs) {
    if (kss_rt::dev_malloc(a.p, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      destroy_batch(B);
      return KSS_ERR_OOM;
    }
  }
  const int rc = relayout(B);
  if (rc) {
    destroy_batch(B);
    return rc;
  }
  *out = B;
  return KSS_OK;
}

void kss_batch_destroy(kss_batch* B) { destroy_batch(B); }

kss_lattice* kss_batch_member(kss_batch* B, int32_t k) {
  if (!B || k < 0 || k >= B->n) return nullptr;
  return B->mem[k];
}

const char* kss_batch_last_error(const kss_batch* B) { return B ? B->msg.c_str() : "null batch"; }

int kss_batch_get_tuning(const kss_batch* B, kss_batch_tuning* t) {
  if (!B || !t) return KSS_ERR_ARG;
  *t = B->tun;
  return KSS_OK;
}

int kss_batch_set_tuning(kss_batch* B, const kss_batch_tuning* t) {
  if (!B || !t) return KSS_ERR_ARG;
  const int rows = t->rows == 0 ? default_rows(B) : t->rows;
  if (!valid_rows(B, rows)) return bfail(B, KSS_ERR_ARG, "rows must be 16, 32 or 64 and a multiple of every tile");
  if (t->ctas_per_sm < 0 || t->ctas_per_sm > 64) return bfail(B, KSS_ERR_ARG, "ctas_per_sm out of range");
  if (t->graph != 0 && t->graph != 1) return bfail(B, KSS_ERR_ARG, "graph must be 0 or 1");
  if (t->multi_step != 0 && t->multi_step != 1)
    return bfail(B, KSS_ERR_ARG, "multi_step must be 0 or 1");
  DeviceGuard g(B->device);
  const bool layout = rows != B->tun.rows || t->ctas_per_sm != B->tun.ctas_per_sm;
  B->tun.rows = rows;
  B->tun.ctas_per_sm = t->ctas_per_sm;
  B->tun.graph = t->graph;
  B->tun.multi_step = t->multi_step;
  return layout ? relayout(B) : KSS_OK;
}

int kss_batch_step(kss_batch* B, int32_t nsteps) {
  const kss_rt::NvtxRange nvtx_range("kss_batch_step");
  if (!B) return KSS_ERR_ARG;
  if (nsteps < 0) return bfail(B, KSS_ERR_ARG, "negative step count");
  for (kss_lattice* L : B->mem) {
    const int rc = enter(L);
    if (rc) return rc;
  }
  if (nsteps == 0) return KSS_OK;
  if (B->aar) {
    // the output steps of AAR members must be theirs: members in phase
    const int every = B->mem[0]->cfg.output_every;
    for (const kss_lattice* L : B->mem)
      if (every > 1 && L->step % every != B->mem[0]->step % every)
        return bfail(B, KSS_ERR_STATE, "members with the two-relaxation model are out of "
                                       "phase with the batch's output steps");
  }
  DeviceGuard g(B->device);
  int rc = check_tables(B);
  if (rc) return rc;
  std::string modes(size_t(nsteps), 'P');
  for (int s = 0; s < nsteps; ++s) {
    for (const kss_lattice* L : B->mem) {
      const int every = L->cfg.output_every;
      if (every > 0 && (L->step + s + 1) % every == 0) {
        modes[s] = mode_char(B->mode_out);
        break;
      }
    }
  }
  const bool all_std = B->mode_out == kss::MODE_STD && !B->aar &&
                       modes.find_first_not_of('S') == std::string::npos;
  if (B->tun.multi_step && nsteps >= 2 && all_std &&
      (long long)nsteps * B->nitems < (1LL << 30)) {
    KSS_BCUDA(B, launch_multi(B, nsteps));
  } else if (B->tun.graph && nsteps >= 2) {
    cudaGraphExec_t exec = nullptr;
    if ((rc = graph_for(B, nsteps, modes, &exec))) return rc;
    KSS_BCUDA(B, cudaGraphLaunch(exec, B->stream));
  } else {
    for (int s = 0; s < nsteps; ++s)
      KSS_BCUDA(B, launch_one(B, B->par ^ (s & 1), char_mode(modes[s]), B->stream));
  }
  for (kss_lattice* L : B->mem) {
    for (int s = 0; s < nsteps; ++s) {
      L->cur ^= 1;
      L->step += 1;
      if (modes[s] != 'P') L->out_step = L->rec_step = L->step;
    }
  }
  B->par ^= nsteps & 1;
  return KSS_OK;
}

int kss_batch_autotune(kss_batch* B, const char* cache_path, int32_t steps,
                       kss_batch_tuning* chosen) {
  if (!B) return KSS_ERR_ARG;
  if (steps < 1 || steps > 100000) return bfail(B, KSS_ERR_ARG, "steps out of range");
  for (kss_lattice* L : B->mem) {
    const int rc = enter(L);
    if (rc) return rc;
    if (L->step != 0) return bfail(B, KSS_ERR_STATE, "autotune needs every member at step 0");
  }
  DeviceGuard g(B->device);
  const std::string key = tune_key(B);
  kss_batch_tuning best = B->tun;
  int rc = KSS_OK;
  // multi-step launches are timed too when the members' steps qualify for them (every
  // member an output step of the {Kn, KL, neq} set every step) and they are enabled
  bool multi_ok = B->tun.multi_step && B->mode_out == kss::MODE_STD && !B->aar;
  for (const kss_lattice* L : B->mem) multi_ok = multi_ok && L->cfg.output_every == 1;
  if (cache_path && cache_lookup(cache_path, key, &best) && valid_rows(B, best.rows) &&
      best.ctas_per_sm >= 0 && best.ctas_per_sm <= 64) {
    best.graph = B->tun.graph;
    if (!multi_ok) best.multi_step = B->tun.multi_step;
    const double ms = best.ms_per_step;
    if ((rc = kss_batch_set_tuning(B, &best))) return rc;
    B->tun.ms_per_step = ms;
    if (chosen) *chosen = B->tun;
    return KSS_OK;
  }
  if ((rc = check_tables(B))) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KSS_BCUDA(B, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaGetLastError();
    return bfail(B, KSS_ERR_CUDA, "cudaEventCreate failed");
  }
  const int rows_c[] = {16, 32, 64};
  const int cps_c[] = {0, 2, 3, 4};
  best.ms_per_step = -1;
  for (int rows : rows_c) {
    if (!valid_rows(B, rows)) continue;
    for (int cps : cps_c) {
      kss_batch_tuning t = B->tun;
      t.rows = rows;
      t.ctas_per_sm = cps;
      if (multi_ok) t.multi_step = 0;  // these are per-step launches
      if ((rc = kss_batch_set_tuning(B, &t))) break;
      // every launch reads the stored states (table[par]) and writes the other buffers
      cudaError_t e = cudaSuccess;
      for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_one(B, B->par, B->mode_out, B->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, B->stream);
      for (int s = 0; s < steps && e == cudaSuccess; ++s) e = launch_one(B, B->par, B->mode_out, B->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, B->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rc = bfail(B, KSS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        break;
      }
      const double per = double(ms) / steps;
      if (best.ms_per_step < 0 || per < best.ms_per_step) {
        best = t;
        best.ms_per_step = per;
      }
    }
    if (rc) break;
  }
  if (!rc && multi_ok) {
    // a multi-step launch advances the states: keep every member's stored state aside
    size_t total = 0;
    for (const kss_lattice* L : B->mem) total += 9 * size_t(L->plane) * L->esz;
    unsigned char* snap = nullptr;
    if (kss_rt::dev_malloc(&snap, total) != cudaSuccess) {
      cudaGetLastError();
      rc = bfail(B, KSS_ERR_OOM, "autotune: state snapshot allocation failed");
    }
    size_t o = 0;
    for (kss_lattice* L : B->mem) {
      if (rc) break;
      const size_t bytes = 9 * size_t(L->plane) * L->esz;
      if (cudaMemcpyAsync(snap + o, L->f[L->cur], bytes, cudaMemcpyDeviceToDevice, B->stream) !=
          cudaSuccess)
        rc = bfail(B, KSS_ERR_CUDA, "autotune: state snapshot copy failed");
      o += bytes;
    }
    for (int rows : rows_c) {
      if (rc || !valid_rows(B, rows)) continue;
      kss_batch_tuning t = B->tun;
      t.rows = rows;
      t.ctas_per_sm = 0;
      t.multi_step = 1;
      if ((rc = kss_batch_set_tuning(B, &t))) break;
      cudaError_t e = launch_multi(B, 2);
      if (e == cudaSuccess) e = cudaEventRecord(e0, B->stream);
      if (e == cudaSuccess) e = launch_multi(B, std::max(2, int(steps)));
      if (e == cudaSuccess) e = cudaEventRecord(e1, B->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rc = bfail(B, KSS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        break;
      }
      const double per = double(ms) / std::max(2, int(steps));
      if (best.ms_per_step < 0 || per < best.ms_per_step) {
        best = t;
        best.ms_per_step = per;
      }
    }
    if (snap) {
      o = 0;
      for (kss_lattice* L : B->mem) {
        const size_t bytes = 9 * size_t(L->plane) * L->esz;
        if (cudaMemcpyAsync(L->f[L->cur], snap + o, bytes, cudaMemcpyDeviceToDevice,
                            B->stream) != cudaSuccess && !rc)
          rc = bfail(B, KSS_ERR_CUDA, "autotune: state restore failed");
        o += bytes;
      }
      cudaStreamSynchronize(B->stream);
      kss_rt::dev_free(snap);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timed launches overwrote every member's outputs of its current step
  for (kss_lattice* L : B->mem) L->out_step = L->rec_step = -1;
  if (rc) return rc;
  const double ms = best.ms_per_step;
  if ((rc = kss_batch_set_tuning(B, &best))) return rc;
  B->tun.ms_per_step = ms;
  if (cache_path) cache_append(cache_path, key, B->tun);
  if (chosen) *chosen = B->tun;
  return KSS_OK;
}

}  // extern "C"
