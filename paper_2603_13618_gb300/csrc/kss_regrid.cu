// kss_regrid.cu -- regrid steps (1)-(2) on the GPU (include/kss.h): the tagging tiles
// within `buffer` cells of a refine-flagged cell are marked, and the marked tiles are
// clustered into rectangular boxes by the signature method of Berger & Rigoutsos (the
// clustering the paper's regridding routine cites, section "Adaptive refinement and
// parallel processing"), breadth first: each level of boxes is clustered by CTAs striding
// over its boxes, and the host checks the level sizes every few levels.
//
// Clustering rules (all integer except one efficiency comparison in FP64), for a box:
//   1. signatures sx[i] = marked tiles of column i, sy[j] = of row j;
//   2. no mark: drop; else shrink to the bounding box of the marks;
//   3. accept if marks >= efficiency * area (FP64), or if the box is a single tile;
//   4. else cut at the interior hole (zero signature) nearest the centre (ties: x before
//      y, lower index first), leaving the hole out of both halves;
//   5. else at the strongest inflection of d[i] = s[i-1] - 2 s[i] + s[i+1]: a cut between
//      i and i+1 with d[i] d[i+1] < 0, strength |d[i+1] - d[i]| (ties: cut nearest the
//      centre, then x before y, then lower index);
//   6. else bisect the longer side (x if equal) at x0 + w / 2.
// Children of a level enter the next level in order (lower half first); accepted boxes
// are appended level by level in list order, so the result is deterministic.
#include <algorithm>
#include <cstdint>
#include <new>
#include <string>

#include "runtime.h"

using namespace kss_rt;

namespace {

constexpr int kMaxSide = 8192;  // tiles per side (signatures live in shared memory)

struct Box {
  int x0, y0, x1, y1;
};

// ---- kernels ----

// mask[ty][tx] = 1 if a cell within `buffer` cells (periodic) of tile (tx, ty) has the
// refine flag.  One thread per tile.
__global__ void tile_mask_kernel(const uint8_t* __restrict__ flags, long long pitch, int nx,
                                 int ny, int tile, int buffer, int ntx, int nty,
                                 uint8_t* __restrict__ mask) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)ntx * nty) return;
  const int ty = int(t / ntx), tx = int(t - (long long)ty * ntx);
  const int ya = ty * tile - buffer, yb = min((ty + 1) * tile, ny) + buffer;
  const int xa = tx * tile - buffer, xb = min((tx + 1) * tile, nx) + buffer;
  uint8_t any = 0;
  for (int y = ya; y < yb && !any; ++y) {
    const int yy = ((y % ny) + ny) % ny;
    const uint8_t* row = flags + (long long)yy * pitch;
    for (int x = xa; x < xb; ++x) {
      const int xx = ((x % nx) + nx) % nx;
      if (row[xx] & 1u) {
        any = 1;
        break;
      }
    }
  }
  mask[t] = any;
}

// Prefix sums of the mask: pc[j][i] = marked tiles of column i in rows < j ((nty + 1) x
// ntx), pr[j][i] = of row j in columns < i (nty x (ntx + 1)).  One thread per column,
// then one per row.
__global__ void mask_prefix_kernel(const uint8_t* __restrict__ mask, int ntx, int nty,
                                   int* __restrict__ pc, int* __restrict__ pr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntx) {
    int acc = 0;
    for (int j = 0; j < nty; ++j) {
      pc[(long long)j * ntx + t] = acc;
      acc += mask[(long long)j * ntx + t];
    }
    pc[(long long)nty * ntx + t] = acc;
  } else if (t < ntx + nty) {
    const int j = t - ntx;
    int acc = 0;
    const uint8_t* row = mask + (long long)j * ntx;
    int* out = pr + (long long)j * (ntx + 1);
    for (int i = 0; i < ntx; ++i) {
      out[i] = acc;
      acc += row[i];
    }
    out[ntx] = acc;
  }
}

__device__ __forceinline__ int tile_key(int i, int lo, int hi) { return abs(2 * i - (lo + hi - 1)); }
__device__ __forceinline__ int cut_key(int i, int lo, int hi) { return abs(2 * i - (lo + hi)); }

// The boxes of one level, *count of them (written by the previous compaction), CTAs
// striding over them.  acc[i]: box i accepted (shrunk) or x0 = -1; kids[2i], kids[2i+1]:
// its two halves or x0 = -1.
__device__ __forceinline__ void cluster_box(const int* __restrict__ pc,
                                            const int* __restrict__ pr, int ntx, Box b, int bi,
                                            double efficiency, Box* __restrict__ acc,
                                            Box* __restrict__ kids, int* sig);

__global__ void __launch_bounds__(256) cluster_level_kernel(const int* __restrict__ pc,
                                                            const int* __restrict__ pr,
                                                            int ntx, const Box* __restrict__ in,
                                                            const int* __restrict__ count,
                                                            const double* __restrict__ eff,
                                                            Box* __restrict__ acc,
                                                            Box* __restrict__ kids) {
  extern __shared__ int sig[];  // sx[w] then sy[h]
  const int n = *count;
  const double efficiency = *eff;
  for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
    cluster_box(pc, pr, ntx, in[bi], bi, efficiency, acc, kids, sig);
    __syncthreads();  // the signatures are reused by the next box
  }
}

__device__ __forceinline__ void cluster_box(const int* __restrict__ pc,
                                            const int* __restrict__ pr, int ntx, Box b, int bi,
                                            double efficiency, Box* __restrict__ acc,
                                            Box* __restrict__ kids, int* sig) {
  const int w = b.x1 - b.x0, h = b.y1 - b.y0;
  int* sx = sig;
  int* sy = sig + w;
  // signatures from the prefix sums
  for (int k = threadIdx.x; k < w + h; k += blockDim.x) {
    if (k < w) {
      const int i = b.x0 + k;
      sx[k] = pc[(long long)b.y1 * ntx + i] - pc[(long long)b.y0 * ntx + i];
    } else {
      const long long r = (long long)(b.y0 + k - w) * (ntx + 1);
      sy[k - w] = pr[r + b.x1] - pr[r + b.x0];
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;  // (the caller's barrier follows for every thread)
  const Box none{-1, -1, -1, -1};
  Box out_acc = none, k0 = none, k1 = none;
  long long total = 0;
  int ia = -1, ib = -1, ja = -1, jb = -1;
  for (int i = 0; i < w; ++i) {
    if (sx[i]) {
      if (ia < 0) ia = i;
      ib = i;
      total += sx[i];
    }
  }
  for (int j = 0; j < h; ++j) {
    if (sy[j]) {
      if (ja < 0) ja = j;
      jb = j;
    }
  }
  if (total > 0) {
    // the shrunk box [x0, x1) x [y0, y1) and its signatures sx[ia..ib], sy[ja..jb]
    const int x0 = b.x0 + ia, x1 = b.x0 + ib + 1, y0 = b.y0 + ja, y1 = b.y0 + jb + 1;
    const int sw = x1 - x0, sh = y1 - y0;
    const int* s[2] = {sx + ia, sy + ja};
    const int n[2] = {sw, sh};
    const int lo[2] = {x0, y0}, hi[2] = {x1, y1};
    if (double(total) >= efficiency * double((long long)sw * sh) || (sw == 1 && sh == 1)) {
      out_acc = Box{x0, y0, x1, y1};
    } else {
      int best_axis = -1, best_i = 0, best_k = 0;
      bool hole = false;
      // 4. interior holes
      for (int a = 0; a < 2; ++a) {
        for (int k = 1; k < n[a] - 1; ++k) {
          if (s[a][k] != 0) continue;
          const int i = lo[a] + k, key = tile_key(i, lo[a], hi[a]);
          if (best_axis < 0 || key < best_k) {  // x first, lower index first on ties
            best_axis = a;
            best_i = i;
            best_k = key;
          }
        }
      }
      hole = best_axis >= 0;
      if (!hole) {
        // 5. strongest inflection
        int best_str = -1;
        for (int a = 0; a < 2; ++a) {
          for (int k = 1; k < n[a] - 2; ++k) {
            const int dk = s[a][k - 1] - 2 * s[a][k] + s[a][k + 1];
            const int dk1 = s[a][k] - 2 * s[a][k + 1] + s[a][k + 2];
            if ((long long)dk * dk1 >= 0) continue;
            const int i = lo[a] + k + 1, str = abs(dk1 - dk), key = cut_key(i, lo[a], hi[a]);
            if (best_axis < 0 || str > best_str || (str == best_str && key < best_k)) {
              best_axis = a;
              best_i = i;
              best_str = str;
              best_k = key;
            }
          }
        }
      }
      if (best_axis < 0) {
        // 6. bisection of the longer side
        best_axis = sw >= sh ? 0 : 1;
        best_i = best_axis == 0 ? x0 + sw / 2 : y0 + sh / 2;
      }
      const int skip = hole ? 1 : 0;
      if (best_axis == 0) {
        k0 = Box{x0, y0, best_i, y1};
        k1 = Box{best_i + skip, y0, x1, y1};
      } else {
        k0 = Box{x0, y0, x1, best_i};
        k1 = Box{x0, best_i + skip, x1, y1};
      }
    }
  }
  acc[bi] = out_acc;
  kids[2 * bi] = k0;
  kids[2 * bi + 1] = k1;
}

// Appends the accepted boxes to the result (in order) and compacts the valid children
// into the next level's list.  One CTA of 1024 threads; counts[0] = result size,
// counts[1] = next level size.
__global__ void __launch_bounds__(1024) compact_kernel(const Box* __restrict__ acc,
                                                       const Box* __restrict__ kids,
                                                       Box* __restrict__ result,
                                                       int result_cap, Box* __restrict__ next,
                                                       int* __restrict__ counts) {
  __shared__ int s_warp[32];
  __shared__ int s_base[2];
  __shared__ int s_n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_base[0] = counts[0];
    s_base[1] = 0;
    s_n = counts[1];  // boxes of the level just clustered
  }
  __syncthreads();
  const int n = s_n;
  // two passes of the same block-wide ordered scan: accepted boxes, then children
  for (int pass = 0; pass < 2; ++pass) {
    const Box* src = pass == 0 ? acc : kids;
    const int m = pass == 0 ? n : 2 * n;
    for (int c0 = 0; c0 < m; c0 += blockDim.x) {
      const int c = c0 + threadIdx.x;
      const bool valid = c < m && src[c].x0 >= 0;
      const unsigned bal = __ballot_sync(0xffffffffu, valid);
      if (lane == 0) s_warp[warp] = __popc(bal);
      __syncthreads();
      int before = 0, chunk = 0;
      for (int w2 = 0; w2 < int(blockDim.x >> 5); ++w2) {
        if (w2 < warp) before += s_warp[w2];
        chunk += s_warp[w2];
      }
      const int pos = s_base[pass] + before + __popc(bal & ((1u << lane) - 1u));
      if (valid) {
        if (pass == 0) {
          if (pos < result_cap) result[pos] = src[c];
        } else {
          next[pos] = src[c];
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_base[pass] += chunk;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    counts[0] = s_base[0];
    counts[1] = s_base[1];
  }
}

// ---- host side ----

struct Workspace {
  int cap = 0;            // boxes per level list
  Box* level[2] = {nullptr, nullptr};
  Box* acc = nullptr;     // [cap]
  Box* kids = nullptr;    // [2 cap]
  Box* result = nullptr;  // [cap]
  int* counts = nullptr;  // [2]
  double* eff = nullptr;  // the efficiency threshold of the current call
  uint8_t* mask = nullptr;
  int* pc = nullptr;      // column prefix sums [(nty + 1) ntx]
  int* pr = nullptr;      // row prefix sums [nty (ntx + 1)]
  void release() {
    void* b[] = {level[0], level[1], acc, kids, result, counts, eff, mask, pc, pr};
    for (void* p : b)
      if (p) kss_rt::dev_free(p);
    *this = Workspace{};
  }
};

cudaError_t ws_alloc(Workspace& ws, int ntx, int nty) {
  const int ntiles = ntx * nty;
  ws.cap = ntiles + 1;
  const size_t bb = sizeof(Box) * size_t(ws.cap);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.level[0], 2 * bb);
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.level[1], 2 * bb);
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.acc, bb);
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.kids, 2 * bb);
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.result, bb);
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.counts, 2 * sizeof(int));
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.eff, sizeof(double));
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.mask, size_t(ntiles));
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.pc, sizeof(int) * size_t(nty + 1) * ntx);
  if (e == cudaSuccess) e = kss_rt::dev_malloc(&ws.pr, sizeof(int) * size_t(nty) * (ntx + 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws.release();
  }
  return e;
}

// Workspace of one tile grid, kept by a lattice between calls: the device arrays, a
// stream to record on, and the recorded chunk of kChunk clustering levels.
struct RegridWS {
  Workspace ws;
  int ntx = 0, nty = 0, ctas = 0;
  size_t smem = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t chunk = nullptr;
  void destroy() {
    if (chunk) cudaGraphExecDestroy(chunk);
    if (cap) cudaStreamDestroy(cap);
    ws.release();
    chunk = nullptr;
    cap = nullptr;
    ntx = nty = 0;
  }
};

constexpr int kChunk = 8;  // clustering levels between host checks of the level size

cudaError_t ws_setup(RegridWS& R, int ntx, int nty) {
  if (R.ntx == ntx && R.nty == nty && R.chunk) return cudaSuccess;
  R.destroy();
  cudaError_t e = ws_alloc(R.ws, ntx, nty);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 1;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  R.ctas = std::max(1, std::min(ntx * nty, 2 * nsm));
  R.smem = sizeof(int) * size_t(ntx + nty);
  if (R.smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(cluster_level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(R.smem))) != cudaSuccess)
    return e;
  if ((e = cudaStreamCreateWithFlags(&R.cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  // one chunk: kChunk levels; the level lists alternate, so a chunk ends where it began
  if ((e = cudaStreamBeginCapture(R.cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
  int cur = 0;
  for (int k = 0; k < kChunk; ++k) {
    cluster_level_kernel<<<R.ctas, 256, R.smem, R.cap>>>(R.ws.pc, R.ws.pr, ntx, R.ws.level[cur],
                                                         R.ws.counts + 1, R.ws.eff, R.ws.acc,
                                                         R.ws.kids);
    compact_kernel<<<1, 1024, 0, R.cap>>>(R.ws.acc, R.ws.kids, R.ws.result, R.ws.cap,
                                          R.ws.level[cur ^ 1], R.ws.counts);
    cur ^= 1;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t le = cudaGetLastError();
  e = cudaStreamEndCapture(R.cap, &graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return le != cudaSuccess ? le : e;
  }
  e = cudaGraphInstantiate(&R.chunk, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  R.ntx = ntx;
  R.nty = nty;
  return cudaSuccess;
}

// The whole regrid on device flags; outputs to host or device pointers.
int regrid_run(RegridWS& R, const uint8_t* d_flags, long long pitch, int nx, int ny, int tile,
               int buffer, double efficiency, uint8_t* tile_mask, kss_box* boxes,
               int32_t max_boxes, int32_t* nboxes, int on_device, cudaStream_t s,
               std::string* msg) {
  const int ntx = (nx + tile - 1) / tile, nty = (ny + tile - 1) / tile;
  if (ntx > kMaxSide || nty > kMaxSide) return KSS_ERR_UNSUPPORTED;
  const int ntiles = ntx * nty;
  auto fail_cuda = [&](cudaError_t e) {
    if (msg) *msg = std::string("regrid: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return KSS_ERR_CUDA;
  };
  cudaError_t e = ws_setup(R, ntx, nty);
  if (e != cudaSuccess) {
    R.destroy();
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return KSS_ERR_OOM;
    }
    return fail_cuda(e);
  }
  Workspace& ws = R.ws;
  tile_mask_kernel<<<(ntiles + 255) / 256, 256, 0, s>>>(d_flags, pitch, nx, ny, tile, buffer,
                                                         ntx, nty, ws.mask);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e);
  mask_prefix_kernel<<<(ntx + nty + 255) / 256, 256, 0, s>>>(ws.mask, ntx, nty, ws.pc, ws.pr);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e);
  // first level: the whole tile grid; results so far 0; this call's efficiency (pageable
  // sources: each copy completes before the call returns)
  const Box whole{0, 0, ntx, nty};
  const int init[2] = {0, 1};
  if ((e = cudaMemcpyAsync(ws.level[0], &whole, sizeof(Box), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ws.counts, init, sizeof(init), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ws.eff, &efficiency, sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail_cuda(e);
  int count[2] = {0, 1};
  // every level splits some box, and a box splits at most w + h - 2 times on any path
  for (int level = 0; count[1] > 0 && level <= ntx + nty + 2; level += kChunk) {
    if ((e = cudaGraphLaunch(R.chunk, s)) != cudaSuccess) return fail_cuda(e);
    if ((e = cudaMemcpyAsync(count, ws.counts, sizeof(count), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return fail_cuda(e);
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const int total = count[0];
  const int ncopy = std::min(total, max_boxes);
  static_assert(sizeof(Box) == sizeof(kss_box), "box layout");
  if (boxes && ncopy > 0 &&
      (e = cudaMemcpyAsync(boxes, ws.result, sizeof(Box) * size_t(ncopy), kind, s)) != cudaSuccess)
    return fail_cuda(e);
  if (tile_mask && (e = cudaMemcpyAsync(tile_mask, ws.mask, size_t(ntiles), kind, s)) != cudaSuccess)
    return fail_cuda(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e);
  *nboxes = total;
  return KSS_OK;
}

bool valid_args(int tile, int buffer, double efficiency, int32_t max_boxes, int32_t* nboxes) {
  return (tile == 8 || tile == 16 || tile == 32 || tile == 64) && buffer >= 0 &&
         buffer <= 1024 && efficiency >= 0.0 && efficiency <= 1.0 && max_boxes >= 0 && nboxes;
}

}  // namespace

namespace kss_rt {
void regrid_release(kss_lattice* L) {
  if (!L || !L->regrid) return;
  RegridWS* R = static_cast<RegridWS*>(L->regrid);
  R->destroy();
  delete R;
  L->regrid = nullptr;
}
}  // namespace kss_rt

extern "C" {

int kss_regrid(kss_lattice* L, int32_t buffer, double efficiency, uint8_t* tile_mask,
               kss_box* boxes, int32_t max_boxes, int32_t* nboxes, int on_device) {
  const kss_rt::NvtxRange nvtx_range("kss_regrid");
  int rc = enter(L);
  if (rc) return rc;
  if (!valid_args(L->cfg.tile, buffer, efficiency, max_boxes, nboxes))
    return fail(L, KSS_ERR_ARG, "invalid regrid argument");
  DeviceGuard g(L->device);
  // the flags of the current step (evaluated if this step had no outputs)
  if ((rc = kss_read_flags(L, nullptr, nullptr, nullptr, 1)) < 0) return rc;
  if (!L->regrid) {
    L->regrid = new (std::nothrow) RegridWS();
    if (!L->regrid) return fail(L, KSS_ERR_OOM, "regrid workspace");
  }
  rc = regrid_run(*static_cast<RegridWS*>(L->regrid), L->flags, L->pitch, L->cfg.nx, L->cfg.ny,
                  L->cfg.tile, buffer, efficiency, tile_mask, boxes, max_boxes, nboxes, on_device,
                  L->stream, &L->msg);
  if (rc == KSS_ERR_CUDA) L->err = rc;  // sticky
  return rc;
}

int kss_regrid_flags(const uint8_t* flags, int32_t nx, int32_t ny, int32_t tile, int32_t buffer,
                     double efficiency, uint8_t* tile_mask, kss_box* boxes, int32_t max_boxes,
                     int32_t* nboxes, int on_device, void* stream) {
  if (!flags || nx < 1 || ny < 1 || (long long)nx * ny > 0x7fffffffLL) return KSS_ERR_ARG;
  if (!valid_args(tile, buffer, efficiency, max_boxes, nboxes)) return KSS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint8_t* d = flags;
  uint8_t* staged = nullptr;
  const size_t bytes = size_t(nx) * ny;
  if (!on_device) {
    if (kss_rt::dev_malloc(&staged, bytes) != cudaSuccess) {
      cudaGetLastError();
      return KSS_ERR_OOM;
    }
    if (cudaMemcpyAsync(staged, flags, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      kss_rt::dev_free(staged);
      return KSS_ERR_CUDA;
    }
    d = staged;
  }
  RegridWS R;
  const int rc = regrid_run(R, d, nx, nx, ny, tile, buffer, efficiency, tile_mask, boxes, max_boxes,
                            nboxes, on_device, s, nullptr);
  cudaStreamSynchronize(s);
  R.destroy();
  if (staged) kss_rt::dev_free(staged);
  return rc;
}

}  // extern "C"
