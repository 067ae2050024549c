// step_tma.cuh -- the fused step with TMA (cp.async.bulk) staging of the source rows.
//
// The register-pipelined kernel (step_kernel) keeps every load in flight in
// registers, which caps the number of resident warps and with it the bytes in
// flight per SM.  Here the loads are bulk copies into shared memory that complete
// on an mbarrier, so no register is held by a load in flight:
//
//   * Persistent grid: one CTA per SM, two independent groups of 8 warps.  A group
//     owns a contiguous run of rows of one strip of 8*32*V columns (4 KiB per
//     population row); the groups on a strip split its rows evenly.
//   * Per group, a ring of 3 stages.  A stage is one output row: for each population
//     q, the segment [x0 - 16 B, x0 + 4 KiB + 16 B) of source row j - cy_q (the strip's
//     cells plus the x-halos on both sides), one 4128-byte bulk copy (large copies:
//     the copy engine's per-request cost, not the bytes, limits small ones).  Two rows
//     are in flight while the group works on a third.
//   * Lanes read their 16-byte vector and the two halo elements straight from the
//     stage (no shuffles).  A named barrier over the group (with an AND vote of the
//     wait results) marks the stage as read, and the group's leader thread requests
//     the row three ahead into it.  The periodic seams and a ragged row end take one
//     scalar global load, as in step_kernel.
//   * Tag counts per tile are accumulated over the rows of a tile band and added to
//     the (zeroed) tile counters with one atomic per tile per band; sums and counts
//     are reduced per warp, per CTA and by the last CTA, in a fixed order.
//   * Every mbarrier wait is bounded by a clock budget (about one second).  If a wait
//     runs out anywhere in a group, the whole group stops, the error word is set, the
//     leader waits (bounded again) for the group's copies still in flight, and the
//     host reports KSS_ERR_TIMEOUT.
#pragma once

#include "step_kernel.cuh"

namespace kss {

constexpr int kTmaWarps = 16;
constexpr int kTmaThreads = 32 * kTmaWarps;
constexpr int kTmaGroups = 2;                          // independent row pipelines per CTA
constexpr int kGroupWarps = kTmaWarps / kTmaGroups;    // warps sharing one row
constexpr int kGroupThreads = 32 * kGroupWarps;
constexpr int kTmaStages = 3;                          // ring depth per group
constexpr int kSegBytes = kGroupWarps * 512 + 32;      // largest row segment: 4 KiB + 16 B halos
constexpr int kStageBytes = 9 * kSegBytes;
constexpr int kBarrierBytes = 128;
constexpr size_t kTmaSmemBytes =
    kBarrierBytes + size_t(kTmaGroups) * kTmaStages * kStageBytes;  // 223,040 B
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
static_assert(kTmaGroups * kTmaStages * 8 <= kBarrierBytes, "barrier area too small");

// Rows of strip s are split into `chunks` contiguous runs; task = chunk * strips + s.
// A strip is kGroupWarps * 32 * V columns.
struct TmaPlan {
  int strips;
  int chunks;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Named barrier over the kGroupThreads threads of group `id` (ids 1..kTmaGroups; 0 is
// __syncthreads) that also returns whether `pred` held in every one of them.
__device__ __forceinline__ bool group_barrier_and(int id, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"(uint32_t(pred)), "r"(id), "r"(kGroupThreads)
      : "memory");
  return out != 0;
}

// Wait for phase `parity` of `bar` to complete, for at most `deadline` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long deadline = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > deadline) return false;
  }
  return true;
}

// One arrival on `bar` (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <class T, int MODE>
__global__ void __launch_bounds__(kTmaThreads, 1)
step_tma_kernel(const StepParams<T> p, const TmaPlan plan) {
  constexpr int V = Vec<T>::N;
  constexpr int H = 16 / int(sizeof(T));  // halo elements on each side of a segment
  constexpr int W = kGroupWarps * 32 * V;  // columns of a strip
  constexpr int SEG = W + 2 * H;  // segment elements (stage slots are kSegBytes apart)
  constexpr int SEGS = kSegBytes / int(sizeof(T));  // slot stride in elements
  constexpr bool OUT = MODE != MODE_PLAIN;
  constexpr int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  static_assert(SEG <= SEGS, "segment layout");
  using VT = typename Vec<T>::type;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ Red<T> s_sum[kTmaWarps][3];
  __shared__ uint32_t s_cnt[kTmaWarps][3];
  __shared__ int s_last;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp / kGroupWarps, lw = warp % kGroupWarps;
  const bool leader = (threadIdx.x % kGroupThreads) == 0;  // issues the group's copies
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + grp * kTmaStages;
  T* stages = reinterpret_cast<T*>(smem + kBarrierBytes) + size_t(grp) * kTmaStages * 9 * SEGS;

  if (leader) {
#pragma unroll
    for (int st = 0; st < kTmaStages; ++st) mbar_init(bars + st, 1);
    fence_mbarrier_init();
  }
  __syncthreads();

  Acc<T> a_rho, a_jx, a_jy;
  uint32_t n_ref = 0, n_sw = 0, n_np = 0;
  bool ok = true;
  uint32_t consumed = 0, issued = 0;  // rows of this group read / requested so far
  const int ngroups = gridDim.x * kTmaGroups;
  const int tasks = plan.strips * plan.chunks;

  for (int task = blockIdx.x * kTmaGroups + grp; task < tasks && ok; task += ngroups) {
    const int s = task % plan.strips, c = task / plan.strips;
    const int r0 = int((long long)c * p.ny / plan.chunks);
    const int r1 = int((long long)(c + 1) * p.ny / plan.chunks);
    const int x0 = s * W;
    const int L = max(x0 - H, 0), R = min(x0 + W + H, p.pitch);
    const uint32_t bytes = uint32_t(R - L) * uint32_t(sizeof(T));
    const int soff = L - (x0 - H);

    // leader: request row `row` into stage (n % stages)
    auto request = [&](int row, uint32_t n) {
      const int st = int(n % kTmaStages);
      T* dst = stages + st * 9 * SEGS + soff;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bars + st, 9 * bytes);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        int sr = row - CY[q];
        sr = sr < 0 ? sr + p.ny : (sr >= p.ny ? sr - p.ny : sr);
        bulk_copy_g2s(dst + q * SEGS, p.src + q * p.plane + (long long)sr * p.pitch + L, bytes,
                      bars + st);
      }
    };
    if (leader) {
#pragma unroll
      for (int d = 0; d < kTmaStages; ++d)
        if (r0 + d < r1) request(r0 + d, issued + d);
    }
    issued += uint32_t(min(kTmaStages, r1 - r0));

    const int col = V * (32 * lw + lane);  // this lane's first cell, relative to x0
    const int i0 = x0 + col;
    const bool cv = i0 < p.nx;
    const bool tail = i0 + V >= p.nx;
    int tr = 0, ts = 0, td = 0;  // this lane's tags (and deferred cells) in the tile band
    for (int r = r0; r < r1; ++r) {
      const int st = int(consumed % kTmaStages);
      const bool got = mbar_wait_bounded(bars + st, (consumed / kTmaStages) & 1u);
      T ft[9][V];
      if (got) {
        const T* sg = stages + st * 9 * SEGS + H + col;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const VT a = *reinterpret_cast<const VT*>(sg + q * SEGS);
          T v[V];
          if constexpr (V == 4) {
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
          } else {
            v[0] = a.x; v[1] = a.y;
          }
          if (CX[q] == 0) {
#pragma unroll
            for (int k = 0; k < V; ++k) ft[q][k] = v[k];
          } else {
            int sr = r - CY[q];
            sr = sr < 0 ? sr + p.ny : (sr >= p.ny ? sr - p.ny : sr);
            const T* grow = p.src + q * p.plane + (long long)sr * p.pitch;
            if (CX[q] == 1) {  // source column i - 1
              T left = sg[q * SEGS - 1];
              if (i0 == 0) left = __ldg(grow + (p.nx - 1));
              ft[q][0] = left;
#pragma unroll
              for (int k = 1; k < V; ++k) ft[q][k] = v[k - 1];
            } else {  // source column i + 1
              T right = sg[q * SEGS + V];
              if (cv && tail) right = __ldg(grow);
#pragma unroll
              for (int k = 0; k < V - 1; ++k) ft[q][k] = v[k + 1];
              ft[q][V - 1] = right;
              if (tail) {
#pragma unroll
                for (int k = 0; k < V - 1; ++k)
                  if (i0 + k == p.nx - 1) ft[q][k] = right;
              }
            }
          }
        }
      }
      // every thread of the group has read the stage (or the wait ran out somewhere)
      if (!group_barrier_and(1 + grp, got)) {
        ok = false;
        break;
      }
      ++consumed;
      if (r + kTmaStages < r1) {
        if (leader) request(r + kTmaStages, issued);
        ++issued;
      }

      const uint32_t fbits = fused_row<T, MODE, true, true>(p, ft, i0, r, cv, a_rho, a_jx, a_jy);
      if (OUT) {
        n_ref += __popc(fbits & 0x01010101u);
        n_sw += __popc(fbits & 0x02020202u);
        n_np += __popc(fbits & 0x80808080u);
        tr += __popc(fbits & 0x01010101u);
        ts += __popc(fbits & 0x02020202u);
        td += __popc(fbits & 0x40404040u);
        if (MODE == MODE_STD)
          append_deferred<V>(fbits, i0, r, p.nx, p.defer_count, p.defer_list, p.defer_cap);
        if ((r + 1) % p.tile == 0 || r + 1 == r1) {
          // end of a tile band (or of this run of rows): add the band's counts
          const int lpt = p.tile / V;
          for (int o = lpt >> 1; o > 0; o >>= 1) {
            tr += __shfl_xor_sync(kFull, tr, o);
            ts += __shfl_xor_sync(kFull, ts, o);
            td += __shfl_xor_sync(kFull, td, o);
          }
          const int tx = i0 / p.tile;
          if ((lane & (lpt - 1)) == 0 && tx < p.ntx) {
            const long long t = (long long)(r / p.tile) * p.ntx + tx;
            if (tr) atomicAdd(p.tiles + t, tr);
            if (ts) atomicAdd(p.tiles + (long long)p.ntx * p.nty + t, ts);
            if (td) atomicAdd(p.tiles_def + t, td);
          }
          tr = ts = td = 0;
        }
      }
    }
  }
  if (!ok) {
    // a wait ran out: record it, then let the group's copies still in flight land
    // before the CTA can exit (bounded as well)
    if (leader) {
      atomicOr(p.err, 1u);
      for (uint32_t n = consumed; n < issued; ++n)
        mbar_wait_bounded(bars + (n % kTmaStages), (n / kTmaStages) & 1u);
    }
  }
  __syncthreads();

  if (!OUT) return;

  // ---- per-CTA reduction (fixed order), then the last CTA adds the CTA partials ----
  a_rho.warp_reduce();
  a_jx.warp_reduce();
  a_jy.warp_reduce();
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n_ref += __shfl_xor_sync(kFull, n_ref, off);
    n_sw += __shfl_xor_sync(kFull, n_sw, off);
    n_np += __shfl_xor_sync(kFull, n_np, off);
  }
  if (lane == 0) {
    s_sum[warp][0] = Red<T>::of(a_rho);
    s_sum[warp][1] = Red<T>::of(a_jx);
    s_sum[warp][2] = Red<T>::of(a_jy);
    s_cnt[warp][0] = n_ref;
    s_cnt[warp][1] = n_sw;
    s_cnt[warp][2] = n_np;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Red<T> t0, t1, t2;
    uint32_t c0 = 0, c1 = 0, c2 = 0;
    for (int w = 0; w < kTmaWarps; ++w) {
      t0.add(s_sum[w][0]);
      t1.add(s_sum[w][1]);
      t2.add(s_sum[w][2]);
      c0 += s_cnt[w][0];
      c1 += s_cnt[w][1];
      c2 += s_cnt[w][2];
    }
    const int b = blockIdx.x;
    t0.store(p.part_sum + 3 * b + 0);
    t1.store(p.part_sum + 3 * b + 1);
    t2.store(p.part_sum + 3 * b + 2);
    p.part_cnt[4 * b + 0] = c0;
    p.part_cnt[4 * b + 1] = c1;
    p.part_cnt[4 * b + 2] = c2;
    __threadfence();
    s_last = atomicAdd(p.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  finalize_partials<T, kTmaThreads>(p, gridDim.x);
}

}  // namespace kss
