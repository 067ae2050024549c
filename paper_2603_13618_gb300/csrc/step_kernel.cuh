// step_kernel.cuh -- the fused D2Q9 pull-stream + BGK collide + sensor + tagging
// kernel, and the small per-cell helper kernels (equilibrium initialisation,
// moments, layout conversion).
//
// Data layout in HBM (per lattice, storage type T = float or double):
//   populations   9 planes f[q][j][i], row pitch P (elements, a multiple of 128 bytes),
//                 plane stride P*ny; two buffers (A/B) swapped every step
//   sensor fields one plane of T per recorded sensor, same pitch
//   flags         uint8 [ny][P]
//   tile counts   int32 [2][nty][ntx]   (refine, switch)
//   scratch       per-block partial sums (3 doubles) and counts (4 uint32), a
//                 block-completion counter, and the final sums/counts
//
// Work decomposition: a CTA of 8 warps owns a 32*V-column x (bands * tile)-row block
// of the lattice (V = 16 bytes / sizeof(T) cells per thread, one 16-byte vector per
// population per row; about 32 rows).  Warp w handles rows w, w+8, ... of the block;
// lane L the V cells starting at column (32*bx + L)*V.  Because CTA blocks consist
// of whole tagging tiles, every tile count is formed inside one CTA (in shared
// memory, per band) and written once.
//
// Pull streaming: f~_q(i, j) = f_q(i - cx_q, j - cy_q).  Populations with cx_q = 0
// are single aligned vector loads of row j - cy_q.  For cx_q = +1 (source i - 1) a
// thread loads its own aligned vector and takes the element left of it from lane
// L-1's vector by a warp shuffle; lane 0 loads that one element itself.  cx_q = -1
// is the mirror image with lane 31.  The periodic wrap in x (cells 0 and nx-1) and
// a row end inside a vector (nx not a multiple of V) are fixed up by one scalar
// load.  The periodic wrap in y selects rows j-1 and j+1 modulo ny.
//
// Reductions are deterministic: per-thread and per-warp in a fixed order
// (double-float for FP32 storage), per block in a fixed order, and the last block
// to finish (ticket from an atomic counter, no waiting) adds the per-block partials
// in block order.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "d2q9.cuh"
#include "f32x2.cuh"

namespace kss {

// Minimum resident CTAs per SM requested from the register allocator (build-time tuning
// knobs, -DKSS_..._MIN_BLOCKS=n):
//   KSS_F32_MIN_BLOCKS   FP32 plain and {Kn, KL, neq} steps (one-step, multi-step and
//                        batched kernels): two 256-thread CTAs at up to 128 registers.  With
//                        the paired row and warp-uniform row arithmetic, 4096^2 multi-step
//                        launches take 0.2029 ms per step against 0.2241 ms at three CTAs
//                        (80 registers, spilling), one-step launches 0.838 against 0.725 of
//                        the measured bandwidth.
//   KSS_STEP_MIN_BLOCKS  FP64 and FP16-deviation plain steps, FP64 {Kn, KL, neq} steps: three
//                        CTAs (80 registers).
//   KSS_F16_MIN_BLOCKS   FP16-deviation {Kn, KL, neq} steps: three (0.659 ms per 8192^2 step
//                        against 0.706 ms at two: its 8-byte rows need more warps in flight).
//   KSS_FULL_MIN_BLOCKS  the all-sensor steps (much more per-cell state): two CTAs (at most
//                        128 registers) against one (158 registers).
#ifndef KSS_F32_MIN_BLOCKS
#define KSS_F32_MIN_BLOCKS 2
#endif
#ifndef KSS_STEP_MIN_BLOCKS
#define KSS_STEP_MIN_BLOCKS 3
#endif
#ifndef KSS_FULL_MIN_BLOCKS
#define KSS_FULL_MIN_BLOCKS 2
#endif
#ifndef KSS_F16_MIN_BLOCKS
#define KSS_F16_MIN_BLOCKS KSS_STEP_MIN_BLOCKS
#endif
//   KSS_H8_MIN_BLOCKS    the FP16 {Kn, KL, neq} step with eight cells per lane
//   KSS_H8_WARPS         warps per CTA of that step (8; 4 takes five CTAs per SM at 96
//                        registers, where the row spills: 0.672 vs 0.591 ms per 8192^2 step)
#ifndef KSS_H8_WARPS
#define KSS_H8_WARPS 8
#endif
#ifndef KSS_H8_MIN_BLOCKS
#define KSS_H8_MIN_BLOCKS (KSS_H8_WARPS == 4 ? 5 : 2)
#endif

// The knob of a step kernel with storage S and sensor set MODE.
template <class S, int MODE>
__host__ __device__ constexpr int step_min_blocks() {
  return MODE == MODE_FULL ? KSS_FULL_MIN_BLOCKS
         : std::is_same<S, float>::value ? KSS_F32_MIN_BLOCKS
         : (std::is_same<S, __half>::value && MODE == MODE_STD) ? KSS_F16_MIN_BLOCKS
                                                                : KSS_STEP_MIN_BLOCKS;
}

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kMaxBands = 8;  // tile bands per CTA of step_kernel (rows = bands * tile)
// Deferred cells a warp of step_kernel can hold: all of its cells (at most 64 rows per CTA
// / 8 warps, 32 * V <= 128 columns, or 256 with eight cells per lane), as CTA-local
// offsets.
constexpr int kWarpDefer = 8 * 128;
constexpr int kWarpDefer8 = 8 * 256;

// Tile bands per CTA: about KSS_STEP_ROWS rows per CTA (32: 4 per warp) amortise the
// CTA's epilogue; taller CTAs would leave a longer tail of partly filled waves.
#ifndef KSS_STEP_ROWS
#define KSS_STEP_ROWS 32
#endif
__host__ __device__ constexpr int step_bands(int tile) {
  return tile >= KSS_STEP_ROWS ? 1 : KSS_STEP_ROWS / tile;
}
constexpr unsigned kFull = 0xffffffffu;
// Flag bit of a cell whose {Kn, KL, neq} the fused pass could not prove exact; set only
// between the fused pass and fixup_kernel, which replaces the byte.
constexpr uint32_t kFlagDeferred = 0x40u;

// Debug builds (-DKSS_DEBUG_BOUNDS=1): a CTA block checks its coordinates and rows
// against the lattice before it touches memory, and every deferred-cell slot and tile
// index against its shared array.  A failed check sets bit 2 of the lattice's error word
// and the access is skipped; the next synchronising call returns KSS_ERR_BOUNDS.  Release
// builds compile the checks away.
#ifndef KSS_DEBUG_BOUNDS
#define KSS_DEBUG_BOUNDS 0
#endif
constexpr uint32_t kErrBounds = 4u;
__device__ __forceinline__ bool bounds_ok(bool ok, uint32_t* err) {
  if (!KSS_DEBUG_BOUNDS || ok) return true;
  if (err) atomicOr(err, kErrBounds);
  return false;
}

// Cells per thread and the vector type of one population's load/store.  FP32 takes
// 4 cells (16-byte vectors) by default; -DKSS_F32_VEC=2 selects 8-byte vectors (half the
// per-thread state, more resident warps).
#ifndef KSS_F32_VEC
#define KSS_F32_VEC 4
#endif
template <class T> struct Vec;
template <> struct Vec<float> {
  static constexpr int N = KSS_F32_VEC;
  using type = typename std::conditional<KSS_F32_VEC == 4, float4, float2>::type;
};
template <> struct Vec<double> {
  static constexpr int N = 2;
  using type = double2;
};

// Vector type of V elements of T (one 8- or 16-byte load or store).
template <class T, int V> struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<double, 2> { using type = double2; };

template <class VT, class T, int N>
__device__ __forceinline__ VT make_vec(const T (&v)[N]) {
  if constexpr (N == 4) {
    return VT{v[0], v[1], v[2], v[3]};
  } else {
    return VT{v[0], v[1]};
  }
}

// ---------------------------------------------------------------- storage ----
// Population storage S and the arithmetic type T = arith_t<S> of the step:
//   float, double  the populations themselves (T = S);
//   __half         FP16 deviations from the rest equilibrium of a reference density
//                  rho0, h_q = RN_fp16((f_q - b_q) s_q) with b_q = RN_fp32(w_q rho0) and
//                  s_q = 2^(k_q + K) (k_q = 1, 3, 5 for w_q = 4/9, 1/9, 1/36: s_q w_q =
//                  (8/9) 2^K for every q), decoded as f_q = RN_fp32(b_q + h_q / s_q) and
//                  collided in FP32 (T = float).  (s_q = 1 is the literal unscaled form.)
template <class S> struct Store;
template <> struct Store<float> {
  using T = float;
  struct Codec {};
};
template <> struct Store<double> {
  using T = double;
  struct Codec {};
};
template <> struct Store<__half> {
  using T = float;
  struct Codec {
    float base[9];   // b_q
    float scale[9];  // s_q
    float inv[9];    // 1 / s_q (exact: a power of two)
  };
};
template <class S>
using arith_t = typename Store<S>::T;
template <class S>
using codec_t = typename Store<S>::Codec;
template <> struct Vec<__half> {
  static constexpr int N = KSS_F32_VEC;  // as FP32: the same cells per thread
};
template <> struct VecT<__half, 4> { using type = uint2; };
template <> struct VecT<__half, 2> { using type = unsigned int; };

template <class S>
__device__ __forceinline__ arith_t<S> decode(S v, int q, const codec_t<S>& c) {
  if constexpr (std::is_same<S, __half>::value) {
    return fmaf(__half2float(v), c.inv[q], c.base[q]);
  } else {
    return v;
  }
}

template <class S>
__device__ __forceinline__ S encode(arith_t<S> f, int q, const codec_t<S>& c) {
  if constexpr (std::is_same<S, __half>::value) {
    return __float2half_rn((f - c.base[q]) * c.scale[q]);
  } else {
    return f;
  }
}

template <class S>
struct StepParams {
  using T = arith_t<S>;
  const S* src;          // population buffer read this step
  S* dst;                // population buffer written this step (STORE)
  T* rec;                // recorded sensor planes (arithmetic type)
  uint8_t* flags;        // [ny][pitch]
  int32_t* tiles;        // [2][nty][ntx] refine, switch tags per tile
  int32_t* tiles_def;    // [nty][ntx] cells deferred to fixup_kernel per tile
  uint32_t* defer_list;  // indices j * nx + i of deferred cells (capacity defer_cap)
  uint32_t* defer_count; // entries requested (> defer_cap: overflow, fixup scans instead)
  uint32_t* defer_ticket;  // CTA completion counter of fixup_kernel, 0 between launches
  uint32_t defer_cap;
  double* part_sum;      // [nblocks][3]
  uint32_t* part_cnt;    // [nblocks][4]
  uint32_t* done;        // block-completion counter, 0 between launches
  double* stat_sums;     // [3]
  unsigned long long* stat_counts;  // [3]
  uint32_t* err;         // error word: bit 0 = a bounded device wait ran out
  long long plane;       // elements per population plane
  int pitch, nx, ny, tile, ntx, nty;
  T omega, tau;          // 1/tau and tau
  T thr_r, thr_s;        // largest T values <= the thresholds: eps > thr exactly
  int refine_s, switch_s, switch_on;
  int bands;             // tile bands per CTA of step_kernel (CTA height = bands * tile)
  int grid_x, nblocks;   // step grid of the lattice: CTAs per block row, CTAs in all
                         // (read by the batched step only; step_kernel uses its grid)
  int mode;              // the lattice's sensor set on output steps (batched step only)
  T zero;                // 0, read at run time (see product2): every builder value-initialises
  int slab;              // 0: periodic in y; 1: a y-slab of a decomposed lattice, whose rows
                         // -1 and ny are halo rows held next to its own (kss_slab_create)
  int rec_slot[S_COUNT];  // plane index of each recorded sensor, -1 if not recorded
  codec_t<S> codec;      // FP16 deviation codec (empty for float / double storage)
  uint8_t* region;       // two-relaxation region [ny][pitch], a byte per cell (AAR steps):
                         // read before the collision, rewritten with the switch flags
                         // (0 / 1) on output steps
  Trt<T> trt;            // two-relaxation coefficients, and the model of eps_qe
};

// Offsets (elements) of rows j - 1 and j + 1 from row j: periodic in y, or, in a slab
// (p.slab), the halo rows -1 and ny that sit next to the slab's own rows.
template <class S>
__device__ __forceinline__ void row_neighbours(const StepParams<S>& p, int j, long long& up,
                                               long long& dn) {
  const bool lo = (j == 0) & (p.slab == 0), hi = (j + 1 == p.ny) & (p.slab == 0);
  up = (long long)((lo ? p.ny : j) - 1 - j) * p.pitch;
  dn = (long long)((hi ? 0 : j + 1) - j) * p.pitch;
}

// ---------------------------------------------------------------- loads ----
// Population loads: through the read-only data path (CG = false; the source buffer is
// not written during the launch), or as ordinary cached loads (CG = true: the multi-step
// kernel, whose source buffers other CTAs write during the launch; its loads follow an
// acquire of the writers' release, which the read-only path would not honour).
template <bool CG, class VT>
__device__ __forceinline__ VT ld_pop(const VT* p) {
  if constexpr (CG) {
    return __ldca(p);
  } else {
    return __ldg(p);
  }
}

// V cells per thread (default: the fused step's Vec<T>::N).
template <class T, int V = Vec<T>::N, bool CG = false>
__device__ __forceinline__ void vload(const T* p, bool ok, T (&v)[V]) {
  using VT = typename VecT<T, V>::type;
  if (ok) {
    const VT a = ld_pop<CG>(reinterpret_cast<const VT*>(p));
    if constexpr (V == 4) {
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
      v[0] = a.x; v[1] = a.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = T(0);
  }
}

// Pull streaming along x.  Loads and assembly are split so that a row's nine
// vector loads and its six halo loads are all in flight before the first shuffle
// waits on any of them.
//
// Halo element of a cx = +1 population (source column i - 1): lane 0 of each warp
// needs the element left of its vector (column nx-1 at the periodic seam).
template <class T, bool CG = false>
__device__ __forceinline__ T load_left_halo(const T* row, int i0, int nx, int lane, bool cv) {
  return (lane == 0 && cv) ? ld_pop<CG>(row + (i0 == 0 ? nx - 1 : i0 - 1)) : T(0);
}

// Halo element of a cx = -1 population (source column i + 1): lane 31, and any lane
// whose vector reaches the row end (then the element is column 0, periodic seam).
template <class T, int V = Vec<T>::N, bool CG = false>
__device__ __forceinline__ T load_right_halo(const T* row, int i0, int nx, int lane, bool cv) {
  const bool tail = i0 + V >= nx;
  return (cv && (lane == 31 || tail)) ? ld_pop<CG>(row + (tail ? 0 : i0 + V)) : T(0);
}

// Cells i0..i0+V-1 pulled from column i - 1: the left neighbour's last element by
// shuffle, lane 0 from its halo load.
template <class T, int V = Vec<T>::N>
__device__ __forceinline__ void assemble_from_left(T (&v)[V], T halo, int lane) {
  const T left = __shfl_up_sync(kFull, v[V - 1], 1);
#pragma unroll
  for (int k = V - 1; k > 0; --k) v[k] = v[k - 1];
  v[0] = lane == 0 ? halo : left;
}

// Cells i0..i0+V-1 pulled from column i + 1; cell nx-1 takes column 0 wherever it
// sits in the vector.
template <class T, int V = Vec<T>::N>
__device__ __forceinline__ void assemble_from_right(T (&v)[V], T halo, int i0, int nx,
                                                    int lane) {
  const T right = __shfl_down_sync(kFull, v[0], 1);
  const bool tail = i0 + V >= nx;
#pragma unroll
  for (int k = 0; k < V - 1; ++k) v[k] = v[k + 1];
  v[V - 1] = (lane == 31 || tail) ? halo : right;
  if (tail) {
#pragma unroll
    for (int k = 0; k < V - 1; ++k)
      if (i0 + k == nx - 1) v[k] = halo;
  }
}

// ---------------------------------------------------------------- row prefetch ----
// The multi-step kernels with FP32 storage (single lattices with BGK or two-relaxation,
// and batches) stage each warp's next row in shared memory with asynchronous copies
// (cp.async), issued before the current row's arithmetic, so that a row's loads are in
// flight while the previous row is computed; the register file holds no second row.  A
// warp's slots are written only by its own lanes' copies and read back by the same
// lanes, so the copies need no CTA barrier, only the wait for their own group and a warp
// barrier that orders the reads of a row before the copies of the next one.  Measured at
// 4096^2: BGK 0.2202 vs 0.2284 ms per step (three CTAs per SM); two-relaxation 0.2207 vs
// 0.2561 ms with two CTAs per SM at up to 128 registers (at three CTAs and 80 registers
// it spills, and the slots leave too little L1 for the spills: 0.2932 ms); the 64-lattice
// batch 0.2015 vs 0.2194 ms, also at two CTAs per SM (at three it was slower, 0.2302 ms).
// Build knob: -DKSS_MULTI_PREFETCH=0 loads every row directly.
#ifndef KSS_MULTI_PREFETCH
#define KSS_MULTI_PREFETCH 1
#endif

struct PfWarp {
  float4 pop[9][32];  // the nine population vectors of each lane
  float hr[3][32];    // right halo of q = 3, 6, 7 (lane 31 and the row's tail lanes)
  float hl[4];        // left halo of q = 1, 5, 8 (lane 0)
  uint32_t rg[32];    // region bytes of each lane's cells (two-relaxation steps)
};
constexpr int kPfBytes = kWarps * int(sizeof(PfWarp));
static_assert(sizeof(PfWarp) % 16 == 0, "16-byte aligned warp slots");

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// The same slots for FP16 deviation codes (see pf_issue_half): nine 8-byte vectors per lane
// and the 4-byte words that hold the halo codes.
struct PfWarpH {
  uint2 pop[9][32];     // the nine code vectors of each lane
  uint32_t hr[3][32];   // words holding the right halo of q = 3, 6, 7 (lane 31, tail lanes)
  uint32_t hl[4];       // words holding the left halo of q = 1, 5, 8 (lane 0)
};
constexpr int kPfBytesH = kWarps * int(sizeof(PfWarpH));
static_assert(sizeof(PfWarpH) % 16 == 0, "16-byte aligned warp slots");

// Dynamic shared memory of step_kernel_multi<S, MODE, AAR>: the row prefetch slots, or 0
// where the kernel loads its rows directly (either collision takes the FP32 slots; FP16
// deviations stage their codes with BGK).
template <class S, int MODE, bool AAR>
__host__ __device__ constexpr int multi_prefetch_smem() {
  return !KSS_MULTI_PREFETCH || MODE != MODE_STD ? 0
         : std::is_same<S, float>::value ? kPfBytes
         : (std::is_same<S, __half>::value && !AAR) ? kPfBytesH
                                                    : 0;
}

// ---------------------------------------------------------------- accumulators ----
// FP32 storage: a thread adds its few cells (at most 4 rows x 4 cells) in plain FP32,
// then the warp combines the partials as double-floats (hi + lo, Knuth two-sum), so
// the warp sums keep ~48 bits; FP64 storage: plain double.
template <class T> struct Acc;
template <> struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) { hi += v; }
  __device__ __forceinline__ void add2(float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float oh = __shfl_xor_sync(kFull, hi, off);
      const float ol = __shfl_xor_sync(kFull, lo, off);
      add2(oh);
      lo += ol;
    }
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};
template <> struct Acc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  }
  __device__ __forceinline__ double value() const { return v; }
};

// ---------------------------------------------------------------- stores ----
template <class T, int V = Vec<T>::N>
__device__ __forceinline__ void vstore(T* p, const T (&v)[V]) {
  using VT = typename VecT<T, V>::type;
  __stcs(reinterpret_cast<VT*>(p), make_vec<VT, T, V>(v));
}

// Populations of plane q: V cells loaded and decoded to the arithmetic type, or encoded
// and stored (streaming stores).  FP16 deviations move as 8- (V = 4) or 4-byte vectors.
template <class S, int V = Vec<S>::N, bool CG = false>
__device__ __forceinline__ void pop_vload(const S* p, bool ok, arith_t<S> (&v)[V], int q,
                                          const codec_t<S>& c) {
  if constexpr (std::is_same<S, __half>::value) {
    if (!ok) {
#pragma unroll
      for (int k = 0; k < V; ++k) v[k] = 0.f;
      return;
    }
    using VT = typename VecT<S, V>::type;
    const VT raw = ld_pop<CG>(reinterpret_cast<const VT*>(p));
    const __half2* h = reinterpret_cast<const __half2*>(&raw);
    // two codes per paired FMA (each half rounded as fmaf rounds it)
    const F2 inv = pack2(c.inv[q], c.inv[q]), base = pack2(c.base[q], c.base[q]);
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      const float2 a = __half22float2(h[k]);
      unpack2(fma2(pack2(a.x, a.y), inv, base), v[2 * k], v[2 * k + 1]);
    }
  } else {
    vload<S, V, CG>(p, ok, v);
  }
}

template <class S, int V = Vec<S>::N>
__device__ __forceinline__ void pop_vstore(S* p, const arith_t<S> (&v)[V], int q,
                                           const codec_t<S>& c) {
  if constexpr (std::is_same<S, __half>::value) {
    using VT = typename VecT<S, V>::type;
    VT raw;
    __half2* h = reinterpret_cast<__half2*>(&raw);
    // (f - b_q) s_q for two cells per paired subtract and multiply (the scalar roundings)
    const F2 base = pack2(c.base[q], c.base[q]), scale = pack2(c.scale[q], c.scale[q]);
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      float d0, d1;
      unpack2(mul2(sub2(pack2(v[2 * k], v[2 * k + 1]), base), scale), d0, d1);
      h[k] = __floats2half2_rn(d0, d1);
    }
    __stcs(reinterpret_cast<VT*>(p), raw);
  } else {
    vstore<S, V>(p, v);
  }
}

template <int V>
__device__ __forceinline__ void store_flags(uint8_t* p, uint32_t bits) {
  if constexpr (V == 4) {
    *reinterpret_cast<uint32_t*>(p) = bits;
  } else {
    *reinterpret_cast<uint16_t*>(p) = uint16_t(bits);
  }
}

// The region bytes of V cells (one per cell, in the low bytes).  An ordinary load: the
// step rewrites them later in the same launch.
template <int V>
__device__ __forceinline__ uint32_t load_bytes(const uint8_t* p) {
  if constexpr (V == 4) {
    return *reinterpret_cast<const uint32_t*>(p);
  } else {
    return *reinterpret_cast<const uint16_t*>(p);
  }
}

// ---------------------------------------------------------------- fused Kn/KL/neq ----
// Per-cell accumulators of the {Kn, KL, neq} set.
template <class T>
struct StdAcc {
  T kn[Vec<T>::N], neq[Vec<T>::N], kl[Vec<T>::N];
  T qe[Vec<T>::N];  // AAR steps only: the quasi-equilibrium sensor
};

// Relax one population of V cells in place (BGK: f <- f - (f - f^eq)/tau) and, on
// output steps, accumulate Kn += |x|, neq += |f^neq| and the Kullback-Leibler term
// f^eq phi(x) = f^neq x (phi(x)/x^2), x = f^neq / f^eq, by the series of phi.  The
// series is exact to FP32 for |x| < 1/16; a cell where that, or positivity, cannot be
// shown is deferred to fixup_kernel (see fused_row).
//
// FP32 (KSS_PAIRED_F32, default on): cells are processed in pairs with the paired FP32
// instructions; every operation and its rounding are those of the scalar form.
#ifndef KSS_PAIRED_F32
#define KSS_PAIRED_F32 1
#endif
// The two-relaxation update of AAR steps in paired FP32 instructions too (a build-time
// tuning knob, -DKSS_AAR_PAIRED=0 for the scalar form; the results are the same).
#ifndef KSS_AAR_PAIRED
#define KSS_AAR_PAIRED 1
#endif
template <class T, bool OUT, bool COLLIDE>
__device__ __forceinline__ void relax_pop(T (&f)[Vec<T>::N], const T (&feq)[Vec<T>::N], T omega,
                                          StdAcc<T>& a) {
#if KSS_PAIRED_F32
  if constexpr (std::is_same<T, float>::value) {
    constexpr int N = Num<float>::kPhiFastOrder;
    const F2 nom = pack2(-omega, -omega);
#pragma unroll
    for (int k = 0; k < Vec<T>::N; k += 2) {
      const F2 F = pack2(f[k], f[k + 1]);
      const F2 fneq = sub2(F, pack2(feq[k], feq[k + 1]));
      if (OUT) {
        const F2 x = mul2(fneq, pack2(Num<float>::rcp(feq[k]), Num<float>::rcp(feq[k + 1])));
        float x0, x1, n0, n1;
        unpack2(x, x0, x1);
        unpack2(fneq, n0, n1);
        a.kn[k] += fabsf(x0);
        a.kn[k + 1] += fabsf(x1);
        a.neq[k] += fabsf(n0);
        a.neq[k + 1] += fabsf(n1);
        // phi(x)/x^2 by Horner from the top coefficient, as phi_over_x2
        F2 acc = pack2(float(PhiCoef<N>::value), float(PhiCoef<N>::value));
        constexpr float kC[8] = {0.f, 0.f, float(PhiCoef<2>::value), float(PhiCoef<3>::value),
                                 float(PhiCoef<4>::value), float(PhiCoef<5>::value),
                                 float(PhiCoef<6>::value), float(PhiCoef<7>::value)};
        static_assert(N <= 7, "coefficient table");
#pragma unroll
        for (int n = N - 1; n >= 2; --n) acc = fma2(acc, x, pack2(kC[n], kC[n]));
        const F2 kl = fma2(mul2(fneq, x), acc, pack2(a.kl[k], a.kl[k + 1]));
        unpack2(kl, a.kl[k], a.kl[k + 1]);
      }
      if (COLLIDE) {
        const F2 nf = fma2(nom, fneq, F);
        unpack2(nf, f[k], f[k + 1]);
      }
    }
    return;
  }
#endif
#pragma unroll
  for (int k = 0; k < Vec<T>::N; ++k) {
    const T fneq = f[k] - feq[k];
    if (OUT) {
      const T x = fneq * Num<T>::rcp(feq[k]);
      a.kn[k] += fabs(x);
      a.neq[k] += fabs(fneq);
      a.kl[k] = fma(fneq * x, phi_over_x2<T, Num<T>::kPhiFastOrder>(x), a.kl[k]);
    }
    if (COLLIDE) f[k] = fma(-omega, fneq, f[k]);
  }
}

// The pair of opposite populations (+c, -c) with c.u = cu: f^eq = w rho (base + 9/2 cu^2
// +- 3 cu); both relaxed and (STORE) written out.  AAR: the cells whose region byte (in
// mbits, one per cell) is set take the two-relaxation update of cell_update, which
// couples the pair; the others the BGK update, bit for bit.
template <class S, bool OUT, bool STORE, int QP, int QM, bool AAR = false>
__device__ __forceinline__ void pair_pops(arith_t<S> (&fp)[Vec<S>::N], arith_t<S> (&fm)[Vec<S>::N],
                                          const arith_t<S> (&cu)[Vec<S>::N],
                                          const arith_t<S> (&base)[Vec<S>::N],
                                          const arith_t<S> (&rw)[Vec<S>::N], arith_t<S> omega,
                                          StdAcc<arith_t<S>>& a, S* dst_p, S* dst_m,
                                          const codec_t<S>& codec, bool cv, uint32_t mbits = 0,
                                          const Trt<arith_t<S>>& trt = Trt<arith_t<S>>{}) {
  using T = arith_t<S>;
  constexpr int V = Vec<S>::N;
  T ep[V], em[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const T t = fma(T(4.5) * cu[k], cu[k], base[k]);
    ep[k] = Num<T>::mul(rw[k], fma(T(3), cu[k], t));
    em[k] = Num<T>::mul(rw[k], fma(T(-3), cu[k], t));
  }
  if constexpr (AAR) {
    relax_pop<T, OUT, false>(fp, ep, omega, a);  // the sensors only
    relax_pop<T, OUT, false>(fm, em, omega, a);
    if (STORE) {
#if KSS_PAIRED_F32 && KSS_AAR_PAIRED
      if constexpr (std::is_same<T, float>::value) {
        // two cells per paired instruction, the roundings of the scalar form below
#pragma unroll
        for (int k = 0; k < V; k += 2) {
          const bool s0 = ((mbits >> (8 * k)) & 0xffu) != 0u;
          const bool s1 = ((mbits >> (8 * k + 8)) & 0xffu) != 0u;
          const F2 nA = pack2(s0 ? -trt.a : -omega, s1 ? -trt.a : -omega);
          const F2 nB = pack2(s0 ? -trt.b : -0.f, s1 ? -trt.b : -0.f);
          const F2 P = pack2(fp[k], fp[k + 1]), M = pack2(fm[k], fm[k + 1]);
          const F2 np = sub2(P, pack2(ep[k], ep[k + 1]));
          const F2 nm = sub2(M, pack2(em[k], em[k + 1]));
          if (OUT) {
            float d0, d1;
            unpack2(sub2(np, nm), d0, d1);
            a.qe[k] += fabsf(d0);
            a.qe[k + 1] += fabsf(d1);
          }
          unpack2(fma2(nB, nm, fma2(nA, np, P)), fp[k], fp[k + 1]);
          unpack2(fma2(nB, np, fma2(nA, nm, M)), fm[k], fm[k + 1]);
        }
      } else
#endif
      {
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const bool sw = ((mbits >> (8 * k)) & 0xffu) != 0u;
          const T A = sw ? trt.a : omega, B = sw ? trt.b : T(0);
          const T np = fp[k] - ep[k], nm = fm[k] - em[k];
          if (OUT) a.qe[k] += fabs(np - nm);
          fp[k] = fma(-B, nm, fma(-A, np, fp[k]));
          fm[k] = fma(-B, np, fma(-A, nm, fm[k]));
        }
      }
      if (cv) {
        pop_vstore<S>(dst_p, fp, QP, codec);
        pop_vstore<S>(dst_m, fm, QM, codec);
      }
    }
    return;
  }
  relax_pop<T, OUT, STORE>(fp, ep, omega, a);
  if (STORE && cv) pop_vstore<S>(dst_p, fp, QP, codec);
  relax_pop<T, OUT, STORE>(fm, em, omega, a);
  if (STORE && cv) pop_vstore<S>(dst_m, fm, QM, codec);
}

// Which of {Kn, KL, neq} (and, on AAR steps, qe) a flag tests (ids validated on the
// host); decided once per thread so the per-cell choice is a few selects.
struct Pick3 {
  bool is_kn, is_kl, is_qe;
  __device__ explicit Pick3(int id) : is_kn(id == S_KN), is_kl(id == S_KL), is_qe(id == S_QE) {}
  template <class T>
  __device__ __forceinline__ T operator()(T kn, T kl, T neq) const {
    return is_kn ? kn : (is_kl ? kl : neq);
  }
  template <class T>
  __device__ __forceinline__ T operator()(T kn, T kl, T neq, T qe) const {
    return is_kn ? kn : (is_kl ? kl : (is_qe ? qe : neq));
  }
};

// The nine populations of cell (i, j) as the step sees them (pulled when PULL), for the
// exact recomputation of deferred cells.
template <class S, bool PULL, bool CG = false>
__device__ __forceinline__ void reload_cell(const StepParams<S>& p, int i, int j,
                                            arith_t<S> (&c)[9]) {
  constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    int si = i, sj = j;
    if (PULL) {
      si = i - cx[q];
      sj = j - cy[q];
      si = si < 0 ? si + p.nx : (si >= p.nx ? si - p.nx : si);
      if (!p.slab) sj = sj < 0 ? sj + p.ny : (sj >= p.ny ? sj - p.ny : sj);
    }
    c[q] = decode<S>(ld_pop<CG>(p.src + q * p.plane + (long long)sj * p.pitch + si), q, p.codec);
  }
}

// Append the deferred cells among this lane's V cells of row j (flag bytes 0x40 in
// fbits) to a list through one atomic on `counter` per warp; entries at or beyond `cap`
// are dropped (the caller detects that from the counter).  All lanes must call.
template <int V>
__device__ __forceinline__ void append_deferred(uint32_t fbits, int i0, int j, int nx,
                                                uint32_t* counter, uint32_t* list, uint32_t cap) {
  const uint32_t dbits = fbits & 0x40404040u;
  if (!__any_sync(kFull, dbits != 0)) return;
  const int lane = threadIdx.x & 31;
  const int nd = __popc(dbits);
  int incl = nd;  // inclusive prefix sum over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(counter, uint32_t(total));
  base = __shfl_sync(kFull, base, 31) + uint32_t(incl - nd);
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if ((dbits >> (8 * k)) & 0x40u) {
      if (base < cap) list[base] = uint32_t(j) * uint32_t(nx) + uint32_t(i0 + k);
      ++base;
    }
  }
}

// Partial sums above the warp level: FP32 storage keeps them as double-floats (hi + lo,
// ~48 bits) so that no FP64 arithmetic (a slow pipe on GB300) sits in any CTA's
// epilogue; FP64 storage uses double.  Stored in the double slots of part_sum.
template <class T> struct Red;
template <> struct Red<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(const Red& o) {
    const float s = hi + o.hi;
    const float bp = s - hi;
    lo += ((hi - (s - bp)) + (o.hi - bp)) + o.lo;
    hi = s;
  }
  __device__ __forceinline__ Red shfl_xor(int off) const {
    return Red{__shfl_xor_sync(kFull, hi, off), __shfl_xor_sync(kFull, lo, off)};
  }
  __device__ __forceinline__ void store(double* p) const {
    *reinterpret_cast<float2*>(p) = make_float2(hi, lo);
  }
  __device__ static __forceinline__ Red load(const double* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return Red{v.x, v.y};
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
  __device__ static __forceinline__ Red of(const Acc<float>& a) { return Red{a.hi, a.lo}; }
};
template <> struct Red<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(const Red& o) { v += o.v; }
  __device__ __forceinline__ Red shfl_xor(int off) const {
    return Red{__shfl_xor_sync(kFull, v, off)};
  }
  __device__ __forceinline__ void store(double* p) const { *p = v; }
  __device__ static __forceinline__ Red load(const double* p) { return Red{__ldcg(p)}; }
  __device__ __forceinline__ double value() const { return v; }
  __device__ static __forceinline__ Red of(const Acc<double>& a) { return Red{a.v}; }
};

// The last CTA's reduction of the per-CTA partials, in CTA order within each thread and
// a fixed shuffle/shared-memory tree across threads (bitwise reproducible).
template <class S, int NTHREADS>
__device__ __forceinline__ void finalize_sums(const double* part_sum, const uint32_t* part_cnt,
                                              int nblocks, double* out_sums,
                                              unsigned long long* out_counts) {
  using T = arith_t<S>;
  __shared__ Red<T> f_sum[NTHREADS / 32][3];
  __shared__ unsigned long long f_cnt[NTHREADS / 32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Red<T> t[3];
  unsigned long long u[3] = {0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += NTHREADS) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      t[m].add(Red<T>::load(part_sum + 3 * b + m));
      u[m] += __ldcg(part_cnt + 4 * b + m);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      t[m].add(t[m].shfl_xor(off));
      u[m] += __shfl_xor_sync(kFull, u[m], off);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      f_sum[warp][m] = t[m];
      f_cnt[warp][m] = u[m];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      Red<T> r = f_sum[0][m];
      unsigned long long c = f_cnt[0][m];
      for (int w = 1; w < NTHREADS / 32; ++w) {
        r.add(f_sum[w][m]);
        c += f_cnt[w][m];
      }
      out_sums[m] = r.value();
      out_counts[m] = c;
    }
  }
}

template <class S, int NTHREADS>
__device__ __forceinline__ void finalize_partials(const StepParams<S>& p, int nblocks) {
  finalize_sums<S, NTHREADS>(p.part_sum, p.part_cnt, nblocks, p.stat_sums, p.stat_counts);
  if (threadIdx.x == 0) *p.done = 0u;  // ready for the next launch (stream-ordered)
}

// Is sensor s in the compiled set of MODE?
template <int MODE>
__host__ __device__ constexpr bool mode_has(int s) {
  return MODE == MODE_FULL ? true : (MODE == MODE_STD ? ((kStdMask >> s) & 1u) != 0 : false);
}

// ---------------------------------------------------------------- deferred cells ----
// Exact {Kn, KL, neq}, flags and counts of one deferred cell (i, j), recomputed from
// the pass's source buffer (which the pass does not modify) with the exact per-cell
// arithmetic of the full sensor set (cell_update).  Returns the refine/switch/non-
// positive tags; the tile counts are corrected here.
template <class S, bool PULL, bool CG = false>
__device__ __forceinline__ uint32_t fix_cell(const StepParams<S>& p, const Pick3& pr,
                                             const Pick3& ps, int i, int j) {
  using T = arith_t<S>;
  T cell[9], dummy[9];
  reload_cell<S, PULL, CG>(p, i, j, cell);
  CellOut<T> co;
  cell_update<T, MODE_STD, false>(cell, p.omega, p.tau, dummy, co, p.trt);
  const T kn = co.sv[S_KN], kl = co.sv[S_KL], neq = co.sv[S_NEQ], qe = co.sv[S_QE];
  const bool rr = pr(kn, kl, neq, qe) > p.thr_r;
  const bool ss = p.switch_on && (ps(kn, kl, neq, qe) > p.thr_s);
  const bool np = co.nonpos;
  const long long off = (long long)j * p.pitch + i;
  p.flags[off] = uint8_t(uint32_t(rr) | (uint32_t(ss) << 1) | (uint32_t(np) << 7));
  if (p.rec_slot[S_KN] >= 0) p.rec[p.rec_slot[S_KN] * p.plane + off] = kn;
  if (p.rec_slot[S_KL] >= 0) p.rec[p.rec_slot[S_KL] * p.plane + off] = kl;
  if (p.rec_slot[S_NEQ] >= 0) p.rec[p.rec_slot[S_NEQ] * p.plane + off] = neq;
  if (p.trt.qe && p.rec_slot[S_QE] >= 0) p.rec[p.rec_slot[S_QE] * p.plane + off] = qe;
  return uint32_t(rr) | (uint32_t(ss) << 1) | (uint32_t(np) << 2);
}

// ---------------------------------------------------------------- one row, paired ----
// The plain and {Kn, KL, neq} rows of FP32 arithmetic (FP32 storage and FP16 deviations)
// with every operation that is the same for two cells issued as one paired instruction
// (f32x2.cuh): moments, velocities, the equilibrium, the relaxation, the Kullback-Leibler
// series and the codec.  Each operation and its rounding are exactly those of the scalar
// row (fused_row below and cell_update), so the populations, sensors, flags and sums are
// the same bit for bit; only the instruction count differs.  A lane's V = 4 cells are the
// pairs (0, 1) and (2, 3).  Build knob: -DKSS_ROW_PAIRED=0 takes the scalar row.
#ifndef KSS_ROW_PAIRED
#define KSS_ROW_PAIRED 1
#endif

__device__ __forceinline__ F2 splat2(float c) { return pack2(c, c); }

// |a| of both halves (the sign bits cleared).
__device__ __forceinline__ F2 abs2(F2 a) {
  F2 r;
  r.v = a.v & 0x7fffffff7fffffffull;
  return r;
}

// Reciprocal of both halves (the hardware approximation of Num<float>::rcp).
__device__ __forceinline__ F2 rcp2(F2 a) {
  float x, y;
  unpack2(a, x, y);
  return pack2(Num<float>::rcp(x), Num<float>::rcp(y));
}

// Codec constants of one weight class (all populations of equal weight share b_q and s_q):
// decode f = b + h / s as one FMA per value, encode (f - b) s as f s - s b (s a power of
// two, so that is (f - b) s with the same single rounding).
template <class S>
struct PairCodec {
  __device__ PairCodec(const codec_t<S>&, int) {}
};
template <>
struct PairCodec<__half> {
  F2 inv, base, scale, nsb;
  __device__ PairCodec(const codec_t<__half>& c, int q)
      : inv(splat2(c.inv[q])), base(splat2(c.base[q])), scale(splat2(c.scale[q])),
        nsb(splat2(-(c.scale[q] * c.base[q]))) {}
};

// Stores of the paired row under a per-lane condition ok (the lane's cells lie in the
// lattice).  With KSS_PRED_STORES each is one predicated store instruction, so the row
// body has no branch per store and its arithmetic forms one block that the compiler can
// schedule as a whole (the values are computed by every lane).  Build knob:
// -DKSS_PRED_STORES=0 takes an ordinary conditional store.
#ifndef KSS_PRED_STORES
#define KSS_PRED_STORES 1
#endif
__device__ __forceinline__ void st_cs_if(uint2* p, uint2 v, bool ok) {
#if KSS_PRED_STORES
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %3, 0;\n @q st.global.cs.v2.b32 [%0], {%1, %2};\n}"
      ::"l"(p), "r"(v.x), "r"(v.y), "r"(int(ok)) : "memory");
#else
  if (ok) __stcs(p, v);
#endif
}
__device__ __forceinline__ void st_cs_if(float4* p, float4 v, bool ok) {
#if KSS_PRED_STORES
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n"
      " @q st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};\n}"
      ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(int(ok)) : "memory");
#else
  if (ok) __stcs(p, v);
#endif
}
__device__ __forceinline__ void st_u32_if(uint8_t* p, uint32_t v, bool ok) {
#if KSS_PRED_STORES
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.global.b32 [%0], %1;\n}"
               ::"l"(p), "r"(v), "r"(int(ok)) : "memory");
#else
  if (ok) *reinterpret_cast<uint32_t*>(p) = v;
#endif
}

// Store the four cells of one population (two pairs), encoded for FP16 deviations, where
// ok holds.
template <class S>
__device__ __forceinline__ void pop_store2(S* p, const F2 (&f)[2], const PairCodec<S>& pc,
                                           bool ok) {
  if constexpr (std::is_same<S, __half>::value) {
    uint2 raw;
    float a, b;
    unpack2(fma2(f[0], pc.scale, pc.nsb), a, b);
    const __half2 h0 = __floats2half2_rn(a, b);
    unpack2(fma2(f[1], pc.scale, pc.nsb), a, b);
    const __half2 h1 = __floats2half2_rn(a, b);
    raw.x = *reinterpret_cast<const unsigned int*>(&h0);
    raw.y = *reinterpret_cast<const unsigned int*>(&h1);
    st_cs_if(reinterpret_cast<uint2*>(p), raw, ok);
  } else {
    float a, b, c, d;
    unpack2(f[0], a, b);
    unpack2(f[1], c, d);
    st_cs_if(reinterpret_cast<float4*>(p), make_float4(a, b, c, d), ok);
  }
}

// a b rounded once, for a product whose only use is a subtraction.  The device compiler
// contracts a paired multiply into a following paired subtract (one rounding instead of
// two) even with explicit round-to-nearest modifiers; an FMA whose addend is a zero it
// cannot see (a kernel parameter) is the same rounded product and cannot be contracted.
// This keeps f^eq rounded exactly as the scalar arithmetic rounds it (Num<T>::mul).
__device__ __forceinline__ F2 product2(F2 a, F2 b, F2 zero) { return fma2(a, b, zero); }

// Per-cell accumulators of the paired row: Kn and neq per pair, KL per pair.
struct PairAcc {
  F2 kn[2], neq[2], kl[2];
  F2 qe[2];  // two-relaxation steps only: the quasi-equilibrium sensor
};

// Relax one population (two pairs) toward its equilibrium feq and accumulate the sensor
// terms, as relax_pop does per pair.
template <bool OUT, bool COLLIDE = true>
__device__ __forceinline__ void relax2(F2 (&f)[2], const F2 (&feq)[2], F2 nom, PairAcc& a) {
  constexpr int N = Num<float>::kPhiFastOrder;
  static_assert(N == 5, "series order of the paired row");
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const F2 fneq = sub2(f[m], feq[m]);
    if (OUT) {
      const F2 x = mul2(fneq, rcp2(feq[m]));
      // |x| and |f^neq| accumulate per cell (a scalar add with the absolute value as an
      // operand modifier is one instruction; the paired add would need the sign bits
      // cleared first)
      float x0, x1, n0, n1, k0, k1, e0, e1;
      unpack2(x, x0, x1);
      unpack2(fneq, n0, n1);
      unpack2(a.kn[m], k0, k1);
      unpack2(a.neq[m], e0, e1);
      a.kn[m] = pack2(k0 + fabsf(x0), k1 + fabsf(x1));
      a.neq[m] = pack2(e0 + fabsf(n0), e1 + fabsf(n1));
      F2 acc = splat2(float(PhiCoef<5>::value));
      acc = fma2(acc, x, splat2(float(PhiCoef<4>::value)));
      acc = fma2(acc, x, splat2(float(PhiCoef<3>::value)));
      acc = fma2(acc, x, splat2(float(PhiCoef<2>::value)));
      a.kl[m] = fma2(mul2(fneq, x), acc, a.kl[m]);
    }
    if (COLLIDE) f[m] = fma2(nom, fneq, f[m]);
  }
}

// The opposite pair (QP, QM) with c.u = cu: f^eq = w rho (base + 9/2 cu^2 +- 3 cu),
// relaxed and (STORE) written.
template <class S, bool OUT, bool STORE>
__device__ __forceinline__ void pair2(F2 (&fp)[2], F2 (&fm)[2], const F2 (&cu)[2],
                                      const F2 (&base)[2], const F2 (&rw)[2], F2 nom, F2 zero,
                                      PairAcc& a, S* dst_p, S* dst_m, const PairCodec<S>& pc,
                                      bool cv) {
  F2 ep[2], em[2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const F2 t = fma2(mul2(splat2(4.5f), cu[m]), cu[m], base[m]);
    ep[m] = product2(rw[m], fma2(splat2(3.f), cu[m], t), zero);
    em[m] = product2(rw[m], fma2(splat2(-3.f), cu[m], t), zero);
  }
  relax2<OUT>(fp, ep, nom, a);
  if (STORE) pop_store2<S>(dst_p, fp, pc, cv);
  relax2<OUT>(fm, em, nom, a);
  if (STORE) pop_store2<S>(dst_m, fm, pc, cv);
}

// The same pair on a two-relaxation step (adaptive algorithm refinement): the sensors of
// relax2, then in the cells whose region byte (in mbits) is set the coupled update
// f'_q = f_q - A f^neq_q - B f^neq_-q of cell_update, and in the others BGK (A = 1/tau,
// B = 0, which adds a zero product): the operations and roundings of pair_pops.
template <class S, bool OUT, bool STORE>
__device__ __forceinline__ void pair2_aar(F2 (&fp)[2], F2 (&fm)[2], const F2 (&cu)[2],
                                          const F2 (&base)[2], const F2 (&rw)[2], F2 nom,
                                          F2 zero, PairAcc& a, S* dst_p, S* dst_m,
                                          const PairCodec<S>& pc, bool cv, uint32_t mbits,
                                          float omega, const Trt<float>& trt) {
  F2 ep[2], em[2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const F2 t = fma2(mul2(splat2(4.5f), cu[m]), cu[m], base[m]);
    ep[m] = product2(rw[m], fma2(splat2(3.f), cu[m], t), zero);
    em[m] = product2(rw[m], fma2(splat2(-3.f), cu[m], t), zero);
  }
  relax2<OUT, false>(fp, ep, nom, a);  // the sensors only
  relax2<OUT, false>(fm, em, nom, a);
  if (!STORE) return;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const bool s0 = ((mbits >> (16 * m)) & 0xffu) != 0u;
    const bool s1 = ((mbits >> (16 * m + 8)) & 0xffu) != 0u;
    const F2 nA = pack2(s0 ? -trt.a : -omega, s1 ? -trt.a : -omega);
    const F2 nB = pack2(s0 ? -trt.b : -0.f, s1 ? -trt.b : -0.f);
    const F2 np = sub2(fp[m], ep[m]), nm = sub2(fm[m], em[m]);
    if (OUT) {
      float d0, d1, q0, q1;
      unpack2(sub2(np, nm), d0, d1);
      unpack2(a.qe[m], q0, q1);
      a.qe[m] = pack2(q0 + fabsf(d0), q1 + fabsf(d1));
    }
    fp[m] = fma2(nB, nm, fma2(nA, np, fp[m]));
    fm[m] = fma2(nB, np, fma2(nA, nm, fm[m]));
  }
  pop_store2<S>(dst_p, fp, pc, cv);
  pop_store2<S>(dst_m, fm, pc, cv);
}

template <class S, int MODE, bool STORE, bool AAR = false>
__device__ __forceinline__ uint32_t fused_row_paired(const StepParams<S>& p,
                                                     F2 (&f)[9][2], int i0, int j, bool cv,
                                                     Acc<float>& a_rho, Acc<float>& a_jx,
                                                     Acc<float>& a_jy, uint32_t mbits = 0) {
  constexpr bool OUT = MODE != MODE_PLAIN;
  // row parts are the same for the whole warp (one row per warp): the lane's column is
  // added last, so that they stay warp-uniform
  const long long row = (long long)j * p.pitch;
  // cells past the row end hold padding or stale data: zeroed (they add nothing to the
  // sums, and their NaN sensors raise no flag)
  const int nvalid = cv ? min(4, p.nx - i0) : 0;
  if (nvalid < 4) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      float c0, c1, c2, c3;
      unpack2(f[q][0], c0, c1);
      unpack2(f[q][1], c2, c3);
      f[q][0] = pack2(nvalid > 0 ? c0 : 0.f, nvalid > 1 ? c1 : 0.f);
      f[q][1] = pack2(nvalid > 2 ? c2 : 0.f, 0.f);
    }
  }
  F2 rw1[2], ux[2], uy[2], base[2];
  float rs[4], xs[4], ys[4];
  PairAcc a;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const F2 rho = add2(add2(add2(add2(f[0][m], f[1][m]), add2(f[2][m], f[3][m])),
                             add2(add2(f[4][m], f[5][m]), add2(f[6][m], f[7][m]))),
                        f[8][m]);
    const F2 jx = sub2(add2(add2(f[1][m], f[5][m]), f[8][m]),
                       add2(add2(f[3][m], f[6][m]), f[7][m]));
    const F2 jy = sub2(add2(add2(f[2][m], f[5][m]), f[6][m]),
                       add2(add2(f[4][m], f[7][m]), f[8][m]));
    const F2 ir = rcp2(rho);
    ux[m] = mul2(jx, ir);
    uy[m] = mul2(jy, ir);
    base[m] = fma2(splat2(-1.5f), fma2(ux[m], ux[m], mul2(uy[m], uy[m])), splat2(1.f));
    rw1[m] = mul2(rho, splat2(float(1.0 / 9.0)));
    unpack2(rho, rs[2 * m], rs[2 * m + 1]);
    unpack2(jx, xs[2 * m], xs[2 * m + 1]);
    unpack2(jy, ys[2 * m], ys[2 * m + 1]);
    a.kn[m] = a.neq[m] = a.kl[m] = a.qe[m] = splat2(0.f);
  }
  if (OUT) {  // the row's moments, cell by cell in order (as the scalar row adds them)
    a_rho.add(((rs[0] + rs[1]) + rs[2]) + rs[3]);
    a_jx.add(((xs[0] + xs[1]) + xs[2]) + xs[3]);
    a_jy.add(((ys[0] + ys[1]) + ys[2]) + ys[3]);
  }
  const F2 nom = splat2(-p.omega), zero = splat2(p.zero);
  const PairCodec<S> c0(p.codec, 0), c1(p.codec, 1), c5(p.codec, 5);
  S* const dst = p.dst + row;
  {
    F2 feq[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) feq[m] = product2(mul2(splat2(4.f), rw1[m]), base[m], zero);
    relax2<OUT>(f[0], feq, nom, a);
    if (STORE) pop_store2<S>(dst + i0, f[0], c0, cv);
  }
  // the four opposite pairs: (1, 3) c.u = +-ux; (2, 4) +-uy; (5, 7) +-(ux + uy);
  // (6, 8) +-(uy - ux)
  auto pair = [&](F2 (&fp)[2], F2 (&fm)[2], const F2 (&cu)[2], const F2 (&rw)[2], int qp,
                  int qm, const PairCodec<S>& pc) {
    if constexpr (AAR) {
      pair2_aar<S, OUT, STORE>(fp, fm, cu, base, rw, nom, zero, a, dst + qp * p.plane + i0,
                               dst + qm * p.plane + i0, pc, cv, p.region ? mbits : 0u,
                               p.omega, p.trt);
    } else {
      pair2<S, OUT, STORE>(fp, fm, cu, base, rw, nom, zero, a, dst + qp * p.plane + i0,
                           dst + qm * p.plane + i0, pc, cv);
    }
  };
  pair(f[1], f[3], ux, rw1, 1, 3, c1);
  pair(f[2], f[4], uy, rw1, 2, 4, c1);
  {
    F2 sd[2], rw2[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      sd[m] = add2(ux[m], uy[m]);
      rw2[m] = mul2(splat2(0.25f), rw1[m]);
    }
    pair(f[5], f[7], sd, rw2, 5, 7, c5);
#pragma unroll
    for (int m = 0; m < 2; ++m) sd[m] = sub2(uy[m], ux[m]);
    pair(f[6], f[8], sd, rw2, 6, 8, c5);
  }
  uint32_t fbits = 0;
  if (OUT) {
    const Pick3 pr(p.refine_s), ps(p.switch_s);
    float kn[4], neq[4], kl[4], rw[4], bs[4], qe[4];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      unpack2(a.qe[m], qe[2 * m], qe[2 * m + 1]);
      unpack2(a.kn[m], kn[2 * m], kn[2 * m + 1]);
      unpack2(a.neq[m], neq[2 * m], neq[2 * m + 1]);
      unpack2(abs2(a.kl[m]), kl[2 * m], kl[2 * m + 1]);
      unpack2(rw1[m], rw[2 * m], rw[2 * m + 1]);
      unpack2(base[m], bs[2 * m], bs[2 * m + 1]);
    }
    // rho > 0 and |u|^2 < 0.3 make every f^eq_q >= 0.05 w_q rho > 0, and Kn < 1/16
    // bounds every |x_q| (see fused_row): otherwise the cell is deferred.  The common
    // choice (refine on Kn, switch on neq) takes its sensors without a selection.
    if (!AAR && p.refine_s == S_KN && p.switch_s == S_NEQ) {  // (uniform)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool fast = (rw[k] > 0.f) & (bs[k] > 0.55f) & (kn[k] < 0.0625f);
        const bool r = kn[k] > p.thr_r;
        const bool sw = p.switch_on && (neq[k] > p.thr_s);
        const uint32_t b = fast ? (uint32_t(r) | (uint32_t(sw) << 1)) : kFlagDeferred;
        fbits |= b << (8 * k);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool fast = (rw[k] > 0.f) & (bs[k] > 0.55f) & (kn[k] < 0.0625f);
        const bool r =
            (AAR ? pr(kn[k], kl[k], neq[k], qe[k]) : pr(kn[k], kl[k], neq[k])) > p.thr_r;
        const bool sw = p.switch_on && ((AAR ? ps(kn[k], kl[k], neq[k], qe[k])
                                             : ps(kn[k], kl[k], neq[k])) > p.thr_s);
        const uint32_t b = fast ? (uint32_t(r) | (uint32_t(sw) << 1)) : kFlagDeferred;
        fbits |= b << (8 * k);
      }
    }
    if (nvalid < 4) fbits &= nvalid > 0 ? 0xffffffffu >> (32 - 8 * nvalid) : 0u;
    // (uniform conditions on the recorded set; the lane's own condition is the store's)
    st_u32_if(p.flags + row + i0, fbits, cv);
    // (a deferred cell's byte is 0x40: its region byte is set by the epilogue)
    if (AAR && STORE && p.region)
      st_u32_if(p.region + row + i0, (fbits >> 1) & 0x01010101u, cv);
    if (AAR && p.rec_slot[S_QE] >= 0)
      st_cs_if(reinterpret_cast<float4*>(p.rec + p.rec_slot[S_QE] * p.plane + row + i0),
               make_float4(qe[0], qe[1], qe[2], qe[3]), cv);
    if (p.rec_slot[S_KN] >= 0)
      st_cs_if(reinterpret_cast<float4*>(p.rec + p.rec_slot[S_KN] * p.plane + row + i0),
               make_float4(kn[0], kn[1], kn[2], kn[3]), cv);
    if (p.rec_slot[S_KL] >= 0)
      st_cs_if(reinterpret_cast<float4*>(p.rec + p.rec_slot[S_KL] * p.plane + row + i0),
               make_float4(kl[0], kl[1], kl[2], kl[3]), cv);
    if (p.rec_slot[S_NEQ] >= 0)
      st_cs_if(reinterpret_cast<float4*>(p.rec + p.rec_slot[S_NEQ] * p.plane + row + i0),
               make_float4(neq[0], neq[1], neq[2], neq[3]), cv);
  }
  return fbits;
}

// ---------------------------------------------------------------- one row ----
// Everything after the loads for one row of V-cell vectors: moments, equilibrium,
// sensors of the compiled set, flags, BGK collision, and the stores of the new
// populations, the flag bytes and the recorded sensor fields.  ft holds the
// post-streaming populations of cells i0..i0+V-1 of row j.  Returns the lane's flag
// word (one byte per cell); the row's moments are added to the accumulators.  MULTI: the
// row of a multi-step launch (whose two-relaxation row keeps the scalar form: the paired
// one spills there and measured slower, 0.2257 vs 0.2133 ms per 4096^2 step, while it is
// faster in one-step launches, 0.2375 vs 0.2769 ms; both give the same results bit for
// bit).
template <class S, int MODE, bool PULL, bool STORE, bool AAR = false, bool MULTI = false>
__device__ __forceinline__ uint32_t fused_row(const StepParams<S>& p,
                                              arith_t<S> (&ft)[9][Vec<S>::N], int i0, int j,
                                              bool cv, Acc<arith_t<S>>& a_rho,
                                              Acc<arith_t<S>>& a_jx, Acc<arith_t<S>>& a_jy,
                                              uint32_t mbits = 0) {
  // (AAR: mbits holds the row's region bytes, loaded by the caller with the populations)
  using T = arith_t<S>;
  constexpr int V = Vec<S>::N;
  constexpr bool OUT = MODE != MODE_PLAIN;
  const long long off = (long long)j * p.pitch + i0;
  uint32_t fbits = 0;
  if constexpr (MODE == MODE_FULL) {
    // ---- all sensors of Table 1: cell-major, generic per-cell arithmetic ----
    T fo[9][V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      T c[9], o9[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) c[q] = ft[q][k];
      CellOut<T> co;
      cell_update<T, MODE, STORE, AAR>(c, p.omega, p.tau, o9, co, p.trt,
                                       ((mbits >> (8 * k)) & 0xffu) != 0u);
      const bool valid = cv && (i0 + k < p.nx);
      if (STORE) {
#pragma unroll
        for (int q = 0; q < 9; ++q) fo[q][k] = o9[q];
      }
      if (valid) {
        a_rho.add(co.rho);
        a_jx.add(co.jx);
        a_jy.add(co.jy);
      }
      const bool r = valid && (pick<T>(co.sv, p.refine_s) > p.thr_r);
      const bool sw = valid && p.switch_on && (pick<T>(co.sv, p.switch_s) > p.thr_s);
      const bool np = valid && co.nonpos;
      fbits |= (uint32_t(r) | (uint32_t(sw) << 1) | (uint32_t(np) << 7)) << (8 * k);
      // recorded sensors: one value per cell as soon as it is known (the lanes of a warp
      // still cover contiguous bytes), so no sensor values stay live across the cells
      if (valid) {
#pragma unroll
        for (int sid = 0; sid < S_COUNT; ++sid) {
          const int slot = p.rec_slot[sid];
          if (slot >= 0) p.rec[slot * p.plane + off + k] = co.sv[sid];
        }
      }
    }
    if (STORE && cv) {
#pragma unroll
      for (int q = 0; q < 9; ++q) pop_vstore<S>(p.dst + q * p.plane + off, fo[q], q, p.codec);
    }
    if (cv) {
      store_flags<V>(p.flags + off, fbits);
      if (AAR && STORE && p.region) store_flags<V>(p.region + off, (fbits >> 1) & 0x01010101u);
    }
  } else if constexpr (KSS_ROW_PAIRED && std::is_same<T, float>::value && V == 4 &&
                       !(AAR && MULTI)) {
    // ---- the same row in paired instructions (fused_row_paired) ----
    F2 f[9][2];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      f[q][0] = pack2(ft[q][0], ft[q][1]);
      f[q][1] = pack2(ft[q][2], ft[q][3]);
    }
    fbits = fused_row_paired<S, MODE, STORE, AAR>(p, f, i0, j, cv, a_rho, a_jx, a_jy, mbits);
  } else {
    // ---- plain stream + collide, or with the {Kn, KL, neq} sensor set:
    //      population-major so each population's vector is stored as soon as it
    //      is relaxed (fewer live registers) ----
    // cells past the row end (a ragged last vector, or a whole vector beyond it) hold
    // padding or stale staging data: zero them, so that they add nothing to the sums
    // and raise no flag (their sensors are NaN)
    const int nvalid = cv ? min(V, p.nx - i0) : 0;
    if (nvalid < V) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int k = 0; k < V; ++k)
          if (k >= nvalid) ft[q][k] = T(0);
    }
    // per cell: rho/9 (the rest and diagonal weights are exact power-of-two multiples:
    // 4/9 = 4 (1/9), 1/36 = (1/9)/4), u and 1 - 3/2 u^2; kept small for registers
    T rw1[V], ux[V], uy[V], base[V];
    StdAcc<T> a;
    T rs = T(0), xs = T(0), ys = T(0);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const T rho = ((ft[0][k] + ft[1][k]) + (ft[2][k] + ft[3][k])) +
                    ((ft[4][k] + ft[5][k]) + (ft[6][k] + ft[7][k])) + ft[8][k];
      const T jx = (ft[1][k] + ft[5][k] + ft[8][k]) - (ft[3][k] + ft[6][k] + ft[7][k]);
      const T jy = (ft[2][k] + ft[5][k] + ft[6][k]) - (ft[4][k] + ft[7][k] + ft[8][k]);
      const T ir = Num<T>::rcp(rho);
      ux[k] = Num<T>::mul(jx, ir);
      uy[k] = Num<T>::mul(jy, ir);
      base[k] = fma(T(-1.5), fma(ux[k], ux[k], uy[k] * uy[k]), T(1));
      rw1[k] = rho * T(1.0 / 9.0);
      a.kn[k] = a.neq[k] = a.kl[k] = T(0);
      if (AAR) a.qe[k] = T(0);
      if (OUT) {
        rs += rho;
        xs += jx;
        ys += jy;
      }
    }
    if (OUT) {
      a_rho.add(rs);
      a_jx.add(xs);
      a_jy.add(ys);
    }
    T feq[V];
    // q = 0 (rest)
#pragma unroll
    for (int k = 0; k < V; ++k) feq[k] = Num<T>::mul(T(4) * rw1[k], base[k]);
    relax_pop<T, OUT, STORE>(ft[0], feq, p.omega, a);
    if (STORE && cv) pop_vstore<S>(p.dst + 0 * p.plane + off, ft[0], 0, p.codec);
    // axis pairs (1, 3): c.u = +-ux ; (2, 4): +-uy ; diagonal pairs (5, 7): +-(ux + uy),
    // (6, 8): +-(uy - ux)
    pair_pops<S, OUT, STORE, 1, 3, AAR>(ft[1], ft[3], ux, base, rw1, p.omega, a,
                                        p.dst + 1 * p.plane + off, p.dst + 3 * p.plane + off,
                                        p.codec, cv, mbits, p.trt);
    pair_pops<S, OUT, STORE, 2, 4, AAR>(ft[2], ft[4], uy, base, rw1, p.omega, a,
                                        p.dst + 2 * p.plane + off, p.dst + 4 * p.plane + off,
                                        p.codec, cv, mbits, p.trt);
    {
      T sd[V];
#pragma unroll
      for (int k = 0; k < V; ++k) sd[k] = Num<T>::add(ux[k], uy[k]);
      T rw2[V];
#pragma unroll
      for (int k = 0; k < V; ++k) rw2[k] = T(0.25) * rw1[k];
      pair_pops<S, OUT, STORE, 5, 7, AAR>(ft[5], ft[7], sd, base, rw2, p.omega, a,
                                          p.dst + 5 * p.plane + off, p.dst + 7 * p.plane + off,
                                          p.codec, cv, mbits, p.trt);
#pragma unroll
      for (int k = 0; k < V; ++k) sd[k] = Num<T>::sub(uy[k], ux[k]);
      pair_pops<S, OUT, STORE, 6, 8, AAR>(ft[6], ft[8], sd, base, rw2, p.omega, a,
                                          p.dst + 6 * p.plane + off, p.dst + 8 * p.plane + off,
                                          p.codec, cv, mbits, p.trt);
    }
    if (OUT) {
      const Pick3 pr(p.refine_s), ps(p.switch_s);
#pragma unroll
      for (int k = 0; k < V; ++k) {
        // rho > 0 and |u|^2 < 0.3 make every f^eq_q >= 0.05 w_q rho > 0, and Kn < 1/16
        // bounds every |x_q|, so f_q = f^eq_q (1 + x_q) > 0 (nothing non-positive) and
        // the series of phi is exact to FP32.  Any other valid cell is deferred: its
        // flag byte is KSS_FLAG_DEFERRED only, it is not counted here, and it is
        // recomputed exactly from the unchanged source populations (CTA epilogue or
        // fixup_kernel).
        const bool fast = (rw1[k] > T(0)) & (base[k] > T(0.55)) & (a.kn[k] < T(0.0625));
        a.kl[k] = fabs(a.kl[k]);
        const T er = AAR ? pr(a.kn[k], a.kl[k], a.neq[k], a.qe[k]) : pr(a.kn[k], a.kl[k], a.neq[k]);
        const T es = AAR ? ps(a.kn[k], a.kl[k], a.neq[k], a.qe[k]) : ps(a.kn[k], a.kl[k], a.neq[k]);
        const bool r = er > p.thr_r;  // NaN (zeroed padding cells) compares false
        const bool sw = p.switch_on && (es > p.thr_s);
        const uint32_t b = fast ? (uint32_t(r) | (uint32_t(sw) << 1)) : kFlagDeferred;
        fbits |= b << (8 * k);
      }
      // padding cells (zeroed above) raise no flag
      if (nvalid < V) fbits &= nvalid > 0 ? 0xffffffffu >> (32 - 8 * nvalid) : 0u;
      if (cv) {
        store_flags<V>(p.flags + off, fbits);
        // (a deferred cell's byte is 0x40: its region byte is set by the epilogue)
        if (AAR && STORE && p.region) store_flags<V>(p.region + off, (fbits >> 1) & 0x01010101u);
        if (p.rec_slot[S_KN] >= 0) vstore<T>(p.rec + p.rec_slot[S_KN] * p.plane + off, a.kn);
        if (p.rec_slot[S_KL] >= 0) vstore<T>(p.rec + p.rec_slot[S_KL] * p.plane + off, a.kl);
        if (p.rec_slot[S_NEQ] >= 0) vstore<T>(p.rec + p.rec_slot[S_NEQ] * p.plane + off, a.neq);
        if (AAR && p.rec_slot[S_QE] >= 0) vstore<T>(p.rec + p.rec_slot[S_QE] * p.plane + off, a.qe);
      }
    }
  }
  return fbits;
}

// One row of FP16 deviation codes, pulled and decoded into pairs: the nine 8-byte code
// vectors of the lane's 4 cells (rows j - cy_q), shifted along x as binary16 words (a cx =
// +1 population takes the code left of each cell: the left lane's last code by one
// shuffle of a 32-bit word, or lane 0's halo code; cx = -1 the mirror image, with the
// periodic seam and a row end inside the vector taking the halo code), then decoded
// f = b_q + h / s_q two codes per paired FMA.  The values are those of pop_vload and
// assemble_from_left / _right (the same codes, decoded by the same FMA).
__device__ __forceinline__ uint32_t half_bits(__half h) { return __half_as_ushort(h); }

// Source rows of q = 0..8 for row j (pull: row j - cy_q), warp-uniform.
__device__ __forceinline__ void half_rows(const StepParams<__half>& p, int j,
                                          const __half* (&r)[9]) {
  const __half* base = p.src + (long long)j * p.pitch;
  long long up, dn;  // rows j - 1 and j + 1
  row_neighbours(p, j, up, dn);
  r[0] = base;
  r[1] = base + 1 * p.plane;
  r[2] = base + 2 * p.plane + up;
  r[3] = base + 3 * p.plane;
  r[4] = base + 4 * p.plane + dn;
  r[5] = base + 5 * p.plane + up;
  r[6] = base + 6 * p.plane + up;
  r[7] = base + 7 * p.plane + dn;
  r[8] = base + 8 * p.plane + dn;
}

// The lane's code vectors w[q] of row j and the halo codes h[q] of the populations with
// cx = +1 (q = 1, 5, 8: column i0 - 1, periodic; lane 0) and cx = -1 (q = 3, 6, 7: column
// i0 + 4, or 0 at the row end; lane 31 and the lanes whose vector reaches the row end).
template <bool CG>
__device__ __forceinline__ void gather_half_row(const StepParams<__half>& p, int j, int i0,
                                                int lane, bool cv, uint2 (&w)[9],
                                                uint32_t (&h)[9]) {
  const __half* r[9];
  half_rows(p, j, r);
#pragma unroll
  for (int q = 0; q < 9; ++q)
    w[q] = cv ? ld_pop<CG>(reinterpret_cast<const uint2*>(r[q] + i0)) : make_uint2(0u, 0u);
  const bool tail = i0 + 4 >= p.nx;
  const int cl = i0 == 0 ? p.nx - 1 : i0 - 1, cr = tail ? 0 : i0 + 4;
  const bool hl = lane == 0 && cv, hr = cv && (lane == 31 || tail);
  h[1] = hl ? half_bits(ld_pop<CG>(r[1] + cl)) : 0u;
  h[5] = hl ? half_bits(ld_pop<CG>(r[5] + cl)) : 0u;
  h[8] = hl ? half_bits(ld_pop<CG>(r[8] + cl)) : 0u;
  h[3] = hr ? half_bits(ld_pop<CG>(r[3] + cr)) : 0u;
  h[6] = hr ? half_bits(ld_pop<CG>(r[6] + cr)) : 0u;
  h[7] = hr ? half_bits(ld_pop<CG>(r[7] + cr)) : 0u;
}

// Pull along x and decode: w and h as gather_half_row leaves them.
__device__ __forceinline__ void assemble_half_row(const StepParams<__half>& p, int i0, int lane,
                                                  uint2 (&w)[9], const uint32_t (&h)[9],
                                                  F2 (&f)[9][2]) {
  const bool tail = i0 + 4 >= p.nx;
  // cx = +1 (q = 1, 5, 8): codes [left, h0, h1, h2]
#pragma unroll
  for (int q : {1, 5, 8}) {
    uint32_t left = __shfl_up_sync(kFull, w[q].y, 1);
    if (lane == 0) left = h[q] << 16;
    const uint32_t x0 = __byte_perm(left, w[q].x, 0x5432), x1 = __byte_perm(w[q].x, w[q].y, 0x5432);
    w[q] = make_uint2(x0, x1);
  }
  // cx = -1 (q = 3, 6, 7): codes [h1, h2, h3, right]; cell nx - 1 takes column 0
#pragma unroll
  for (int q : {3, 6, 7}) {
    uint32_t right = __shfl_down_sync(kFull, w[q].x, 1);
    if (lane == 31 || tail) right = h[q];
    uint32_t x0 = __byte_perm(w[q].x, w[q].y, 0x5432), x1 = __byte_perm(w[q].y, right, 0x5432);
    if (tail) {  // a row end inside the vector (nx not a multiple of 4)
      if (i0 + 0 == p.nx - 1) x0 = (x0 & 0xffff0000u) | h[q];
      if (i0 + 1 == p.nx - 1) x0 = (x0 & 0x0000ffffu) | (h[q] << 16);
      if (i0 + 2 == p.nx - 1) x1 = (x1 & 0xffff0000u) | h[q];
    }
    w[q] = make_uint2(x0, x1);
  }
  const PairCodec<__half> c0(p.codec, 0), c1(p.codec, 1), c5(p.codec, 5);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const PairCodec<__half>& c = q == 0 ? c0 : (q <= 4 ? c1 : c5);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&w[q].x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&w[q].y));
    f[q][0] = fma2(pack2(a.x, a.y), c.inv, c.base);
    f[q][1] = fma2(pack2(b.x, b.y), c.inv, c.base);
  }
}

// ---- row prefetch of FP16 codes (the one-step {Kn, KL, neq} kernel) ----
// As the FP32 multi-step kernels stage rows (PfWarp), each warp copies its next row's
// codes into shared memory with cp.async before it computes the current row: nine 8-byte
// vectors per lane, and for each halo code the aligned 4-byte word that holds it (cp.async
// copies 4, 8 or 16 bytes; the row pitch is a multiple of 64 codes, so the word's other
// code is inside the row).  Build knob: -DKSS_F16_PREFETCH=0 loads every row directly.
#ifndef KSS_F16_PREFETCH
#define KSS_F16_PREFETCH 1
#endif


__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}

// Copies of row j's codes into the warp's slots (committed as one group).
__device__ __forceinline__ void pf_issue_half(const StepParams<__half>& p, PfWarpH* pw, int j,
                                              int i0, int lane, bool cv) {
  if (cv) {
    const __half* r[9];
    half_rows(p, j, r);
#pragma unroll
    for (int q = 0; q < 9; ++q) cp_async8(&pw->pop[q][lane], r[q] + i0);
    const bool tail = i0 + 4 >= p.nx;
    if (lane == 0) {
      const int cl = (i0 == 0 ? p.nx - 1 : i0 - 1) & ~1;
      cp_async4(&pw->hl[0], r[1] + cl);
      cp_async4(&pw->hl[1], r[5] + cl);
      cp_async4(&pw->hl[2], r[8] + cl);
    }
    if (lane == 31 || tail) {
      const int cr = tail ? 0 : i0 + 4;  // even: the word starts at the code
      cp_async4(&pw->hr[0][lane], r[3] + cr);
      cp_async4(&pw->hr[1][lane], r[6] + cr);
      cp_async4(&pw->hr[2][lane], r[7] + cr);
    }
  }
  cp_async_commit();
}

// The staged row back from the slots (after the copies of this lane completed).  Slots
// that no copy filled (a lane past the row end; the halo words of lanes that take no halo
// code) hold stale data: nothing reads it into a result (assemble_half_row takes halo codes
// only in lane 0, lane 31 and the row-end lane, and fused_row_paired zeroes the cells past
// the row end before any arithmetic), so it is read without a select.
__device__ __forceinline__ void pf_read_half(const StepParams<__half>& p, const PfWarpH* pw,
                                             int i0, int lane, bool cv, uint2 (&w)[9],
                                             uint32_t (&h)[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) w[q] = pw->pop[q][lane];
  const int cl = i0 == 0 ? p.nx - 1 : i0 - 1;
  const int sh = (cl & 1) ? 16 : 0;  // the code's half of its word
  h[1] = (pw->hl[0] >> sh) & 0xffffu;
  h[5] = (pw->hl[1] >> sh) & 0xffffu;
  h[8] = (pw->hl[2] >> sh) & 0xffffu;
  h[3] = pw->hr[0][lane] & 0xffffu;
  h[6] = pw->hr[1][lane] & 0xffffu;
  h[7] = pw->hr[2][lane] & 0xffffu;
}

// ---- eight cells per lane (the one-step FP16 {Kn, KL, neq} kernel) ----
// Each lane takes one 16-byte vector of eight codes per population, so a CTA row is 256
// columns wide and the per-row work (the copies and their addresses, the neighbour codes
// of the pull, tile counts, the deferred-cell gather, loop control) is shared by eight
// cells instead of four; the eight cells are evaluated as two groups of four
// (fused_row_paired), one after the other.  A warp's slots hold, per population, 34
// vectors: index 0 the word with the left halo code (in .w; lane 0's left neighbour),
// 1..32 the lanes' vectors, 33 the word with the right halo code (in .x; lane 31's right
// neighbour).  Lane L reads its left neighbour's last code from index L and its right
// neighbour's first code from index L + 2, so no lane selects among sources; the lane
// whose vector reaches the row end copies its right halo (column 0) into index L + 2,
// which no other copy fills (the lanes past the row end copy nothing).
struct PfWarpH8 {
  uint4 pop[9][34];
};
static_assert(sizeof(PfWarpH8) % 16 == 0, "16-byte aligned warp slots");

// Copies of row j's codes for the lane at column i0 (committed as one group).  tail: the
// lane's vector reaches the row end.
__device__ __forceinline__ void pf_issue_h8(const StepParams<__half>& p, PfWarpH8* pw, int j,
                                            int i0, int lane, bool cv, bool tail) {
  if (cv) {
    const __half* r[9];
    half_rows(p, j, r);
#pragma unroll
    for (int q = 0; q < 9; ++q) cp_async16(&pw->pop[q][lane + 1], r[q] + i0);
    if (lane == 0) {  // the word holding column i0 - 1 (periodic)
      const int cl = (i0 == 0 ? p.nx - 1 : i0 - 1) & ~1;
      cp_async4(&pw->pop[1][0].w, r[1] + cl);
      cp_async4(&pw->pop[5][0].w, r[5] + cl);
      cp_async4(&pw->pop[8][0].w, r[8] + cl);
    }
    if (lane == 31 || tail) {  // the word starting at column i0 + 8, or 0 at the row end
      const int cr = tail ? 0 : i0 + 8;
      cp_async4(&pw->pop[3][lane + 2].x, r[3] + cr);
      cp_async4(&pw->pop[6][lane + 2].x, r[6] + cr);
      cp_async4(&pw->pop[7][lane + 2].x, r[7] + cr);
    }
  }
  cp_async_commit();
}

// The lane's staged codes after the pull along x, as binary16 words (four per
// population: cells 0-1, 2-3, 4-5, 6-7).  lsel: the byte selector that takes the left
// neighbour's code from its word (its high half; the low half where lane 0's halo word
// starts at an odd row end, column nx - 1 of an odd nx); kend: the position of cell nx - 1
// in the row-end lane's vector (8 elsewhere).  Slots of lanes past the row end hold stale
// codes: only cells past the row end take them, and fused_row_paired zeroes those.
__device__ __forceinline__ void pf_read_h8(const PfWarpH8* pw, int lane, uint32_t lsel, int kend,
                                           uint4 (&w)[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) w[q] = pw->pop[q][lane + 1];
  // cx = +1 (q = 1, 5, 8): codes [left, c0 .. c6]
#pragma unroll
  for (int q : {1, 5, 8}) {
    const uint32_t left = pw->pop[q][lane].w;
    const uint4 v = w[q];
    w[q] = make_uint4(__byte_perm(left, v.x, lsel), __byte_perm(v.x, v.y, 0x5432),
                      __byte_perm(v.y, v.z, 0x5432), __byte_perm(v.z, v.w, 0x5432));
  }
  // cx = -1 (q = 3, 6, 7): codes [c1 .. c7, right]; cell nx - 1 takes column 0
#pragma unroll
  for (int q : {3, 6, 7}) {
    const uint32_t right = pw->pop[q][lane + 2].x;
    const uint4 v = w[q];
    w[q] = make_uint4(__byte_perm(v.x, v.y, 0x5432), __byte_perm(v.y, v.z, 0x5432),
                      __byte_perm(v.z, v.w, 0x5432), __byte_perm(v.w, right, 0x5432));
    if (kend < 7) {  // a row end inside the vector (the row-end lane only)
      const uint32_t c = right & 0xffffu;
      auto patch = [&](uint32_t& wd, int t) {
        if (kend == 2 * t) wd = (wd & 0xffff0000u) | c;
        if (kend == 2 * t + 1) wd = (wd & 0x0000ffffu) | (c << 16);
      };
      patch(w[q].x, 0);
      patch(w[q].y, 1);
      patch(w[q].z, 2);
      patch(w[q].w, 3);
    }
  }
}

// Decode the codes of one group of four cells (words lo and hi of each population).
__device__ __forceinline__ void decode_h8(const StepParams<__half>& p, const uint4 (&w)[9],
                                          bool upper, F2 (&f)[9][2]) {
  const PairCodec<__half> c0(p.codec, 0), c1(p.codec, 1), c5(p.codec, 5);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const PairCodec<__half>& c = q == 0 ? c0 : (q <= 4 ? c1 : c5);
    const uint32_t lo = upper ? w[q].z : w[q].x, hi = upper ? w[q].w : w[q].y;
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
    f[q][0] = fma2(pack2(a.x, a.y), c.inv, c.base);
    f[q][1] = fma2(pack2(b.x, b.y), c.inv, c.base);
  }
}

// Dynamic shared memory of step_kernel<S, MODE, ..., PF, VC, NW>: the FP16 row prefetch
// slots of the one-step {Kn, KL, neq} kernel (VC cells per lane, NW warps), or 0.
// FP32 one-step {Kn, KL, neq} launches with the row prefetch of the multi-step kernel
// (KSS_F32_ONESTEP_PREFETCH; measured at two CTAs per SM with the paired row: 4096^2
// 0.2165 vs 0.2248 ms per launch, 8192^2 0.7891 vs 0.8188 ms; 0 loads every row directly).
#ifndef KSS_F32_ONESTEP_PREFETCH
#define KSS_F32_ONESTEP_PREFETCH 1
#endif
template <class S, int MODE, bool PF, int VC = Vec<S>::N, int NW = kWarps>
__host__ __device__ constexpr int step_prefetch_smem() {
  return (PF && std::is_same<S, __half>::value && MODE == MODE_STD)
             ? (VC == 8 ? NW * int(sizeof(PfWarpH8)) : kPfBytesH)
         : (PF && KSS_F32_ONESTEP_PREFETCH && std::is_same<S, float>::value && MODE == MODE_STD)
             ? kPfBytes
             : 0;
}

// The populations of row j's V-cell vectors at column i0 after the pull (loads of the nine
// source rows, the halo values of the cx != 0 planes, the shifts along x): the direct-load
// path of step_block, and one row of a plain step on its own (the adjoint's recomputation).
template <class S, bool CG>
__device__ __forceinline__ void pull_row(const StepParams<S>& p, int j, int i0, int lane,
                                         bool cv, arith_t<S> (&ft)[9][Vec<S>::N]) {
  using T = arith_t<S>;
  constexpr int V = Vec<S>::N;
  const S* base = p.src + (long long)j * p.pitch;
  long long up, dn;  // rows j - 1 and j + 1
  row_neighbours(p, j, up, dn);
  // source rows of q = 0..8 (pull: row j - cy_q)
  const S* r0 = base;
  const S* r1 = base + 1 * p.plane;
  const S* r2 = base + 2 * p.plane + up;
  const S* r3 = base + 3 * p.plane;
  const S* r4 = base + 4 * p.plane + dn;
  const S* r5 = base + 5 * p.plane + up;
  const S* r6 = base + 6 * p.plane + up;
  const S* r7 = base + 7 * p.plane + dn;
  const S* r8 = base + 8 * p.plane + dn;
  pop_vload<S, V, CG>(r0 + i0, cv, ft[0], 0, p.codec);
  pop_vload<S, V, CG>(r1 + i0, cv, ft[1], 1, p.codec);
  pop_vload<S, V, CG>(r2 + i0, cv, ft[2], 2, p.codec);
  pop_vload<S, V, CG>(r3 + i0, cv, ft[3], 3, p.codec);
  pop_vload<S, V, CG>(r4 + i0, cv, ft[4], 4, p.codec);
  pop_vload<S, V, CG>(r5 + i0, cv, ft[5], 5, p.codec);
  pop_vload<S, V, CG>(r6 + i0, cv, ft[6], 6, p.codec);
  pop_vload<S, V, CG>(r7 + i0, cv, ft[7], 7, p.codec);
  pop_vload<S, V, CG>(r8 + i0, cv, ft[8], 8, p.codec);
  const T h1 = decode<S>(load_left_halo<S, CG>(r1, i0, p.nx, lane, cv), 1, p.codec);
  const T h5 = decode<S>(load_left_halo<S, CG>(r5, i0, p.nx, lane, cv), 5, p.codec);
  const T h8 = decode<S>(load_left_halo<S, CG>(r8, i0, p.nx, lane, cv), 8, p.codec);
  const T h3 = decode<S>(load_right_halo<S, V, CG>(r3, i0, p.nx, lane, cv), 3, p.codec);
  const T h6 = decode<S>(load_right_halo<S, V, CG>(r6, i0, p.nx, lane, cv), 6, p.codec);
  const T h7 = decode<S>(load_right_halo<S, V, CG>(r7, i0, p.nx, lane, cv), 7, p.codec);
  assemble_from_left<T>(ft[1], h1, lane);
  assemble_from_left<T>(ft[5], h5, lane);
  assemble_from_left<T>(ft[8], h8, lane);
  assemble_from_right<T>(ft[3], h3, i0, p.nx, lane);
  assemble_from_right<T>(ft[6], h6, i0, p.nx, lane);
  assemble_from_right<T>(ft[7], h7, i0, p.nx, lane);
}

// ---------------------------------------------------------------- the fused step ----
// MODE:  MODE_PLAIN (stream + collide only), MODE_STD / MODE_FULL (plus sensors,
//        flags, tile counts, sums).
// PULL:  stream before evaluating (false: evaluate the stored state as it is).
// STORE: collide and write the new populations (false: evaluation only).
// Block (bx, by) of a lattice whose step grid is gx blocks wide: its rows, then (output
// modes) its tile counts and its partial sums and counts in slot bid.  Called by every
// thread of the CTA; the CTA's shared memory is free again when it returns.  VC: cells per
// lane (the storage's vector width, or 8 for the FP16 {Kn, KL, neq} step with the row
// prefetch, whose CTA rows are 256 columns).  NW: warps per CTA (8; the eight-cell kernel
// may take fewer, at most 8 rows per warp).
template <class S, int MODE, bool PULL, bool STORE, bool CG = false, bool AAR = false,
          bool PREFETCH = false, int VC = Vec<S>::N, int NW = kWarps>
__device__ __forceinline__ void step_block(const StepParams<S>& p, const int bx, const int by,
                                           const int gx, double* part_sum, uint32_t* part_cnt) {
  using T = arith_t<S>;
  constexpr int V = Vec<S>::N;
  constexpr bool OUT = MODE != MODE_PLAIN;
  constexpr int NT = 32 * NW;  // threads of the CTA
  // eight cells per lane: two groups of four on the paired FP16 row, staged by pf_issue_h8
  constexpr bool kH8 = VC == 8;
  static_assert(VC == V || (kH8 && std::is_same<S, __half>::value && MODE == MODE_STD &&
                            PULL && STORE && PREFETCH && !AAR && !CG && KSS_ROW_PAIRED),
                "eight cells per lane: the one-step FP16 {Kn, KL, neq} kernel only");
  static_assert(NW == kWarps || (kH8 && NW >= 1 && NW < kWarps), "warps per CTA");
  const int lane = threadIdx.x & 31, warp = __shfl_sync(kFull, int(threadIdx.x >> 5), 0);
  const int i0 = (bx * 32 + lane) * VC;
  const bool cv = i0 < p.nx;
  const int j0 = by * p.tile * p.bands;
  const int j1 = min(j0 + p.tile * p.bands, p.ny);
  // (uniform over the CTA: every thread returns, before any barrier)
  if (!bounds_ok(bx >= 0 && by >= 0 && bx < gx && bx * 32 * VC < p.pitch && j0 < p.ny &&
                     p.bands >= 1 && p.bands <= kMaxBands && p.tile * p.bands <= 64 &&
                     p.tile * p.bands <= 8 * NW,
                 p.err))
    return;

  __shared__ int s_tiles[2][kMaxBands][32];
  constexpr int kDefer = kH8 ? kWarpDefer8 : kWarpDefer;
  __shared__ uint16_t s_dl[NW][kDefer];  // each warp's deferred cells
  __shared__ uint32_t s_wn[NW];              // and their number
  __shared__ uint32_t s_cx[3];                   // their tags (refine, switch, nonpos)
  __shared__ Red<T> s_sum[NW][3];
  __shared__ uint32_t s_cnt[NW][3];
  if (OUT) {
    for (int t = threadIdx.x; t < 2 * kMaxBands * 32; t += NT) (&s_tiles[0][0][0])[t] = 0;
    if (threadIdx.x < 3) s_cx[threadIdx.x] = 0;
    __syncthreads();
  }

  Acc<T> a_rho, a_jx, a_jy;
  uint32_t n_ref = 0, n_sw = 0, n_np = 0;
  uint32_t wn = 0;  // deferred cells gathered by this warp (warp-uniform)
  // tile = 2^tshift rows and columns, covered by lpt = 2^lshift lanes of V cells
  const int tshift = __ffs(p.tile) - 1;
  const int lshift = tshift - (VC == 8 ? 3 : VC == 4 ? 2 : (VC == 2 ? 1 : 0));
  const int lpt = 1 << lshift;

  // row prefetch (see PfWarp): the warp's slots in dynamic shared memory, and the copies
  // of row jj into them
  constexpr bool PF = PREFETCH && PULL && STORE && std::is_same<S, float>::value;
  extern __shared__ __align__(16) unsigned char kss_dyn_smem[];
  PfWarp* const pw = reinterpret_cast<PfWarp*>(kss_dyn_smem) + warp;
  auto pf_issue = [&](int jj) {
    if (cv) {
      const S* base = p.src + (long long)jj * p.pitch;
      long long up, dn;  // rows jj - 1 and jj + 1
      row_neighbours(p, jj, up, dn);
      const S* r1 = base + 1 * p.plane;
      const S* r3 = base + 3 * p.plane;
      const S* r5 = base + 5 * p.plane + up;
      const S* r6 = base + 6 * p.plane + up;
      const S* r7 = base + 7 * p.plane + dn;
      const S* r8 = base + 8 * p.plane + dn;
      cp_async16(&pw->pop[0][lane], base + i0);
      cp_async16(&pw->pop[1][lane], r1 + i0);
      cp_async16(&pw->pop[2][lane], base + 2 * p.plane + up + i0);
      cp_async16(&pw->pop[3][lane], r3 + i0);
      cp_async16(&pw->pop[4][lane], base + 4 * p.plane + dn + i0);
      cp_async16(&pw->pop[5][lane], r5 + i0);
      cp_async16(&pw->pop[6][lane], r6 + i0);
      cp_async16(&pw->pop[7][lane], r7 + i0);
      cp_async16(&pw->pop[8][lane], r8 + i0);
      if (lane == 0) {
        const int c = i0 == 0 ? p.nx - 1 : i0 - 1;
        cp_async4(&pw->hl[0], r1 + c);
        cp_async4(&pw->hl[1], r5 + c);
        cp_async4(&pw->hl[2], r8 + c);
      }
      const bool tail = i0 + V >= p.nx;
      if (lane == 31 || tail) {
        const int c = tail ? 0 : i0 + V;
        cp_async4(&pw->hr[0][lane], r3 + c);
        cp_async4(&pw->hr[1][lane], r6 + c);
        cp_async4(&pw->hr[2][lane], r7 + c);
      }
      if (AAR && p.region) cp_async4(&pw->rg[lane], p.region + (long long)jj * p.pitch + i0);
    }
    cp_async_commit();
  };
  if constexpr (PF) {
    if (j0 + warp < j1) pf_issue(j0 + warp);
  }

  // FP16 deviations on the paired row: the pulled codes are assembled as binary16 words
  // (gather_half_row / assemble_half_row) and decoded in pairs; with PREFETCH each warp's
  // next row is staged in shared memory (PfWarpH)
  constexpr bool kHalfPaired = KSS_ROW_PAIRED && std::is_same<S, __half>::value &&
                               MODE != MODE_FULL && !AAR && PULL && V == 4;
  constexpr bool kHalfPF = kHalfPaired && PREFETCH && STORE;
  PfWarpH* const pwh = reinterpret_cast<PfWarpH*>(kss_dyn_smem) + warp;
  if constexpr (kHalfPF && !kH8) {
    if (j0 + warp < j1) pf_issue_half(p, pwh, j0 + warp, i0, lane, cv);
  }
  PfWarpH8* const pw8 = reinterpret_cast<PfWarpH8*>(kss_dyn_smem) + warp;
  const bool tail8 = cv && i0 + 8 >= p.nx;
  const int kend = tail8 ? p.nx - 1 - i0 : 8;  // cell nx - 1 in the row-end lane's vector
  // lane 0's left halo word: column nx - 1 sits in its low half at the seam of an odd nx
  const uint32_t lsel = (i0 == 0 && (p.nx & 1)) ? 0x5410u : 0x5432u;
  if constexpr (kH8) {
    if (j0 + warp < j1) pf_issue_h8(p, pw8, j0 + warp, i0, lane, cv, tail8);
  }
  for (int j = j0 + warp; j < j1; j += NW) {
    uint32_t fbits, fbits2 = 0;  // flag bytes of cells 0-3 and (eight per lane) 4-7
    if constexpr (kH8) {
      uint4 w[9];
      cp_async_wait_all();
      __syncwarp();  // the neighbouring lanes' copies of this row are complete
      pf_read_h8(pw8, lane, lsel, kend, w);
      __syncwarp();  // the row's reads precede the copies of the next row into the slots
      if (j + NW < j1) pf_issue_h8(p, pw8, j + NW, i0, lane, cv, tail8);
      F2 f[9][2];
      decode_h8(p, w, false, f);
      fbits = fused_row_paired<S, MODE, STORE>(p, f, i0, j, cv, a_rho, a_jx, a_jy);
      decode_h8(p, w, true, f);
      fbits2 = fused_row_paired<S, MODE, STORE>(p, f, i0 + 4, j, i0 + 4 < p.nx, a_rho, a_jx,
                                                a_jy);
    } else if constexpr (kHalfPaired) {
      F2 f[9][2];
      uint2 w[9];
      uint32_t h[9];
      if constexpr (kHalfPF) {
        cp_async_wait_all();
        pf_read_half(p, pwh, i0, lane, cv, w, h);
        __syncwarp();  // the row's reads precede the copies of the next row into the slots
        if (j + kWarps < j1) pf_issue_half(p, pwh, j + kWarps, i0, lane, cv);
      } else {
        gather_half_row<CG>(p, j, i0, lane, cv, w, h);
      }
      assemble_half_row(p, i0, lane, w, h, f);
      fbits = fused_row_paired<S, MODE, STORE>(p, f, i0, j, cv, a_rho, a_jx, a_jy);
    } else {
    T ft[9][V];
    const S* base = p.src + (long long)j * p.pitch;
    // AAR: the region in force for this step's collision (the switch flags of the most
    // recent output step before it), loaded ahead of the populations so that its latency
    // overlaps theirs; output steps replace it with their own flags
    uint32_t mbits = 0;
    if constexpr (PF) {
      cp_async_wait_all();
      T hl[3] = {T(0), T(0), T(0)}, hr[3] = {T(0), T(0), T(0)};
      if (cv) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const float4 a = pw->pop[q][lane];
          ft[q][0] = a.x; ft[q][1] = a.y; ft[q][2] = a.z; ft[q][3] = a.w;
        }
        if (lane == 0) {
          hl[0] = pw->hl[0]; hl[1] = pw->hl[1]; hl[2] = pw->hl[2];
        }
        if (lane == 31 || i0 + V >= p.nx) {
          hr[0] = pw->hr[0][lane]; hr[1] = pw->hr[1][lane]; hr[2] = pw->hr[2][lane];
        }
        if (AAR && p.region) mbits = pw->rg[lane];
      } else {
#pragma unroll
        for (int q = 0; q < 9; ++q)
#pragma unroll
          for (int k = 0; k < V; ++k) ft[q][k] = T(0);
      }
      __syncwarp();  // the row's reads precede the copies of the next row into the slots
      if (j + kWarps < j1) pf_issue(j + kWarps);
      assemble_from_left<T>(ft[1], hl[0], lane);
      assemble_from_left<T>(ft[5], hl[1], lane);
      assemble_from_left<T>(ft[8], hl[2], lane);
      assemble_from_right<T>(ft[3], hr[0], i0, p.nx, lane);
      assemble_from_right<T>(ft[6], hr[1], i0, p.nx, lane);
      assemble_from_right<T>(ft[7], hr[2], i0, p.nx, lane);
    } else {
      if constexpr (AAR && STORE) {
        // (in a batch, a member without the model has no region: it steps as BGK)
        if (cv && p.region) mbits = load_bytes<V>(p.region + (long long)j * p.pitch + i0);
      }
      if (PULL) {
        pull_row<S, CG>(p, j, i0, lane, cv, ft);
      } else {
#pragma unroll
        for (int q = 0; q < 9; ++q)
          pop_vload<S, V, CG>(base + q * p.plane + i0, cv, ft[q], q, p.codec);
      }
    }

    fbits = fused_row<S, MODE, PULL, STORE, AAR, CG>(p, ft, i0, j, cv, a_rho, a_jx, a_jy, mbits);
    }
    if (OUT) {
      // (with eight cells per lane, the tags of cells 4-7 moved to bits no tag of cells
      // 0-3 occupies, so one popcount counts both words)
      const uint32_t fr = kH8 ? (fbits & 0x01010101u) | ((fbits2 & 0x01010101u) << 1)
                              : fbits & 0x01010101u;
      const uint32_t fs = kH8 ? (fbits & 0x02020202u) | ((fbits2 & 0x02020202u) >> 1)
                              : fbits & 0x02020202u;
      n_ref += __popc(fr);
      n_sw += __popc(fs);
      n_np += __popc(kH8 ? (fbits & 0x80808080u) | ((fbits2 & 0x80808080u) >> 1)
                         : fbits & 0x80808080u);
    }
    // per-tile tag counts: this lane's cells all lie in tile (lane / lanes_per_tile);
    // tile and lanes per tile are powers of two (tile 8, 16, 32 or 64)
    if (OUT) {
      int tr = __popc(fbits & 0x01010101u) + (kH8 ? __popc(fbits2 & 0x01010101u) : 0);
      int ts = __popc(fbits & 0x02020202u) + (kH8 ? __popc(fbits2 & 0x02020202u) : 0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        if (o < lpt) {
          tr += __shfl_xor_sync(kFull, tr, o);
          ts += __shfl_xor_sync(kFull, ts, o);
        }
      }
      if ((lane & (lpt - 1)) == 0 && (tr | ts)) {
        const int b = (j - j0) >> tshift;
        if (bounds_ok(b < kMaxBands && (lane >> lshift) < 32, p.err)) {
          atomicAdd(&s_tiles[0][b][lane >> lshift], tr);
          atomicAdd(&s_tiles[1][b][lane >> lshift], ts);
        }
      }
      if (MODE == MODE_STD) {
        // gather this row's deferred cells in the warp's region (CTA-local offsets)
        const uint32_t dbits = fbits & 0x40404040u, dbits2 = fbits2 & 0x40404040u;
        if (__any_sync(kFull, (dbits | dbits2) != 0)) {
          const int nd = __popc(dbits) + (kH8 ? __popc(dbits2) : 0);
          int incl = nd;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
          }
          uint32_t slot = wn + uint32_t(incl - nd);
          const int rowoff = (j - j0) * 32 * VC + lane * VC;
#pragma unroll
          for (int k = 0; k < VC; ++k) {
            if (((k < 4 ? dbits : dbits2) >> (8 * (k & 3))) & 0x40u) {
              if (bounds_ok(slot < uint32_t(kDefer), p.err))
                s_dl[warp][slot] = uint16_t(rowoff + k);
              ++slot;
            }
          }
          wn += uint32_t(__shfl_sync(kFull, incl, 31));
        }
      }
    }
  }

  if (!OUT) return;

  // ---- block reduction (fixed order) ----
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
    s_wn[warp] = wn;
  }
  __syncthreads();
  const int bid = by * gx + bx;
  if (MODE == MODE_STD) {
    // the CTA's deferred cells, all threads at once: exact recomputation from the
    // unchanged source populations, then their tags join the CTA's counts
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) total += s_wn[w];
    if (total) {
      const Pick3 pr(p.refine_s), ps(p.switch_s);
      for (uint32_t e = threadIdx.x; e < total; e += NT) {
        uint32_t w = 0, r = e;
        while (r >= s_wn[w]) r -= s_wn[w++];
        const int o = s_dl[w][r];
        const int rl = o / (32 * VC), cl = o - rl * (32 * VC);
        const int j = j0 + rl, i = bx * 32 * VC + cl;
        if (!bounds_ok(j < j1 && i < p.nx && rl / p.tile < kMaxBands && cl / p.tile < 32, p.err))
          continue;
        const uint32_t tags = fix_cell<S, PULL, CG>(p, pr, ps, i, j);
        if (AAR && STORE && p.region) p.region[(long long)j * p.pitch + i] = uint8_t((tags >> 1) & 1u);
        const int b = rl / p.tile, tl = cl / p.tile;
        if (tags & 1u) {
          atomicAdd(&s_cx[0], 1u);
          atomicAdd(&s_tiles[0][b][tl], 1);
        }
        if (tags & 2u) {
          atomicAdd(&s_cx[1], 1u);
          atomicAdd(&s_tiles[1][b][tl], 1);
        }
        if (tags & 4u) atomicAdd(&s_cx[2], 1u);
      }
      __syncthreads();
    }
  }
  const int tpb = (32 * VC) / p.tile;
  for (int t = threadIdx.x; t < tpb * p.bands; t += NT) {
    const int b = t / tpb, tl = t - b * tpb;
    const int tx = bx * tpb + tl, ty = by * p.bands + b;
    if (tx < p.ntx && ty < p.nty) {
      const long long i = (long long)ty * p.ntx + tx;
      p.tiles[i] = s_tiles[0][b][tl];
      p.tiles[(long long)p.ntx * p.nty + i] = s_tiles[1][b][tl];
    }
  }
  if (threadIdx.x == 0) {
    Red<T> s0, s1, s2;
    uint32_t c0 = 0, c1 = 0, c2 = 0;
    if (MODE == MODE_STD) {
      c0 = s_cx[0];
      c1 = s_cx[1];
      c2 = s_cx[2];
    }
    for (int w = 0; w < NW; ++w) {
      s0.add(s_sum[w][0]);
      s1.add(s_sum[w][1]);
      s2.add(s_sum[w][2]);
      c0 += s_cnt[w][0];
      c1 += s_cnt[w][1];
      c2 += s_cnt[w][2];
    }
    s0.store(part_sum + 3 * bid + 0);
    s1.store(part_sum + 3 * bid + 1);
    s2.store(part_sum + 3 * bid + 2);
    part_cnt[4 * bid + 0] = c0;
    part_cnt[4 * bid + 1] = c1;
    part_cnt[4 * bid + 2] = c2;
  }
}

// After a CTA's last block: one ticket from the completion counter per CTA (nunits CTAs
// in all); the CTA that takes the last one adds the nblocks per-block partials in block
// order.  Called by every thread of the CTA.
template <class S, int NTHREADS = kThreads>
__device__ __forceinline__ void ticket_and_finalize(const StepParams<S>& p, int nunits,
                                                    int nblocks) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {  // thread 0 wrote this CTA's partials

    __threadfence();
    const uint32_t ticket = atomicAdd(p.done, 1u);
    s_last = (ticket == uint32_t(nunits - 1));
  }
  __syncthreads();
  if (!s_last) return;
  // ---- last CTA: add the per-block partials ----
  __threadfence();
  finalize_partials<S, NTHREADS>(p, nblocks);
}

// One CTA per block (bx, by) of a grid gx blocks wide, nblocks in all.  PF: the FP16 row
// prefetch (the launch then gives the kernel step_prefetch_smem bytes of dynamic shared
// memory).
template <class S, int MODE, bool PULL, bool STORE, bool AAR = false, bool PF = false,
          int VC = Vec<S>::N, int NW = kWarps>
__device__ __forceinline__ void step_cta(const StepParams<S>& p, const int bx, const int by,
                                         const int gx, const int nblocks) {
  step_block<S, MODE, PULL, STORE, false, AAR, PF, VC, NW>(p, bx, by, gx, p.part_sum,
                                                          p.part_cnt);
  if (MODE != MODE_PLAIN) ticket_and_finalize<S, 32 * NW>(p, nblocks, nblocks);
}

// AAR: the step with the two-relaxation collision in the region p.region (pull + store).

template <class S, int MODE, bool PULL, bool STORE, bool AAR = false, bool PF = false,
          int VC = Vec<S>::N, int NW = kWarps>
__global__ void __launch_bounds__(32 * NW, VC == 8 ? KSS_H8_MIN_BLOCKS
                                                   : step_min_blocks<S, MODE>())
step_kernel(const StepParams<S> p) {
  step_cta<S, MODE, PULL, STORE, AAR, PF, VC, NW>(p, blockIdx.x, blockIdx.y, gridDim.x,
                                                  gridDim.x * gridDim.y);
}

// The same step with a persistent grid: CTA c takes blocks c, c + gridDim.x, ... of the
// gx-wide step grid (nblocks in all) in a fixed assignment, so that no CTA is launched or
// retired between blocks and the completion counter is taken once per CTA.  Each block's
// partials keep their slot, so the sums are those of step_kernel bit for bit.
template <class S, int MODE, bool PULL, bool STORE>
__global__ void __launch_bounds__(kThreads, step_min_blocks<S, MODE>())
step_kernel_persistent(const StepParams<S> p, int gx, int nblocks) {
  for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int by = b / gx;
    step_block<S, MODE, PULL, STORE>(p, b - by * gx, by, gx, p.part_sum, p.part_cnt);
    if (MODE != MODE_PLAIN) __syncthreads();  // shared memory is reused by the next block
  }
  if (MODE != MODE_PLAIN) ticket_and_finalize<S>(p, gridDim.x, nblocks);
}

// ---------------------------------------------------------------- multi-step ----
// nsteps steps in one cooperative launch (every CTA resident).  The (step, block) work
// items are handed out in order from an atomic counter (as the hardware hands out the
// blocks of a launch); block b of step s first waits until the blocks of its 3 x 3
// neighbourhood (periodic) have completed step s - 1: they wrote the halo it reads and
// have read the cells it overwrites.  So a step starts where the previous one has
// finished, with no launch boundary between them, and every item it waits for was
// handed out earlier (no cycle).  Each block's partial sums of step s go to ring slot
// s % ring; the block that completes step s last adds them in block order (the step's
// sums; the last step's are the lattice's), and a slot is reused only after its previous
// step's sums were formed.  Every wait is bounded by a clock64 deadline, after which the
// CTA sets bit 1 of the error word and returns (its neighbours then run out too).
// Population loads are ordinary cached loads after an acquire (CG).
struct MultiState {
  uint32_t* done;      // [nblocks] steps each block has completed (0 at launch)
  uint32_t* ticket;    // [ring] blocks of the slot's step completed (0 when free)
  uint32_t* fin;       // [ring] 1 + the last step whose sums the slot formed (0 at launch)
  uint32_t* work;      // next work item (0 at launch)
  double* part_sum;    // [ring][nblocks][3]
  uint32_t* part_cnt;  // [ring][nblocks][4]
  double* ring_sums;   // [ring][3] each step's sums
  unsigned long long* ring_counts;  // [ring][3]
  uint32_t* err;       // bit 1: a wait ran out
  long long deadline;  // clock64 cycles one wait may take
  int ring, nsteps, gx, gy, nblocks;
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread: wait until *p >= want, at most m.deadline cycles.
__device__ __forceinline__ bool wait_at_least(const MultiState& m, const uint32_t* p,
                                              uint32_t want) {
  if (ld_acquire_u32(p) >= want) return true;
  const long long t0 = clock64();
  while (ld_acquire_u32(p) < want) {
    if (clock64() - t0 > m.deadline) {
      atomicOr(m.err, 2u);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Work item (step s, block b); returns false if a wait ran out.  s_next receives the
// CTA's next work item (taken early, so that the counter's latency is hidden).
template <class S, int MODE, bool AAR = false, bool PREFETCH = false>
__device__ __forceinline__ bool multi_block(const StepParams<S>& p, const MultiState& m, int s,
                                            int b, int* s_next) {
  constexpr bool OUT = MODE != MODE_PLAIN;
  __shared__ int s_go, s_fin;
  const int slot = s % m.ring;
  double* psum = m.part_sum + (long long)slot * m.nblocks * 3;
  uint32_t* pcnt = m.part_cnt + (long long)slot * m.nblocks * 4;
  const int by = b / m.gx, bx = b - by * m.gx;
  // warp 0: lanes 0..8 wait for the 3 x 3 neighbours, lane 9 for the ring slot, all at
  // once (one round trip to L2 instead of ten in a row); each lane's acquire is ordered
  // before the CTA's loads by the barrier below
  if (threadIdx.x < 32) {
    const int t = threadIdx.x;
    if (t == 0) *s_next = int(atomicAdd(m.work, 1u));
    bool ok = true;
    if (s > 0 && t < 9) {
      const int dy = t / 3 - 1, dx = t - 3 * (t / 3) - 1;
      const int yy = by + dy < 0 ? m.gy - 1 : (by + dy == m.gy ? 0 : by + dy);
      const int xx = bx + dx < 0 ? m.gx - 1 : (bx + dx == m.gx ? 0 : bx + dx);
      ok = wait_at_least(m, m.done + yy * m.gx + xx, uint32_t(s));
    }
    // the slot's previous step (s - ring) must have its sums formed
    if (OUT && t == 9 && s >= m.ring) ok = wait_at_least(m, m.fin + slot, uint32_t(s - m.ring + 1));
    ok = __all_sync(kFull, ok);
    if (t == 0) s_go = ok;
  }
  __syncthreads();
  if (!s_go) return false;
  // (AAR: block b's region bytes of step s - 1 were written before its release, which
  // the wait on block b itself -- part of its 3 x 3 neighbourhood -- acquired)
  step_block<S, MODE, true, true, true, AAR, PREFETCH>(p, bx, by, m.gx, psum, pcnt);
  __syncthreads();  // every store of the block precedes thread 0's release
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_u32(m.done + b, uint32_t(s + 1));
    s_fin = OUT && atomicAdd(m.ticket + slot, 1u) == uint32_t(m.nblocks - 1);
  }
  __syncthreads();
  if (OUT && s_fin) {
    __threadfence();
    const bool last = s == m.nsteps - 1;
    finalize_sums<S, kThreads>(psum, pcnt, m.nblocks, last ? p.stat_sums : m.ring_sums + 3 * slot,
                               last ? p.stat_counts : m.ring_counts + 3 * slot);
    __syncthreads();
    if (threadIdx.x == 0) {
      m.ticket[slot] = 0u;
      __threadfence();
      st_release_u32(m.fin + slot, uint32_t(s + 1));
    }
  }
  return true;
}

// pa: buffer A -> B (even steps); pb: B -> A (odd steps).  AAR: the two-relaxation
// collision in the region (adaptive algorithm refinement), two CTAs per SM (its per-cell
// state needs more than 80 registers).
template <class S, int MODE, bool AAR = false>
__global__ void __launch_bounds__(kThreads, AAR ? 2 : step_min_blocks<S, MODE>())
step_kernel_multi(const StepParams<S> pa, const StepParams<S> pb, const MultiState m) {
  __shared__ int s_next;
  if (threadIdx.x == 0) s_next = int(atomicAdd(m.work, 1u));
  __syncthreads();
  int w = s_next;
  const int total = m.nsteps * m.nblocks;
  while (w < total) {
    const int s = w / m.nblocks, b = w - s * m.nblocks;
    __syncthreads();  // every thread has read s_next before thread 0 rewrites it
    constexpr bool pf = multi_prefetch_smem<S, MODE, AAR>() > 0;
    const bool ok = (s & 1) ? multi_block<S, MODE, AAR, pf>(pb, m, s, b, &s_next)
                            : multi_block<S, MODE, AAR, pf>(pa, m, s, b, &s_next);
    if (!ok) return;
    __syncthreads();
    w = s_next;
  }
}

// ---------------------------------------------------------------- batched step ----
// One step of many independent lattices of any sizes in one launch.  The lattices'
// step grids are laid end to end in a work list of CTA blocks; CTA b takes work items
// b, b + gridDim.x, ... (one item each when the grid covers the list, persistent CTAs
// otherwise).  Each item is exactly step_kernel's CTA for that block of that lattice,
// with the lattice's parameters copied to shared memory, so every lattice's results
// are those of its own step_kernel launch with the same CTA height.  Each lattice keeps
// its own completion counter and partial sums: the CTA that finishes a lattice's last
// block forms that lattice's sums.
struct BatchItem {
  uint32_t lat;     // lattice index into the parameter table
  uint32_t bx, by;  // CTA block of that lattice's step grid
  uint32_t pad;
};

// MODE: MODE_PLAIN (no outputs), MODE_STD (every lattice with {Kn, KL, neq}) or
// MODE_FULL (each lattice with its own set: p.mode, MODE_STD or MODE_FULL).
// AAR: members with a region take the two-relaxation collision there (members without
// one step as BGK).
template <class S, int MODE, bool AAR = false>
__global__ void __launch_bounds__(kThreads, step_min_blocks<S, MODE>())
batch_step_kernel(const StepParams<S>* __restrict__ table, const BatchItem* __restrict__ items,
                  int nitems) {
  static_assert(sizeof(StepParams<S>) % 8 == 0, "parameter copy in 8-byte words");
  __shared__ __align__(16) unsigned long long s_raw[sizeof(StepParams<S>) / 8];
  const StepParams<S>& sp = *reinterpret_cast<const StepParams<S>*>(s_raw);
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const BatchItem it = items[w];
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(table + it.lat);
    for (int k = threadIdx.x; k < int(sizeof(StepParams<S>) / 8); k += kThreads) s_raw[k] = src[k];
    __syncthreads();
    if (MODE != MODE_FULL || sp.mode != MODE_FULL)
      step_cta<S, MODE == MODE_FULL ? MODE_STD : MODE, true, true, AAR>(
          sp, int(it.bx), int(it.by), sp.grid_x, sp.nblocks);
    else
      step_cta<S, MODE_FULL, true, true, AAR>(sp, int(it.bx), int(it.by), sp.grid_x,
                                              sp.nblocks);
    __syncthreads();  // the CTA's shared memory is reused by the next item
  }
}

// ---------------------------------------------------------------- batched multi-step ----
// nsteps steps of a whole batch in one cooperative launch (FP32 storage: rows staged by
// the row prefetch, two CTAs per SM at up to 128 registers; other storage types load their
// rows directly at the register budget of the one-step kernels): work item w = s * nitems + i is
// block items[i] of step s.  Each lattice has its own MultiState (its blocks' step
// counters, ring of partial sums, ticket and slot counters); all share the work counter,
// so items are handed out in (step, work-list) order and, as in step_kernel_multi, every
// item waits only for items of its own lattice handed out before it.  mtab[k] is lattice
// k's state; ta / tb its parameters for even / odd steps.
template <class S, int MODE>
__global__ void __launch_bounds__(kThreads,
                                  multi_prefetch_smem<S, MODE, false>() > 0 ? 2
                                                                            : step_min_blocks<S, MODE>())
batch_kernel_multi(const StepParams<S>* __restrict__ ta, const StepParams<S>* __restrict__ tb,
                   const MultiState* __restrict__ mtab, const BatchItem* __restrict__ items,
                   int nitems, int nsteps, uint32_t* work) {
  static_assert(sizeof(StepParams<S>) % 8 == 0 && sizeof(MultiState) % 8 == 0,
                "parameter copies in 8-byte words");
  __shared__ __align__(16) unsigned long long s_p[sizeof(StepParams<S>) / 8];
  __shared__ __align__(16) unsigned long long s_m[sizeof(MultiState) / 8];
  __shared__ int s_next;
  const StepParams<S>& sp = *reinterpret_cast<const StepParams<S>*>(s_p);
  const MultiState& sm = *reinterpret_cast<const MultiState*>(s_m);
  if (threadIdx.x == 0) s_next = int(atomicAdd(work, 1u));
  __syncthreads();
  int w = s_next;
  const int total = nsteps * nitems;
  while (w < total) {
    const int s = w / nitems;
    const BatchItem it = items[w - s * nitems];
    __syncthreads();  // every thread has read s_next and is done with the shared copies
    const unsigned long long* src =
        reinterpret_cast<const unsigned long long*>(((s & 1) ? tb : ta) + it.lat);
    for (int k = threadIdx.x; k < int(sizeof(StepParams<S>) / 8); k += kThreads) s_p[k] = src[k];
    const unsigned long long* msrc = reinterpret_cast<const unsigned long long*>(mtab + it.lat);
    for (int k = threadIdx.x; k < int(sizeof(MultiState) / 8); k += kThreads) s_m[k] = msrc[k];
    __syncthreads();
    // the table is shared by calls of any length: the launch's step count goes in here
    // (other threads read it only after multi_block's barriers)
    if (threadIdx.x == 0) reinterpret_cast<MultiState*>(s_m)->nsteps = nsteps;
    if (!multi_block<S, MODE, false, (multi_prefetch_smem<S, MODE, false>() > 0)>(
            sp, sm, s, int(it.by) * sm.gx + int(it.bx), &s_next))
      return;
    __syncthreads();
    w = s_next;
  }
}

// ---------------------------------------------------------------- fixup ----
// Add tags (bit 0 refine, bit 1 switch) of the active lanes' cells to their tiles, one
// atomic per distinct tile per warp (list entries of a warp mostly share tiles).
__device__ __forceinline__ void add_tile_tags(int32_t* tiles, long long ntiles, long long t,
                                              uint32_t tags, unsigned active) {
  const unsigned same = __match_any_sync(active, t);
  const int r = __popc(__ballot_sync(active, tags & 1u) & same);
  const int s = __popc(__ballot_sync(active, tags & 2u) & same);
  if ((threadIdx.x & 31) == __ffs(same) - 1) {
    if (r) atomicAdd(tiles + t, r);
    if (s) atomicAdd(tiles + ntiles + t, s);
  }
}

// The cells the fused pass deferred (flag byte KSS_FLAG_DEFERRED), from its compact
// list: one thread per cell.  If the list overflowed, a grid-stride scan over groups of
// 4 cells of a row finds them instead (skipping tiles with none).  Counts are corrected
// with integer atomics, so they stay exact and reproducible; the last CTA resets the
// list for the next pass.
template <class S, bool PULL>
__global__ void __launch_bounds__(256) fixup_kernel(const StepParams<S> p) {
  const int lane = threadIdx.x & 31;
  const Pick3 pr(p.refine_s), ps(p.switch_s);
  unsigned long long cr = 0, cs = 0, cn = 0;
  const uint32_t count = __ldcg(p.defer_count);
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  if (count <= p.defer_cap) {
    const long long ntiles = (long long)p.ntx * p.nty;
    for (long long e0 = tid - lane; e0 < count; e0 += nthreads) {  // warp-uniform trips
      const long long e = e0 + lane;
      const bool has = e < count;
      const unsigned active = __ballot_sync(kFull, has);
      if (!has) continue;
      const uint32_t cell = __ldcg(p.defer_list + e);
      const int j = int(cell / uint32_t(p.nx)), i = int(cell - uint32_t(j) * uint32_t(p.nx));
      const uint32_t tags = fix_cell<S, PULL>(p, pr, ps, i, j);
      add_tile_tags(p.tiles, ntiles, (long long)(j / p.tile) * p.ntx + i / p.tile, tags, active);
      cr += tags & 1u;
      cs += (tags >> 1) & 1u;
      cn += (tags >> 2) & 1u;
    }
  } else {
    const int qpr = (p.nx + 3) / 4;  // groups per row (tile is a multiple of 4)
    const long long ngroups = (long long)qpr * p.ny;
    for (long long g = tid; g < ngroups; g += nthreads) {
      const int j = int(g / qpr), i0 = int(g - (long long)j * qpr) * 4;
      const long long t = (long long)(j / p.tile) * p.ntx + i0 / p.tile;
      if (__ldcg(p.tiles_def + t) == 0) continue;
      const uint32_t w = __ldcg(reinterpret_cast<const uint32_t*>(p.flags + (long long)j * p.pitch + i0));
      if (!(w & 0x40404040u)) continue;
      for (int k = 0; k < 4; ++k) {
        if (i0 + k >= p.nx || !((w >> (8 * k)) & kFlagDeferred)) continue;
        const uint32_t tags = fix_cell<S, PULL>(p, pr, ps, i0 + k, j);
        if (tags & 1u) atomicAdd(p.tiles + t, 1);
        if (tags & 2u) atomicAdd(p.tiles + (long long)p.ntx * p.nty + t, 1);
        cr += tags & 1u;
        cs += (tags >> 1) & 1u;
        cn += (tags >> 2) & 1u;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cr += __shfl_xor_sync(kFull, cr, o);
    cs += __shfl_xor_sync(kFull, cs, o);
    cn += __shfl_xor_sync(kFull, cn, o);
  }
  if (lane == 0) {
    if (cr) atomicAdd(p.stat_counts + 0, cr);
    if (cs) atomicAdd(p.stat_counts + 1, cs);
    if (cn) atomicAdd(p.stat_counts + 2, cn);
  }
  // the last CTA to finish resets the list for the next pass (no CTA waits)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(p.defer_ticket, 1u) == gridDim.x - 1) {
      *p.defer_count = 0u;
      *p.defer_ticket = 0u;
    }
  }
}

// ---------------------------------------------------------------- helpers ----
// f := f^eq(rho, u), computed in double and rounded once to T.
// The auxiliary kernels below run on a grid of (column blocks of 256) x (rows), rows
// strided by gridDim.y: one row per CTA row, so no 64-bit division per element.

// f := f^eq(rho, u) from dense FP64 (In = double) or FP32 (In = float) fields, evaluated in
// the arithmetic type (the FP64 pipe is a small fraction of the FP32 one on this GPU, and
// an FP32 lattice keeps only FP32 populations) and stored in S.  An FP32 field value gives
// the populations of the same value passed as FP64.
template <class S, class In>
__global__ void init_equilibrium_kernel(const In* __restrict__ rho,
                                        const In* __restrict__ ux,
                                        const In* __restrict__ uy, S* __restrict__ f,
                                        long long plane, int pitch, int nx, int ny,
                                        const codec_t<S> codec) {
  using T = arith_t<S>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  for (int j = blockIdx.y; j < ny; j += gridDim.y) {
    const long long c = (long long)j * nx + i;
    T feq[9];
    equilibrium<T>(T(rho[c]), T(ux[c]), T(uy[c]), feq);
    S* o = f + (long long)j * pitch + i;
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q * plane] = encode<S>(feq[q], q, codec);
  }
}

// rho, ux, uy (double, dense) of a stored state.
template <class S>
__global__ void moments_kernel(const S* __restrict__ f, long long plane, int pitch, int nx,
                               int ny, double* __restrict__ rho, double* __restrict__ ux,
                               double* __restrict__ uy, const codec_t<S> codec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  for (int j = blockIdx.y; j < ny; j += gridDim.y) {
    const long long c = (long long)j * nx + i;
    const S* in = f + (long long)j * pitch + i;
    double v[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] = double(decode<S>(in[q * plane], q, codec));
    const double r = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
    const double jx = (v[1] + v[5] + v[8]) - (v[3] + v[6] + v[7]);
    const double jy = (v[2] + v[5] + v[6]) - (v[4] + v[7] + v[8]);
    rho[c] = r;
    ux[c] = jx / r;
    uy[c] = jy / r;
  }
}

// The nine population planes (decoded) <-> dense double planes [9][ny][nx].
template <class S>
__global__ void pops_to_dense_kernel(const S* __restrict__ src, long long plane, int pitch,
                                     int nx, int ny, double* __restrict__ dst,
                                     const codec_t<S> codec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
#pragma unroll
  for (int q = 0; q < 9; ++q)
    for (int j = blockIdx.y; j < ny; j += gridDim.y)
      dst[((long long)q * ny + j) * nx + i] =
          double(decode<S>(src[q * plane + (long long)j * pitch + i], q, codec));
}

template <class S>
__global__ void dense_to_pops_kernel(const double* __restrict__ src, long long plane,
                                     int pitch, int nx, int ny, S* __restrict__ dst,
                                     const codec_t<S> codec) {
  using T = arith_t<S>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
#pragma unroll
  for (int q = 0; q < 9; ++q)
    for (int j = blockIdx.y; j < ny; j += gridDim.y)
      dst[q * plane + (long long)j * pitch + i] =
          encode<S>(T(src[((long long)q * ny + j) * nx + i]), q, codec);
}

// nplanes pitched T planes <-> dense double planes (sensor fields, weights).
template <class T>
__global__ void pitched_to_dense_kernel(const T* __restrict__ src, long long plane, int pitch,
                                        int nx, int ny, int nplanes, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  for (int q = 0; q < nplanes; ++q)
    for (int j = blockIdx.y; j < ny; j += gridDim.y)
      dst[((long long)q * ny + j) * nx + i] = double(src[q * plane + (long long)j * pitch + i]);
}

template <class T>
__global__ void dense_to_pitched_kernel(const double* __restrict__ src, long long plane,
                                        int pitch, int nx, int ny, int nplanes,
                                        T* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  for (int q = 0; q < nplanes; ++q)
    for (int j = blockIdx.y; j < ny; j += gridDim.y)
      dst[q * plane + (long long)j * pitch + i] = T(src[((long long)q * ny + j) * nx + i]);
}

}  // namespace kss
