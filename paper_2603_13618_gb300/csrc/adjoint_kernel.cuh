// adjoint_kernel.cuh -- discrete adjoint (reverse mode) of the fused step for the
// sensor objective
//   J = sum_x W(x) eps_KL(x)   (Eq. HKL-sensor on the pre-collision populations of
//                               step N, weights W, default 1)
// with respect to the initial density rho0 (initial populations f^eq(rho0, u0), u0
// fixed) and to the relaxation time tau.
//
// Forward map: f^0 = f^eq(rho0, u0), f^{n+1} = C(S f^n) with S the pull streaming and
// C the BGK collision, J = sum W KL(S f^{N-1}).  With ft^n = S f^n the reverse sweep is
//   lt^{N-1} = W dKL/dft (ft^{N-1})                            adj_objective_kernel
//   l^{n+1} = S^T lt^{n+1},   lt^n = (dC/dft (ft^n))^T l^{n+1},
//   dJ/dtau += sum_x l^{n+1} . (ft^n - f^eq(ft^n)) / tau^2      adj_step_kernel
//   dJ/drho0 = sum_q (S^T lt^0)_q f^eq_q(1, u0)                 adj_final_kernel
// where S^T is the pull in the opposite direction, (S^T l)_q(x) = l_q(x + c_q).
//
// Per cell, with rho = sum f, j = sum c f = rho u, D_q = d f^eq_q / d rho and
// E_q = d f^eq_q / d j of the N = 2 Grad-Hermite equilibrium:
//   D_q = w_q (1 + 3/2 u.u - 9/2 (c_q.u)^2),   E_q = w_q ((3 + 9 c_q.u) c_q - 3 u),
// so d f^eq_q / d f_p = D_q + c_p . E_q, and
//   collision:  lt_p = (1 - omega) l_p + omega (A + c_p . B),
//               A = sum_q l_q D_q,  B = sum_q l_q E_q;
//   KL:         K = sum f ln(f / f^eq) = sum f^eq phi(x), x_q = (f_q - f^eq_q) / f^eq_q,
//               dK/df_p = ln(1 + x_p) - (a + c_p . b),  a = sum x_q D_q,  b = sum x_q E_q,
//               and eps_KL = |K| (gradient times sign K).
// The last form is the derivative of sum f ln(f / f^eq) after the exact cancellations
// sum_q D_q = 1 and sum_q E_q = 0, so no O(1) terms cancel in floating point.
//
// Layout and work decomposition as the fused step (pitched SoA planes), with 2 cells
// per thread: a CTA of 8 warps covers 64 columns x p.rows rows (8, 16 or 32: small lattices
// take short CTAs so that the grid fills the GPU).
#pragma once

#include "step_kernel.cuh"

namespace kss {

constexpr int kAdjV = 2;      // cells per thread
constexpr int kAdjRows = 32;  // largest rows per CTA (4 per warp)

template <class T>
struct AdjParams {
  const T* f;            // post-collision state f^n, pulled to ft^n
  const T* lam_in;       // lt^{n+1} (adjoint of ft^{n+1}), pulled in reverse to l^{n+1}
  T* lam_out;            // lt^n
  const T* weight;       // W [ny][pitch], or nullptr for W = 1 (objective kernel)
  const double* ux0;     // u0, dense [ny][nx] (final kernel)
  const double* uy0;
  double* grad;          // dJ/drho0, dense [ny][nx] (final kernel)
  double* part;          // per-CTA partial sums [nblocks]
  uint32_t* done;        // CTA completion counter, 0 between launches
  double* acc;           // the launch's total is added to *acc (FP64)
  long long plane;
  int pitch, nx, ny;
  int rows;              // rows per CTA (grid adj_grid(nx, ny, rows))
  T omega;
};

// Nine populations of V cells of row j pulled from src: forward (REV = false)
// v_q(i, j) = src_q(i - cx_q, j - cy_q); reverse v_q(i, j) = src_q(i + cx_q, j + cy_q).
template <class T, bool REV, bool CG = false>
__device__ __forceinline__ void adj_pull_row(const T* src, long long plane, int pitch, int nx,
                                             int ny, int j, int i0, int lane, bool cv,
                                             T (&v)[9][kAdjV]) {
  constexpr int V = kAdjV;
  const T* base = src + (long long)j * pitch;
  const long long up = (long long)((j == 0 ? ny : j) - 1 - j) * pitch;    // row j-1
  const long long dn = (long long)((j + 1 == ny ? 0 : j + 1) - j) * pitch;  // row j+1
  const long long rp = REV ? dn : up;  // source row of the cy = +1 planes 2, 5, 6
  const long long rm = REV ? up : dn;  // source row of the cy = -1 planes 4, 7, 8
  const T* r[9] = {base,
                   base + plane,
                   base + 2 * plane + rp,
                   base + 3 * plane,
                   base + 4 * plane + rm,
                   base + 5 * plane + rp,
                   base + 6 * plane + rp,
                   base + 7 * plane + rm,
                   base + 8 * plane + rm};
#pragma unroll
  for (int q = 0; q < 9; ++q) vload<T, V, CG>(r[q] + i0, cv, v[q]);
  // cx = +1 planes (1, 5, 8) take column i - 1 forward, i + 1 in reverse; cx = -1
  // planes (3, 6, 7) the opposite
  if (!REV) {
    const T h1 = load_left_halo<T, CG>(r[1], i0, nx, lane, cv);
    const T h5 = load_left_halo<T, CG>(r[5], i0, nx, lane, cv);
    const T h8 = load_left_halo<T, CG>(r[8], i0, nx, lane, cv);
    const T h3 = load_right_halo<T, V, CG>(r[3], i0, nx, lane, cv);
    const T h6 = load_right_halo<T, V, CG>(r[6], i0, nx, lane, cv);
    const T h7 = load_right_halo<T, V, CG>(r[7], i0, nx, lane, cv);
    assemble_from_left<T, V>(v[1], h1, lane);
    assemble_from_left<T, V>(v[5], h5, lane);
    assemble_from_left<T, V>(v[8], h8, lane);
    assemble_from_right<T, V>(v[3], h3, i0, nx, lane);
    assemble_from_right<T, V>(v[6], h6, i0, nx, lane);
    assemble_from_right<T, V>(v[7], h7, i0, nx, lane);
  } else {
    const T h3 = load_left_halo<T, CG>(r[3], i0, nx, lane, cv);
    const T h6 = load_left_halo<T, CG>(r[6], i0, nx, lane, cv);
    const T h7 = load_left_halo<T, CG>(r[7], i0, nx, lane, cv);
    const T h1 = load_right_halo<T, V, CG>(r[1], i0, nx, lane, cv);
    const T h5 = load_right_halo<T, V, CG>(r[5], i0, nx, lane, cv);
    const T h8 = load_right_halo<T, V, CG>(r[8], i0, nx, lane, cv);
    assemble_from_left<T, V>(v[3], h3, lane);
    assemble_from_left<T, V>(v[6], h6, lane);
    assemble_from_left<T, V>(v[7], h7, lane);
    assemble_from_right<T, V>(v[1], h1, i0, nx, lane);
    assemble_from_right<T, V>(v[5], h5, i0, nx, lane);
    assemble_from_right<T, V>(v[8], h8, i0, nx, lane);
  }
}

// Moments and equilibrium of one cell, rounded exactly as the forward step rounds them.
template <class T>
__device__ __forceinline__ void adj_cell_eq(const T (&c)[9], T& ux, T& uy, T (&feq)[9]) {
  const T rho = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7])) + c[8];
  const T jx = (c[1] + c[5] + c[8]) - (c[3] + c[6] + c[7]);
  const T jy = (c[2] + c[5] + c[6]) - (c[4] + c[7] + c[8]);
  const T ir = Num<T>::rcp(rho);
  ux = Num<T>::mul(jx, ir);
  uy = Num<T>::mul(jy, ir);
  equilibrium<T>(rho, ux, uy, feq);
}

// For weights y_q: A = sum y_q D_q and B = sum y_q E_q (see the header comment).
template <class T>
__device__ __forceinline__ void adj_moment_pullback(const T (&y)[9], T ux, T uy, T& A, T& Bx,
                                                    T& By) {
  constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const T w[9] = {T(4.0 / 9.0),  T(1.0 / 9.0),  T(1.0 / 9.0),  T(1.0 / 9.0), T(1.0 / 9.0),
                  T(1.0 / 36.0), T(1.0 / 36.0), T(1.0 / 36.0), T(1.0 / 36.0)};
  const T g = fma(T(1.5), fma(ux, ux, uy * uy), T(1));  // 1 + 3/2 u.u
  T a = T(0), bx = T(0), by = T(0), sw = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const T cu = T(cx[q]) * ux + T(cy[q]) * uy;
    const T wy = w[q] * y[q];
    a = fma(wy, fma(T(-4.5) * cu, cu, g), a);
    const T s = wy * fma(T(9), cu, T(3));  // w y (3 + 9 c.u)
    if (cx[q]) bx = fma(T(cx[q]), s, bx);
    if (cy[q]) by = fma(T(cy[q]), s, by);
    sw += wy;
  }
  A = a;
  Bx = fma(T(-3) * ux, sw, bx);
  By = fma(T(-3) * uy, sw, by);
}

// Per-CTA partial of one sum, then the last CTA adds the partials in CTA order and
// adds the launch total to *p.acc.
template <class T>
__device__ __forceinline__ void adj_reduce(const AdjParams<T>& p, Acc<T>& s) {
  __shared__ Red<T> s_red[kWarps];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s.warp_reduce();
  if (lane == 0) s_red[warp] = Red<T>::of(s);
  __syncthreads();
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  const int nblocks = gridDim.x * gridDim.y;
  if (threadIdx.x == 0) {
    Red<T> t;
    for (int w = 0; w < kWarps; ++w) t.add(s_red[w]);
    t.store(p.part + bid);
    __threadfence();
    s_last = atomicAdd(p.done, 1u) == uint32_t(nblocks - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ Red<T> s_fin[kWarps];
  Red<T> t;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) t.add(Red<T>::load(p.part + b));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t.add(t.shfl_xor(off));
  if (lane == 0) s_fin[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    Red<T> r = s_fin[0];
    for (int w = 1; w < kWarps; ++w) r.add(s_fin[w]);
    *p.acc += r.value();
    *p.done = 0u;  // ready for the next launch (stream-ordered)
  }
}

// Replace the cells past the row end (padding of a ragged vector) by a positive rest
// state, so that they stay finite; they are neither summed nor read by real cells.
template <class T>
__device__ __forceinline__ void adj_pad(T (&v)[9][kAdjV], int nvalid, T value) {
#pragma unroll
  for (int q = 0; q < 9; ++q)
#pragma unroll
    for (int k = 0; k < kAdjV; ++k)
      if (k >= nvalid) v[q][k] = value;
}

// lt^{N-1} = W dKL/dft at ft = S f^{N-1}; adds sum W KL to *acc.
template <class T>
__global__ void __launch_bounds__(kThreads) adj_objective_kernel(const AdjParams<T> p) {
  constexpr int V = kAdjV;
  constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = (blockIdx.x * 32 + lane) * V;
  const bool cv = i0 < p.nx;
  const int nvalid = cv ? min(V, p.nx - i0) : 0;
  const int j0 = blockIdx.y * p.rows, j1 = min(j0 + p.rows, p.ny);
  Acc<T> sum;
  for (int j = j0 + warp; j < j1; j += kWarps) {
    T ft[9][V];
    adj_pull_row<T, false>(p.f, p.plane, p.pitch, p.nx, p.ny, j, i0, lane, cv, ft);
    adj_pad<T>(ft, nvalid, T(1));
    T wv[V];
    if (p.weight) {
      vload<T, V>(p.weight + (long long)j * p.pitch + i0, cv, wv);
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) wv[k] = T(1);
    }
    T g[9][V];
    T rs = T(0);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      T c[9], feq[9], x[9], ux, uy;
#pragma unroll
      for (int q = 0; q < 9; ++q) c[q] = ft[q][k];
      adj_cell_eq<T>(c, ux, uy, feq);
      bool nonpos = false;
      T K = T(0);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        nonpos |= (c[q] <= T(0)) | (feq[q] <= T(0));
        x[q] = (c[q] - feq[q]) / feq[q];
        K = fma(feq[q], phi<T>(x[q]), K);
      }
      T a, bx, by;
      adj_moment_pullback<T>(x, ux, uy, a, bx, by);
      const T sg = K > T(0) ? wv[k] : (K < T(0) ? -wv[k] : T(0));
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const T cb = T(cx[q]) * bx + T(cy[q]) * by;
        g[q][k] = nonpos ? T(CUDART_NAN) : sg * (Num<T>::log1p_(x[q]) - (a + cb));
      }
      if (k < nvalid) rs += wv[k] * (nonpos ? Num<T>::inf() : fabs(K));
    }
    sum.add(rs);
    if (cv) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
        vstore<T, V>(p.lam_out + q * p.plane + (long long)j * p.pitch + i0, g[q]);
    }
  }
  adj_reduce<T>(p, sum);
}

// lt^n from l^{n+1} = S^T lt^{n+1} and ft^n = S f^n for the block (bx, by) of the adjoint
// grid; returns the block's sum l^{n+1} . f^neq per thread (dJ/dtau = that sum over all
// steps / tau^2).  CG: the adjoint buffers are written by other CTAs of the same launch
// (the multi-step reverse sweep), so they are read with ordinary cached loads.
template <class T, bool CG>
__device__ __forceinline__ Acc<T> adj_step_block(const AdjParams<T>& p, int bx, int by) {
  constexpr int V = kAdjV;
  constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = (bx * 32 + lane) * V;
  const bool cv = i0 < p.nx;
  const int nvalid = cv ? min(V, p.nx - i0) : 0;
  const int j0 = by * p.rows, j1 = min(j0 + p.rows, p.ny);
  const T om = p.omega, om1 = T(1) - p.omega;
  Acc<T> sum;
  for (int j = j0 + warp; j < j1; j += kWarps) {
    T ft[9][V], l[9][V];
    adj_pull_row<T, false>(p.f, p.plane, p.pitch, p.nx, p.ny, j, i0, lane, cv, ft);
    adj_pull_row<T, true, CG>(p.lam_in, p.plane, p.pitch, p.nx, p.ny, j, i0, lane, cv, l);
    adj_pad<T>(ft, nvalid, T(1));
    adj_pad<T>(l, nvalid, T(0));
    T rs = T(0);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      T c[9], y[9], feq[9], ux, uy;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        c[q] = ft[q][k];
        y[q] = l[q][k];
      }
      adj_cell_eq<T>(c, ux, uy, feq);
#pragma unroll
      for (int q = 0; q < 9; ++q) rs = fma(y[q], c[q] - feq[q], rs);
      T A, bx_, by_;
      adj_moment_pullback<T>(y, ux, uy, A, bx_, by_);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const T cb = T(cx[q]) * bx_ + T(cy[q]) * by_;
        l[q][k] = fma(om1, y[q], om * (A + cb));
      }
    }
    sum.add(rs);
    if (cv) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
        vstore<T, V>(p.lam_out + q * p.plane + (long long)j * p.pitch + i0, l[q]);
    }
  }
  return sum;
}

template <class T>
__global__ void __launch_bounds__(kThreads) adj_step_kernel(const AdjParams<T> p) {
  Acc<T> sum = adj_step_block<T, false>(p, blockIdx.x, blockIdx.y);
  adj_reduce<T>(p, sum);
}

// ---- the reverse sweep of one segment in one cooperative launch ----
// Reverse iterations it = 0 .. nit - 1 (step k = last - it): work item w = it * nblocks + b
// is block b of iteration it, handed out in order from an atomic counter.  Block b of
// iteration it first waits until the blocks of its 3 x 3 neighbourhood (periodic) have
// completed iteration it - 1: they wrote the adjoint cells its reverse pull reads, and have
// read the cells it overwrites (the buffers alternate).  Every wait is bounded (bit 1 of the
// error word on expiry).  Each block's partial of the dJ/dtau sum goes to part[it][b]; the
// block completing iteration it last adds them as adj_reduce does and stores the
// iteration's total in totals[it]; adj_add_totals then adds the totals in iteration order,
// so the accumulator is that of one launch per step bit for bit.
template <class T>
struct AdjMulti {
  const T* ck;         // the segment's checkpoint state (step s0)
  const T* seg;        // recomputed states of steps s0 + 1 .. last, state_elems apart
  long long state_elems;
  const T* lam0;       // adjoint ping-pong: iteration it reads lam(lc + it), writes
  const T* lam1;       // lam(lc + it + 1), lam(k) = lam0 for even k, lam1 for odd
  uint32_t* done;      // [nblocks] iterations each block completed (0 at launch)
  uint32_t* ticket;    // [nit] blocks of each iteration completed (0 at launch)
  uint32_t* work;      // next work item (0 at launch)
  double* part;        // [nit][nblocks]
  double* totals;      // [nit]
  uint32_t* err;       // bit 1: a wait ran out
  long long deadline;  // clock64 cycles one wait may take
  int s0, last, lc;
  int gx, gy, nblocks;  // the adjoint grid (adj_grid): gx x gy blocks
};

__device__ __forceinline__ bool adj_wait_ge(const uint32_t* p, uint32_t want, uint32_t* err,
                                            long long deadline) {
  if (ld_acquire_u32(p) >= want) return true;
  const long long t0 = clock64();
  while (ld_acquire_u32(p) < want) {
    if (clock64() - t0 > deadline) {
      atomicOr(err, 2u);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Resident CTAs per SM requested from the register allocator for adj_multi_kernel (a
// build-time tuning knob; 0 leaves the choice to the compiler).
#ifndef KSS_ADJ_MULTI_MIN_BLOCKS
#define KSS_ADJ_MULTI_MIN_BLOCKS 0
#endif
template <class T>
__global__ void __launch_bounds__(kThreads, KSS_ADJ_MULTI_MIN_BLOCKS)
adj_multi_kernel(const AdjParams<T> base, const AdjMulti<T> m) {
  __shared__ int s_next, s_go, s_fin;
  __shared__ Red<T> s_red[kWarps];
  __shared__ Red<T> s_tot[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gx = m.gx, gy = m.gy;
  const int nit = m.last - m.s0 + 1;
  const int total = nit * m.nblocks;
  if (threadIdx.x == 0) s_next = int(atomicAdd(m.work, 1u));
  __syncthreads();
  int w = s_next;
  while (w < total) {
    const int it = w / m.nblocks, b = w - it * m.nblocks;
    const int by = b / gx, bx = b - by * gx;
    __syncthreads();  // every thread has read s_next before thread 0 rewrites it
    if (threadIdx.x < 32) {
      const int t = threadIdx.x;
      if (t == 0) s_next = int(atomicAdd(m.work, 1u));
      bool ok = true;
      if (it > 0 && t < 9) {
        const int dy = t / 3 - 1, dx = t - 3 * (t / 3) - 1;
        const int yy = by + dy < 0 ? gy - 1 : (by + dy == gy ? 0 : by + dy);
        const int xx = bx + dx < 0 ? gx - 1 : (bx + dx == gx ? 0 : bx + dx);
        ok = adj_wait_ge(m.done + yy * gx + xx, uint32_t(it), m.err, m.deadline);
      }
      ok = __all_sync(kFull, ok);
      if (t == 0) s_go = ok;
    }
    __syncthreads();
    if (!s_go) return;
    const int k = m.last - it;
    AdjParams<T> p = base;
    p.f = k == m.s0 ? m.ck : m.seg + (long long)(k - m.s0) * m.state_elems;
    const bool odd = ((m.lc + it) & 1) != 0;
    p.lam_in = odd ? m.lam1 : m.lam0;
    p.lam_out = const_cast<T*>(odd ? m.lam0 : m.lam1);
    Acc<T> sum = adj_step_block<T, true>(p, bx, by);
    // the block's partial, as adj_reduce forms it
    sum.warp_reduce();
    if (lane == 0) s_red[warp] = Red<T>::of(sum);
    __syncthreads();  // (also: every store of the block precedes thread 0's release)
    double* part = m.part + (long long)it * m.nblocks;
    if (threadIdx.x == 0) {
      Red<T> t;
      for (int q = 0; q < kWarps; ++q) t.add(s_red[q]);
      t.store(part + b);
      __threadfence();
      st_release_u32(m.done + b, uint32_t(it + 1));
      s_fin = atomicAdd(m.ticket + it, 1u) == uint32_t(m.nblocks - 1);
    }
    __syncthreads();
    if (s_fin) {  // the iteration's total, in adj_reduce's order
      __threadfence();
      Red<T> t;
      for (int q = threadIdx.x; q < m.nblocks; q += kThreads) t.add(Red<T>::load(part + q));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t.add(t.shfl_xor(off));
      if (lane == 0) s_tot[warp] = t;
      __syncthreads();
      if (threadIdx.x == 0) {
        Red<T> r = s_tot[0];
        for (int q = 1; q < kWarps; ++q) r.add(s_tot[q]);
        m.totals[it] = r.value();
      }
    }
    __syncthreads();
    w = s_next;
  }
}

// *acc += totals[0] + ... in iteration order, one addition each (as one launch per step
// adds its total).  (A template, instantiated per storage type, so that the header can be
// included by several translation units.)
template <class T>
__global__ void adj_add_totals(const double* totals, int n, double* acc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = *acc;
    for (int i = 0; i < n; ++i) a += totals[i];
    *acc = a;
  }
}

// dJ/drho0(x) = sum_q (S^T lt^0)_q(x) f^eq_q(1, u0(x)) (f^0 = f^eq(rho0, u0) is linear in
// rho0 at fixed u0), written as doubles to the dense grad array.
template <class T>
__global__ void __launch_bounds__(kThreads) adj_final_kernel(const AdjParams<T> p) {
  constexpr int V = kAdjV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = (blockIdx.x * 32 + lane) * V;
  const bool cv = i0 < p.nx;
  const int j0 = blockIdx.y * p.rows, j1 = min(j0 + p.rows, p.ny);
  for (int j = j0 + warp; j < j1; j += kWarps) {
    T l[9][V];
    adj_pull_row<T, true>(p.lam_in, p.plane, p.pitch, p.nx, p.ny, j, i0, lane, cv, l);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int i = i0 + k;
      if (!cv || i >= p.nx) continue;
      const long long c = (long long)j * p.nx + i;
      T e1[9];
      equilibrium<T>(T(1), T(p.ux0[c]), T(p.uy0[c]), e1);
      T s = T(0);
#pragma unroll
      for (int q = 0; q < 9; ++q) s = fma(l[q][k], e1[q], s);
      p.grad[c] = double(s);
    }
  }
}

}  // namespace kss
