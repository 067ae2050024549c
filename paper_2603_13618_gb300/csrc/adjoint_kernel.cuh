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
  uint32_t* err;         // error word (bit 2: a debug bounds check failed)
  long long plane;
  int pitch, nx, ny;
  int rows;              // rows per CTA (grid adj_grid(nx, ny, rows))
  T omega;
  T zero;                // 0, read at run time (see product2)
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
// state, so that they stay finite; they are neither summed nor read by real cells.  Only
// the lanes that hold such cells take the branch (the others skip its selects).
template <class T>
__device__ __forceinline__ void adj_pad(T (&v)[9][kAdjV], int nvalid, T value) {
  if (nvalid >= kAdjV) return;
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

// Paired FP32 form of the reverse step's cell arithmetic (KSS_ADJ_PAIRED): a thread's two
// cells are one pair of the f32x2 instructions.  Moments and f^eq are rounded as the
// forward step's paired row rounds them (fused_row_paired); the vector-Jacobian product is
// regrouped per opposite pair (p, -p) of populations, with S = w (y_p + y_-p) and
// D = w (y_p - y_-p) (D_p = D_-p, c_-p = -c_p):
//   A = w_0 y_0 g + sum_pairs S (g - 9/2 (c_p.u)^2),                 g = 1 + 3/2 u.u
//   B = sum_pairs c_p (3 D + 9 (c_p.u) S) - 3 u (w_0 y_0 + sum_pairs S),
// the same sums as adj_moment_pullback in another order of rounding.
#ifndef KSS_ADJ_PAIRED
#define KSS_ADJ_PAIRED 1
#endif

__device__ __forceinline__ void adj_cell_pairs(const F2 (&c)[9], const F2 (&y)[9], F2 om,
                                               F2 om1, F2 zero, F2 (&lt)[9], F2& rs) {
  const F2 rho = add2(add2(add2(add2(c[0], c[1]), add2(c[2], c[3])),
                           add2(add2(c[4], c[5]), add2(c[6], c[7]))),
                      c[8]);
  const F2 jx = sub2(add2(add2(c[1], c[5]), c[8]), add2(add2(c[3], c[6]), c[7]));
  const F2 jy = sub2(add2(add2(c[2], c[5]), c[6]), add2(add2(c[4], c[7]), c[8]));
  const F2 ir = rcp2(rho);
  const F2 ux = mul2(jx, ir), uy = mul2(jy, ir);
  const F2 uu = fma2(ux, ux, mul2(uy, uy));
  const F2 base = fma2(splat2(-1.5f), uu, splat2(1.f));
  const F2 r1 = mul2(rho, splat2(float(1.0 / 9.0)));
  const F2 r2 = mul2(splat2(0.25f), r1);
  const F2 sd[2] = {add2(ux, uy), sub2(uy, ux)};
  // f^eq, and the dtau partial sum y . (c - f^eq)
  F2 feq[9];
  feq[0] = product2(mul2(splat2(4.f), r1), base, zero);
  const F2 cu[4] = {ux, uy, sd[0], sd[1]};
  constexpr int qp[4] = {1, 2, 5, 6}, qm[4] = {3, 4, 7, 8};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const F2 rw = k < 2 ? r1 : r2;
    const F2 t = fma2(mul2(splat2(4.5f), cu[k]), cu[k], base);
    feq[qp[k]] = product2(rw, fma2(splat2(3.f), cu[k], t), zero);
    feq[qm[k]] = product2(rw, fma2(splat2(-3.f), cu[k], t), zero);
  }
  F2 acc = splat2(0.f);
#pragma unroll
  for (int q = 0; q < 9; ++q) acc = fma2(y[q], sub2(c[q], feq[q]), acc);
  rs = acc;
  // A and B
  const F2 g = fma2(splat2(1.5f), uu, splat2(1.f));
  const F2 wy0 = mul2(splat2(float(4.0 / 9.0)), y[0]);
  F2 a = mul2(wy0, g), sw = wy0, bx = splat2(0.f), by = splat2(0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const F2 w = splat2(k < 2 ? float(1.0 / 9.0) : float(1.0 / 36.0));
    const F2 S = mul2(w, add2(y[qp[k]], y[qm[k]]));
    const F2 D = mul2(w, sub2(y[qp[k]], y[qm[k]]));
    a = fma2(fma2(mul2(splat2(-4.5f), cu[k]), cu[k], g), S, a);
    const F2 t = fma2(mul2(splat2(9.f), cu[k]), S, mul2(splat2(3.f), D));
    // c_p = (1, 0), (0, 1), (1, 1), (-1, 1)
    if (k == 0 || k == 2) bx = add2(bx, t);
    if (k == 3) bx = sub2(bx, t);
    if (k >= 1) by = add2(by, t);
    sw = add2(sw, S);
  }
  bx = fma2(mul2(splat2(-3.f), ux), sw, bx);
  by = fma2(mul2(splat2(-3.f), uy), sw, by);
  // lt_q = (1 - omega) y_q + omega (A + c_q . B)
  const F2 oa = mul2(om, a), obx = mul2(om, bx), oby = mul2(om, by);
  const F2 ob[4] = {obx, oby, add2(obx, oby), sub2(oby, obx)};
  lt[0] = fma2(om1, y[0], oa);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    lt[qp[k]] = fma2(om1, y[qp[k]], add2(oa, ob[k]));
    lt[qm[k]] = fma2(om1, y[qm[k]], sub2(oa, ob[k]));
  }
}

// One row j of the reverse step: lt^n from l^{n+1} = S^T lt^{n+1} (pulled here) and
// ft^n = S f^n (pulled by the caller into ft); adds the row's l^{n+1} . f^neq to sum.
// CG: the adjoint buffers are written by other CTAs of the same launch (the multi-step
// reverse sweep), so they are read with ordinary cached loads.
template <class T, bool CG>
__device__ __forceinline__ void adj_step_row(const AdjParams<T>& p, int j, int i0, int lane,
                                             bool cv, int nvalid, T (&ft)[9][kAdjV],
                                             Acc<T>& sum) {
  constexpr int V = kAdjV;
  constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const T om = p.omega, om1 = T(1) - p.omega;
  T l[9][V];
  adj_pull_row<T, true, CG>(p.lam_in, p.plane, p.pitch, p.nx, p.ny, j, i0, lane, cv, l);
  adj_pad<T>(ft, nvalid, T(1));
  adj_pad<T>(l, nvalid, T(0));
  if constexpr (KSS_ADJ_PAIRED && std::is_same<T, float>::value && V == 2) {
    F2 c[9], y[9], lt[9], rs2;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      c[q] = pack2(ft[q][0], ft[q][1]);
      y[q] = pack2(l[q][0], l[q][1]);
    }
    adj_cell_pairs(c, y, splat2(om), splat2(om1), splat2(p.zero), lt, rs2);
    float r0, r1;
    unpack2(rs2, r0, r1);
    sum.add(r0 + r1);
    if (cv) {
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        unpack2(lt[q], l[q][0], l[q][1]);
        vstore<T, V>(p.lam_out + q * p.plane + (long long)j * p.pitch + i0, l[q]);
      }
    }
    return;
  }
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

// The reverse step for the block (bx, by) of the adjoint grid; returns the block's sum
// l^{n+1} . f^neq per thread (dJ/dtau = that sum over all steps / tau^2).  PRE: the
// warp's first row of ft^n was pulled by the caller into ft0 (the multi-step sweep issues
// those loads before it waits for its neighbours: the forward state is not written in
// the launch).
template <class T, bool CG, bool PRE = false>
__device__ __forceinline__ Acc<T> adj_step_block(const AdjParams<T>& p, int bx, int by,
                                                 T (*ft0)[kAdjV] = nullptr) {
  constexpr int V = kAdjV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = (bx * 32 + lane) * V;
  const bool cv = i0 < p.nx;
  const int nvalid = cv ? min(V, p.nx - i0) : 0;
  const int j0 = by * p.rows, j1 = min(j0 + p.rows, p.ny);
  Acc<T> sum;
  if (!bounds_ok(bx >= 0 && by >= 0 && bx * 32 * V < p.pitch && j0 < p.ny, p.err)) return sum;
  for (int j = j0 + warp; j < j1; j += kWarps) {
    T ft[9][V];
    if (PRE && j == j0 + warp) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int k = 0; k < V; ++k) ft[q][k] = ft0[q][k];
    } else {
      adj_pull_row<T, false>(p.f, p.plane, p.pitch, p.nx, p.ny, j, i0, lane, cv, ft);
    }
    adj_step_row<T, CG>(p, j, i0, lane, cv, nvalid, ft, sum);
  }
  return sum;
}

template <class T>
__global__ void __launch_bounds__(kThreads) adj_step_kernel(const AdjParams<T> p) {
  Acc<T> sum = adj_step_block<T, false>(p, blockIdx.x, blockIdx.y);
  adj_reduce<T>(p, sum);
}

// ---- the reverse sweep of one segment in one cooperative launch ----
// Reverse iterations it = 0 .. nit - 1 (step k = last - it), each over the nblocks blocks of
// the adjoint grid.  Block b of iteration it first waits until the blocks of its 3 x 3
// neighbourhood (periodic) have completed iteration it - 1: they wrote the adjoint cells its
// reverse pull reads, and have read the cells it overwrites (the buffers alternate).  Each
// block's partial of the dJ/dtau sum goes to part[it][b].  After the launch,
// adj_iteration_totals adds each iteration's partials as adj_reduce does, and the
// iteration totals to the accumulator in iteration order, so the accumulator is that of
// one launch per step bit for bit (and no block of the sweep waits for a counter of its
// iteration before it takes its next item).
//
// The same launch recomputes the previous segment (fsteps > 0): its plain forward steps
// t = 1 .. fsteps from the checkpoint fck into the states fseg + t (the forward step's own
// CTA body over the forward grid, fnblocks blocks).  Those states are not read by the
// reverse iterations of this launch (they belong to the next launch), and the reverse
// sweep's latency-bound waits leave the SMs idle enough to take them.  Forward block fb of
// step t waits until its 3 x 3 neighbourhood has completed step t - 1 (the rows its pull
// reads); every state has a slot of its own, so nothing else is overwritten.
//
// Work items are handed out in order from an atomic counter, in rounds: round r holds the
// reverse iteration r (if r < nit) and the forward step r + 1 (if r < fsteps).  Every item
// waits only for items handed out before it (in its own chain), so the smallest unfinished
// item can always proceed: no deadlock, given co-residency (the cooperative launch).  Every
// wait is bounded (bit 1 of the error word on expiry).
// Resident CTAs per SM requested from the register allocator for the FP32 adj_multi_kernel
// (a build-time tuning knob; FP64 takes the registers it needs).  Measured at 512^2 with
// the paired cell arithmetic: three (80 registers, a little spilling) 2.551 ms per
// gradient, four (64) 2.618 ms; with the scalar arithmetic three 2.609, four 2.634-2.698,
// two (128 registers) 3.144 and five (48 registers, 484 bytes of spills) 3.492 ms.  The
// sweep is bound by the latency of its dependent items, so more of them in flight pays
// more than registers, up to the point where spills lengthen each item.
#ifndef KSS_ADJ_MULTI_MIN_BLOCKS
#define KSS_ADJ_MULTI_MIN_BLOCKS 3
#endif
// Sleep between two polls of a neighbour's counter, in nanoseconds (0: poll back to back).
#ifndef KSS_ADJ_POLL_NS
#define KSS_ADJ_POLL_NS 64
#endif
// Order within a round of adj_multi_kernel's work items: the reverse iteration first (0) or
// the forward step first (1); either order keeps each chain's items in order.
#ifndef KSS_ADJ_FWD_FIRST
#define KSS_ADJ_FWD_FIRST 0
#endif

template <class T>
struct AdjMulti {
  const T* ck;         // the segment's checkpoint state (step s0)
  const T* seg;        // recomputed states of steps s0 + 1 .. last, state_elems apart
  long long state_elems;
  const T* lam0;       // adjoint ping-pong: iteration it reads lam(lc + it), writes
  const T* lam1;       // lam(lc + it + 1), lam(k) = lam0 for even k, lam1 for odd
  uint32_t* done;      // [nblocks] iterations each block completed (0 at launch)
  uint32_t* ticket;    // adj_iteration_totals' block counter (0 at launch)
  uint32_t* work;      // next work item (0 at launch)
  double* part;        // [nit][nblocks]
  double* totals;      // [nit]
  uint32_t* err;       // bit 1: a wait ran out
  long long deadline;  // clock64 cycles one wait may take
  int s0, last, lc;
  int gx, gy, nblocks;  // the adjoint grid (adj_grid): gx x gy blocks
  // the previous segment's recomputation (fsteps = 0: none)
  StepParams<T> fp;    // plain step parameters (src and dst are set per step)
  const T* fck;        // its checkpoint (state 0)
  T* fseg;             // its states 1 .. fsteps at fseg + t state_elems
  uint32_t* fdone;     // [fnblocks] forward steps each block completed (0 at launch)
  int fsteps;
  int fgx, fgy, fnblocks;  // the forward step grid (step_grid)
};

// Orders this thread's earlier memory operations, and those it observed (through the
// CTA barrier before it), before its later ones at GPU scope (a release fence).
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ bool adj_wait_ge(const uint32_t* p, uint32_t want, uint32_t* err,
                                            long long deadline) {
  if (ld_acquire_u32(p) >= want) return true;
  const long long t0 = clock64();
  while (ld_acquire_u32(p) < want) {
    if (clock64() - t0 > deadline) {
      atomicOr(err, 2u);
      return false;
    }
    if (KSS_ADJ_POLL_NS > 0) __nanosleep(KSS_ADJ_POLL_NS);
  }
  return true;
}

// Warp 0: lanes 0..8 wait (bounded) until the 3 x 3 neighbourhood of block (bx, by) of a
// gx x gy grid has done[] >= want; lane 0 also takes the CTA's next work item.  Returns,
// to every thread after the barrier, whether all waits succeeded.
__device__ __forceinline__ bool adj_wait_neighbours(const uint32_t* done, int bx, int by,
                                                    int gx, int gy, uint32_t want, bool wait,
                                                    uint32_t* work, int* s_next, int* s_go,
                                                    uint32_t* err, long long deadline) {
  if (threadIdx.x < 32) {
    const int t = threadIdx.x;
    if (t == 0) *s_next = int(atomicAdd(work, 1u));
    bool ok = true;
    if (wait && t < 9) {
      const int dy = t / 3 - 1, dx = t - 3 * (t / 3) - 1;
      const int yy = by + dy < 0 ? gy - 1 : (by + dy == gy ? 0 : by + dy);
      const int xx = bx + dx < 0 ? gx - 1 : (bx + dx == gx ? 0 : bx + dx);
      ok = adj_wait_ge(done + yy * gx + xx, want, err, deadline);
    }
    ok = __all_sync(kFull, ok);
    if (t == 0) *s_go = ok;
  }
  __syncthreads();
  return *s_go != 0;
}

template <class T>
__global__ void __launch_bounds__(kThreads,
                                  std::is_same<T, float>::value ? KSS_ADJ_MULTI_MIN_BLOCKS : 1)
adj_multi_kernel(const AdjParams<T> base, const AdjMulti<T> m) {
  __shared__ int s_next, s_go;
  __shared__ Red<T> s_red[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gx = m.gx, gy = m.gy;
  const int nit = m.last - m.s0 + 1;
  const int both = min(nit, m.fsteps);
  const int round = m.nblocks + m.fnblocks;
  const int total = nit * m.nblocks + m.fsteps * m.fnblocks;
  if (threadIdx.x == 0) s_next = int(atomicAdd(m.work, 1u));
  __syncthreads();
  int w = s_next;
  while (w < total) {
    // the item: reverse iteration it, block b; or forward step t, block b
    int it = -1, t = 0, b;
    if (w < both * round) {
      const int r = w / round, o = w - r * round;
      if (KSS_ADJ_FWD_FIRST ? o >= m.fnblocks : o < m.nblocks) {
        it = r;
        b = KSS_ADJ_FWD_FIRST ? o - m.fnblocks : o;
      } else {
        t = r + 1;
        b = KSS_ADJ_FWD_FIRST ? o : o - m.nblocks;
      }
    } else {
      const int w2 = w - both * round;
      if (nit > both) {
        it = both + w2 / m.nblocks;
        b = w2 - (it - both) * m.nblocks;
      } else {
        const int r = w2 / m.fnblocks;
        t = both + 1 + r;
        b = w2 - r * m.fnblocks;
      }
    }
    if (it < 0) {  // ---- a forward step of the previous segment's recomputation
      const int fby = b / m.fgx, fbx = b - fby * m.fgx;
      __syncthreads();  // every thread has read s_next before thread 0 rewrites it
      if (!adj_wait_neighbours(m.fdone, fbx, fby, m.fgx, m.fgy, uint32_t(t - 1), t > 1, m.work,
                               &s_next, &s_go, m.err, m.deadline))
        return;
      StepParams<T> q = m.fp;
      q.src = t == 1 ? m.fck : m.fseg + (long long)(t - 1) * m.state_elems;
      q.dst = m.fseg + (long long)t * m.state_elems;
      step_block<T, MODE_PLAIN, true, true, true>(q, fbx, fby, m.fgx, nullptr, nullptr);
      __syncthreads();  // every store of the block precedes thread 0's release
      w = s_next;
      // (the other warps go on to their next item meanwhile; the barrier before its
      // wait keeps s_next until everyone has read it)
      if (threadIdx.x == 0) {
        fence_acq_rel_gpu();
        st_release_u32(m.fdone + b, uint32_t(t));
      }
      continue;
    }
    // ---- a reverse iteration of this segment
    const int by = b / gx, bx = b - by * gx;
    const int k = m.last - it;
    AdjParams<T> p = base;
    p.f = k == m.s0 ? m.ck : m.seg + (long long)(k - m.s0) * m.state_elems;
    const bool odd = ((m.lc + it) & 1) != 0;
    p.lam_in = odd ? m.lam1 : m.lam0;
    p.lam_out = const_cast<T*>(odd ? m.lam0 : m.lam1);
    // the warp's first row of the forward state (written before the launch), pulled
    // while the block waits for its neighbours
    T ft0[9][kAdjV];
    {
      const int i0 = (bx * 32 + lane) * kAdjV, jf = by * p.rows + warp;
      if (jf < min(by * p.rows + p.rows, p.ny))
        adj_pull_row<T, false>(p.f, p.plane, p.pitch, p.nx, p.ny, jf, i0, lane, i0 < p.nx,
                               ft0);
    }
    __syncthreads();  // every thread has read s_next before thread 0 rewrites it
    if (!adj_wait_neighbours(m.done, bx, by, gx, gy, uint32_t(it), it > 0, m.work, &s_next,
                             &s_go, m.err, m.deadline))
      return;
    Acc<T> sum = adj_step_block<T, true, true>(p, bx, by, ft0);
    // the neighbours wait only for the adjoint stores: the release comes first, then the
    // block's partial (read after the launch), as adj_reduce forms it
    sum.warp_reduce();
    if (lane == 0) s_red[warp] = Red<T>::of(sum);
    __syncthreads();  // every store of the block precedes thread 0's release
    w = s_next;
    // (as above; s_red is rewritten only after the next item's barriers)
    if (threadIdx.x == 0) {
      fence_acq_rel_gpu();
      st_release_u32(m.done + b, uint32_t(it + 1));
      Red<T> r;
      for (int q = 0; q < kWarps; ++q) r.add(s_red[q]);
      r.store(m.part + (long long)it * m.nblocks + b);
    }
  }
}

// Block it: the total of iteration it's per-block partials part[it][0 .. nblocks - 1],
// added as adj_reduce adds one launch's partials, into totals[it].  The block finishing
// last (count, 0 at launch) then does *acc += totals[0] + ... in iteration order, one
// addition each (as one launch per step adds its total).
template <class T>
__global__ void __launch_bounds__(kThreads)
adj_iteration_totals(const double* part, int nblocks, int nit, double* totals,
                     uint32_t* count, double* acc) {
  __shared__ Red<T> s_tot[kWarps];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, it = blockIdx.x;
  const double* pp = part + (long long)it * nblocks;
  Red<T> r;
  for (int q = threadIdx.x; q < nblocks; q += kThreads) r.add(Red<T>::load(pp + q));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) r.add(r.shfl_xor(off));
  if (lane == 0) s_tot[warp] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    Red<T> r2 = s_tot[0];
    for (int q = 1; q < kWarps; ++q) r2.add(s_tot[q]);
    totals[it] = r2.value();
    __threadfence();
    s_last = atomicAdd(count, 1u) == uint32_t(nit - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    double a = *acc;
    for (int i = 0; i < nit; ++i) a += __ldcg(totals + i);
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
