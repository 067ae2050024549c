// d2q9.cuh -- per-cell arithmetic of the fused step: moments, Grad-Hermite N = 2
// equilibrium, BGK collision and the local kinetic sensors of Table 1 of
// arXiv 2603.13618 (single distribution), in the storage precision T.
//
// Everything here works on registers only; the kernels in step_kernel.cuh feed it
// the nine post-streaming populations of a cell.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace kss {

// Sensor ids (same numbering as kss_sensor in include/kss.h).
enum : int {
  S_TAU_NS = 0, S_C, S_S, S_E, S_QH, S_KN, S_NEQ, S_QE, S_HR, S_KL, S_SIGMA_H,
  S_SIGMA_KL, S_ALPHA, S_COUNT
};

// Sensor sets compiled into a kernel: none (plain stream + collide), the cheap
// set {Kn, KL, neq} that the flags of a production run use, or all of Table 1.
enum Mode : int { MODE_PLAIN = 0, MODE_STD = 1, MODE_FULL = 2 };
constexpr uint32_t kStdMask = (1u << S_KN) | (1u << S_KL) | (1u << S_NEQ);

template <class T> struct Num;

template <> struct Num<float> {
  // highest power of the Maclaurin series of phi used for |x| < 1/16:
  // the first dropped term x^8/56 is below 2^-24 of x^2/2 there.
  static constexpr int kPhiOrder = 7;
  // order of the series in the fused Kn/KL/neq path (|x| < 1/16; larger |x| take
  // the closed form): the first dropped term, x^6/30, is at most 1.0e-6 of x^2/2.
  static constexpr int kPhiFastOrder = 5;
  // reciprocal: the hardware approximation (rcp.approx, at most 1 ulp error)
  __device__ static __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  __device__ static __forceinline__ float log1p_(float x) { return log1pf(x); }
  __device__ static __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  __device__ static __forceinline__ float inf() { return CUDART_INF_F; }
  // rounded product / sum that the compiler never fuses into an FMA (see equilibrium)
  __device__ static __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ static __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ static __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
};

template <> struct Num<double> {
  // first dropped term x^16/240 is below 2^-53 of x^2/2 for |x| < 1/16
  static constexpr int kPhiOrder = 15;
  static constexpr int kPhiFastOrder = 15;
  __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
  __device__ static __forceinline__ double log1p_(double x) { return log1p(x); }
  __device__ static __forceinline__ double sqrt_(double x) { return sqrt(x); }
  __device__ static __forceinline__ double inf() { return CUDART_INF; }
  __device__ static __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
};

// Coefficient of x^n in phi(x) = (1 + x) ln(1 + x) - x = sum_{n>=2} (-1)^n x^n / (n (n-1)),
// as a compile-time constant (a runtime double division would run on the FP64 pipe).
template <int n>
struct PhiCoef {
  static constexpr double value = ((n & 1) ? -1.0 : 1.0) / double(n * (n - 1));
};

// Horner evaluation of sum_{m=2}^{N} c_m x^(m-2), from the top coefficient down.
template <class T, int n>
struct PhiHorner {
  __device__ static __forceinline__ T eval(T x, T acc) {
    return PhiHorner<T, n - 1>::eval(x, fma(acc, x, T(PhiCoef<n - 1>::value)));
  }
};
template <class T>
struct PhiHorner<T, 2> {
  __device__ static __forceinline__ T eval(T, T acc) { return acc; }
};

// phi(x) / x^2 = sum_{n=2}^{N} c_n x^(n-2), for the fused path (|x| < 1/16 known).
template <class T, int N>
__device__ __forceinline__ T phi_over_x2(T x) {
  return PhiHorner<T, N>::eval(x, T(PhiCoef<N>::value));
}

template <class T, int N>
__device__ __forceinline__ T phi_series(T x) {
  return (x * x) * phi_over_x2<T, N>(x);
}

// phi(x) = (1 + x) ln(1 + x) - x without cancellation near x = 0.
template <class T>
__device__ __forceinline__ T phi(T x) {
  if (fabs(x) < T(0.0625)) return phi_series<T, Num<T>::kPhiOrder>(x);
  return (T(1) + x) * Num<T>::log1p_(x) - x;
}

// Grad-Hermite equilibrium to second order at R T_ref = c_s^2 = 1/3, expanded:
// f^eq_q = w_q rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u).
//
// Every rounding of the collision is fixed: the velocity u = j / rho, the diagonal
// projections u_x +- u_y and each f^eq_q are rounded products / sums (Num::mul, add,
// sub) that the compiler cannot contract with the subtraction f - f^eq that follows,
// and the other operations are explicit FMAs.  The kernels that step with or without
// sensors (and the all-sensor per-cell path) therefore produce the same populations
// bit for bit, and rho w_q is formed as rho (1/9) times 4, 1 or 1/4 (exact scalings).
template <class T>
__device__ __forceinline__ void equilibrium(T rho, T ux, T uy, T (&feq)[9]) {
  const T base = fma(T(-1.5), fma(ux, ux, uy * uy), T(1));
  const T r1 = rho * T(1.0 / 9.0);
  const T r0 = T(4) * r1, r2 = T(0.25) * r1;
  feq[0] = Num<T>::mul(r0, base);
  const T tx = fma(T(4.5) * ux, ux, base), ty = fma(T(4.5) * uy, uy, base);
  feq[1] = Num<T>::mul(r1, fma(T(3), ux, tx));
  feq[3] = Num<T>::mul(r1, fma(T(-3), ux, tx));
  feq[2] = Num<T>::mul(r1, fma(T(3), uy, ty));
  feq[4] = Num<T>::mul(r1, fma(T(-3), uy, ty));
  const T s = Num<T>::add(ux, uy);  // c5 = (1,1): c.u = s ; c7 = -c5
  const T d = Num<T>::sub(uy, ux);  // c6 = (-1,1): c.u = d ; c8 = -c6
  const T ts = fma(T(4.5) * s, s, base), td = fma(T(4.5) * d, d, base);
  feq[5] = Num<T>::mul(r2, fma(T(3), s, ts));
  feq[7] = Num<T>::mul(r2, fma(T(-3), s, ts));
  feq[6] = Num<T>::mul(r2, fma(T(3), d, td));
  feq[8] = Num<T>::mul(r2, fma(T(-3), d, td));
}

// Per-cell results that the kernels reduce or store.
template <class T>
struct CellOut {
  T rho, jx, jy;
  T sv[S_COUNT];  // only the entries of the compiled sensor set are written
  bool nonpos;
};

// Pick sensor `id` with compile-time indices only (keeps sv[] in registers).
template <class T>
__device__ __forceinline__ T pick(const T (&sv)[S_COUNT], int id) {
  switch (id) {
    case S_TAU_NS: return sv[S_TAU_NS];
    case S_C: return sv[S_C];
    case S_S: return sv[S_S];
    case S_E: return sv[S_E];
    case S_QH: return sv[S_QH];
    case S_KN: return sv[S_KN];
    case S_NEQ: return sv[S_NEQ];
    case S_QE: return sv[S_QE];
    case S_HR: return sv[S_HR];
    case S_KL: return sv[S_KL];
    case S_SIGMA_H: return sv[S_SIGMA_H];
    case S_SIGMA_KL: return sv[S_SIGMA_KL];
    default: return sv[S_ALPHA];
  }
}

// Two-relaxation model of adaptive algorithm refinement (section "Conclusions"), in
// cells of the switched region: Eq. new_collision_fi with the quasi-equilibrium
// f*_q = f^eq_q + (f^neq_q - f^neq_-q)/2 (the odd part of f^neq kept), i.e.
//   f'_q = f_q - A f^neq_q - B f^neq_-q,  A = (1/tau1 + 1/tau2)/2,  B = (1/tau1 - 1/tau2)/2,
// and f'_0 = f_0 - f^neq_0 / tau1.  Outside the region A = 1/tau1 and B = 0, which gives
// the BGK update bit for bit (a zero product added).
template <class T>
struct Trt {
  T a = T(0), b = T(0);  // A and B of a switched cell
  bool qe = false;       // the lattice's model is the two-relaxation one: eps_qe is
                         // sum |f* - f^eq| (else f* = f^eq and eps_qe = 0)
};

// Index of the opposite velocity, c_{opp(q)} = -c_q: 0; 1 <-> 3, 2 <-> 4; 5 <-> 7, 6 <-> 8.
__host__ __device__ constexpr int opp(int q) {
  return q == 0 ? 0 : (q <= 4 ? ((q + 1) & 3) + 1 : ((q - 3) & 3) + 5);
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2 && opp(5) == 7 &&
                  opp(6) == 8 && opp(7) == 5 && opp(8) == 6 && opp(0) == 0,
              "opposite velocities");

// One cell: moments of the post-streaming populations ft, equilibrium, the sensors
// of the compiled set, and (COLLIDE) the BGK update fo = ft - (ft - f^eq)/tau, or
// (AAR) the two-relaxation update in a switched cell (sw).
//
// Logarithmic sensors use x = f^neq/f^eq, phi(x) and sum_q f^neq_q = 0 (rho of ft
// and of f^eq coincide), so no O(1) terms cancel:
//   KL = |sum f^eq phi(x)|,  HR = |sum f^neq L + sum f^eq phi(x)|,
//   sigma_H = (sum f^neq L + sum f^neq ln(1+x)) / tau,
//   sigma_KL = sum f^neq ln(1+x) / tau,   L_q = ln(f^eq_q / (w_q rho)).
template <class T, int MODE, bool COLLIDE, bool AAR = false>
__device__ __forceinline__ void cell_update(const T (&ft)[9], T omega, T tau, T (&fo)[9],
                                            CellOut<T>& o, const Trt<T>& trt = Trt<T>{},
                                            bool sw = false) {
  const T rho = ((ft[0] + ft[1]) + (ft[2] + ft[3])) + ((ft[4] + ft[5]) + (ft[6] + ft[7])) + ft[8];
  const T jx = (ft[1] + ft[5] + ft[8]) - (ft[3] + ft[6] + ft[7]);
  const T jy = (ft[2] + ft[5] + ft[6]) - (ft[4] + ft[7] + ft[8]);
  const T inv_rho = Num<T>::rcp(rho);
  const T ux = Num<T>::mul(jx, inv_rho), uy = Num<T>::mul(jy, inv_rho);
  T feq[9];
  equilibrium<T>(rho, ux, uy, feq);
  o.rho = rho;
  o.jx = jx;
  o.jy = jy;
  if (COLLIDE) {
    if constexpr (AAR) {
      const T A = sw ? trt.a : omega, B = sw ? trt.b : T(0);
      T d[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) d[q] = ft[q] - feq[q];
      fo[0] = fma(-omega, d[0], ft[0]);
#pragma unroll
      for (int q = 1; q < 9; ++q) fo[q] = fma(-B, d[opp(q)], fma(-A, d[q], ft[q]));
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) fo[q] = fma(-omega, ft[q] - feq[q], ft[q]);
    }
  }
  if (MODE == MODE_PLAIN) {
    o.nonpos = false;
    return;
  }
  T fneq[9], x[9];
  bool nonpos = false;
  T kn = T(0), neq = T(0), kl = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    fneq[q] = ft[q] - feq[q];
    nonpos |= (ft[q] <= T(0)) | (feq[q] <= T(0));
    x[q] = fneq[q] * Num<T>::rcp(feq[q]);
    kn += fabs(x[q]);
    neq += fabs(fneq[q]);
    kl = fma(feq[q], phi<T>(x[q]), kl);
  }
  const T kInf = Num<T>::inf();
  o.nonpos = nonpos;
  o.sv[S_KN] = nonpos ? kInf : kn;
  o.sv[S_NEQ] = neq;
  o.sv[S_KL] = nonpos ? kInf : fabs(kl);
  // sum_q |f*_q - f^eq_q| = sum_q |f^neq_q - f^neq_-q| / 2 = sum over the 4 pairs of
  // |f^neq_q - f^neq_-q| (in the fused pair order); 0 for BGK, whose quasi-equilibrium is
  // the equilibrium
  o.sv[S_QE] = trt.qe ? ((fabs(fneq[1] - fneq[3]) + fabs(fneq[2] - fneq[4])) +
                         fabs(fneq[5] - fneq[7])) +
                            fabs(fneq[6] - fneq[8])
                      : T(0);
  if (MODE != MODE_FULL) return;

  // ---- class 1: the non-equilibrium pressure tensor P^neq = sum c c f^neq ----
  const T diag = (fneq[5] + fneq[6]) + (fneq[7] + fneq[8]);
  const T pxx = (fneq[1] + fneq[3]) + diag;
  const T pyy = (fneq[2] + fneq[4]) + diag;
  const T pxy = (fneq[5] - fneq[6]) + (fneq[7] - fneq[8]);
  const T mu = rho * (tau * T(1.0 / 3.0));  // mu = rho c_s^2 tau, lambda = 0, eta = mu
  const T inv_mu = Num<T>::rcp(mu);
  const T norm_p = Num<T>::sqrt_(fma(pxx, pxx, fma(pyy, pyy, T(2) * pxy * pxy)));
  const T half_dev = T(0.5) * (pyy - pxx);  // tr P / 2 - P_xx
  o.sv[S_TAU_NS] = norm_p;
  o.sv[S_C] = T(1.4142135623730951) * fabs(pxx + pyy) * (T(0.5) * inv_mu);
  o.sv[S_S] = Num<T>::sqrt_(T(2) * fma(half_dev, half_dev, pxy * pxy)) * inv_mu;
  o.sv[S_E] = norm_p * (T(0.5) * inv_mu);
  {
    const T qx = fma(ux, pxx, uy * pxy), qy = fma(ux, pxy, uy * pyy);
    o.sv[S_QH] = Num<T>::sqrt_(fma(qx, qx, qy * qy));
  }

  // ---- entropy-based sensors ----
  // L_q = ln(f^eq_q / (w_q rho)) = ln(1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
  T lin = T(0), sig = T(0);
  {
    const T usq15 = T(1.5) * fma(ux, ux, uy * uy);
    const T s = ux + uy, d = uy - ux;
    T arg[9];
    arg[0] = -usq15;
    arg[1] = fma(T(4.5) * ux, ux, fma(T(3), ux, -usq15));
    arg[3] = fma(T(4.5) * ux, ux, fma(T(-3), ux, -usq15));
    arg[2] = fma(T(4.5) * uy, uy, fma(T(3), uy, -usq15));
    arg[4] = fma(T(4.5) * uy, uy, fma(T(-3), uy, -usq15));
    arg[5] = fma(T(4.5) * s, s, fma(T(3), s, -usq15));
    arg[7] = fma(T(4.5) * s, s, fma(T(-3), s, -usq15));
    arg[6] = fma(T(4.5) * d, d, fma(T(3), d, -usq15));
    arg[8] = fma(T(4.5) * d, d, fma(T(-3), d, -usq15));
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      lin = fma(fneq[q], Num<T>::log1p_(arg[q]), lin);
      sig = fma(fneq[q], Num<T>::log1p_(x[q]), sig);
    }
  }
  const T inv_tau = omega;  // 1 / tau
  o.sv[S_HR] = nonpos ? kInf : fabs(lin + kl);
  o.sv[S_SIGMA_H] = nonpos ? kInf : (lin + sig) * inv_tau;
  o.sv[S_SIGMA_KL] = nonpos ? kInf : sig * inv_tau;

  // ---- entropic estimate: literal polynomial with f^neq = f - f^eq ----
  // a_n = (-1)^(n-1)/(n(n+1)) sum (f^neq)^(n+1)/f^n ;  |2 - alpha| =
  // |4 r2 - 16 r2^2 + 8 r3 - 80 r2 r3 + 80 r2^3 + 16 r4|, r_n = a_n / a_1.
  {
    T s1 = T(0), s2 = T(0), s3 = T(0), s4 = T(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const T y = fneq[q] * Num<T>::rcp(ft[q]);
      const T t1 = fneq[q] * y, t2 = t1 * y, t3 = t2 * y, t4 = t3 * y;
      s1 += t1;
      s2 += t2;
      s3 += t3;
      s4 += t4;
    }
    const T a1 = T(0.5) * s1, a2 = T(-1.0 / 6.0) * s2, a3 = T(1.0 / 12.0) * s3,
            a4 = T(-1.0 / 20.0) * s4;
    T eps_alpha = T(0);
    if (a1 != T(0)) {
      const T inv_a1 = Num<T>::rcp(a1);
      const T r2 = a2 * inv_a1, r3 = a3 * inv_a1, r4 = a4 * inv_a1;
      const T dev = T(4) * r2 - T(16) * r2 * r2 + T(8) * r3 - T(80) * r2 * r3 +
                    T(80) * r2 * r2 * r2 + T(16) * r4;
      eps_alpha = fabs(dev);
    }
    o.sv[S_ALPHA] = nonpos ? kInf : eps_alpha;
  }
}

}  // namespace kss
