/*
 * orc.c -- plain FP64 CPU oracle (see orc.h).  TEST INFRASTRUCTURE ONLY.
 *
 * Everything here is a direct transcription of a definition of the paper
 * (arXiv 2603.13618), cell by cell, in scalar double precision, with no
 * blocking, fusion or vectorisation.  Each function names the passage it
 * follows.  Readings where the paper is silent (D2Q9 lattice, the mu/lambda
 * of the class-1 sensors, the non-positive convention, the cancellation-free
 * form of the logarithmic sensors) are stated at the point of use.
 */
#include "orc.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocity set and Gauss-Hermite weights (section "Discrete kinetic
 * model": discrete velocities v_i with weights w_i). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* Reference temperature of the lattice, R T_ref = c_s^2 = 1/3. */
static const double CS2 = 1.0 / 3.0;

/* Row-parallel sweeps.  The per-cell loops below that write only their own cell's
 * outputs split their rows over g_threads OpenMP threads (1 by default, set by
 * orc_set_threads); no arithmetic depends on the split, so the results are the same
 * bit for bit at any thread count.  Loops that accumulate (flags and tile counts,
 * the compensated sums, the adjoint) stay serial. */
static int g_threads = 1;
#ifdef _OPENMP
#include <omp.h>
#define ORC_ROWS _Pragma("omp parallel for schedule(static) num_threads(g_threads)")
#else
#define ORC_ROWS
#endif

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int orc_get_threads(void) { return g_threads; }

int orc_have_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

static size_t at(int nx, int ny, int q, int i, int j) {
  return ((size_t)q * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i;
}

static int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

/* Grad-Hermite equilibrium to order N = 2: f^eq_i = w_i sum_n
 * a_n : H_n(v_i) / (n! (R T_ref)^n) with a_0 = rho, a_1 = rho u,
 * a_2 = rho u u (isothermal, T = T_ref) and H_0 = 1, H_1 = v,
 * H_2 = v v - R T_ref I. */
void orc_equilibrium(double rho, double ux, double uy, double feq[9]) {
  const double a1[2] = {rho * ux, rho * uy};
  const double a2[2][2] = {{rho * ux * ux, rho * ux * uy}, {rho * uy * ux, rho * uy * uy}};
  for (int q = 0; q < 9; ++q) {
    const double v[2] = {(double)CX[q], (double)CY[q]};
    double h1 = 0.0;
    for (int a = 0; a < 2; ++a) h1 += a1[a] * v[a];
    double h2 = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) h2 += a2[a][b] * (v[a] * v[b] - (a == b ? CS2 : 0.0));
    feq[q] = W[q] * (rho + h1 / CS2 + h2 / (2.0 * CS2 * CS2));
  }
}

void orc_init_equilibrium(int nx, int ny, const double* rho, const double* ux,
                          const double* uy, double* f) {
  ORC_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t c = (size_t)j * nx + i;
      double feq[9];
      orc_equilibrium(rho[c], ux[c], uy[c], feq);
      for (int q = 0; q < 9; ++q) f[at(nx, ny, q, i, j)] = feq[q];
    }
}

/* Streaming term v_i . grad f_i of the discrete kinetic equations, in its
 * lattice form with dt = dx = 1: pull every population from the neighbour
 * it comes from, periodic in both directions. */
void orc_stream(int nx, int ny, const double* f, double* ft) {
  for (int q = 0; q < 9; ++q)
    ORC_ROWS
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        ft[at(nx, ny, q, i, j)] = f[at(nx, ny, q, wrap(i - CX[q], nx), wrap(j - CY[q], ny))];
}

/* Moments as quadratures, Eqs. eq_quadratur1-2. */
static void cell_moments(const double ft[9], double* rho, double* ux, double* uy) {
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int q = 0; q < 9; ++q) {
    r += ft[q];
    jx += CX[q] * ft[q];
    jy += CY[q] * ft[q];
  }
  *rho = r;
  *ux = jx / r;
  *uy = jy / r;
}

/* Eq. new_collision_fi with tau1 = tau2 = tau (f* = f^eq): the discrete
 * collision operator Omega_i = -(f_i - f^eq_i)/tau, added with dt = 1. */
void orc_collide(int nx, int ny, double tau, const double* ft, double* fnext) {
  ORC_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double c[9], feq[9], rho, ux, uy;
      for (int q = 0; q < 9; ++q) c[q] = ft[at(nx, ny, q, i, j)];
      cell_moments(c, &rho, &ux, &uy);
      orc_equilibrium(rho, ux, uy, feq);
      for (int q = 0; q < 9; ++q) {
        const double omega = -(c[q] - feq[q]) / tau;
        fnext[at(nx, ny, q, i, j)] = c[q] + omega;
      }
    }
}

void orc_step(int nx, int ny, double tau, const double* f, double* fnext) {
  double* ft = (double*)malloc(sizeof(double) * 9 * (size_t)nx * ny);
  orc_stream(nx, ny, f, ft);
  orc_collide(nx, ny, tau, ft, fnext);
  free(ft);
}

/* ---------------------------------------------------------------- AAR ----
 * Adaptive algorithm refinement (section "Conclusions"): where a sensor flags a cell,
 * the single-relaxation BGK model gives way to a two-relaxation model, Eq.
 * new_collision_fi with a quasi-equilibrium f* distinct from f^eq.
 *
 * Reading for the single-distribution D2Q9 lattice.  The quasi-equilibria of the
 * paper are Grad-Hermite expansions built from the equilibrium moments plus the
 * quasi-conserved fields (section "Kinetic model": pressure tensor or heat flux).
 * Without an energy equation, the slow field kept here is the heat-flux-like one:
 * the odd (third-order) non-equilibrium moments, which are exactly the odd part of
 * f^neq under the velocity reversal i -> -i,
 *   f*_i = f^eq_i + (f^neq_i - f^neq_{-i}) / 2,   f^neq = f - f^eq.
 * tau1 (the lattice's tau) relaxes f toward f*, i.e. the even part of f^neq (the
 * stress, so nu = c_s^2 (tau1 - 1/2)); tau2 relaxes f* toward f^eq, i.e. the odd
 * part.  f* has the density and momentum of f, so both are conserved; tau2 = tau1
 * is BGK. */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6}; /* c_{OPP[i]} = -c_i */

void orc_quasi_equilibrium(const double ft[9], double fstar[9]) {
  double rho, ux, uy, feq[9];
  cell_moments(ft, &rho, &ux, &uy);
  orc_equilibrium(rho, ux, uy, feq);
  for (int q = 0; q < 9; ++q) {
    const double odd = 0.5 * ((ft[q] - feq[q]) - (ft[OPP[q]] - feq[OPP[q]]));
    fstar[q] = feq[q] + odd;
  }
}

/* Eq. new_collision_fi, added with dt = 1: in cells with region != 0
 *   Omega_i = -(f_i - f*_i)/tau1 - (f*_i - f^eq_i)/tau2,
 * elsewhere the BGK operator of orc_collide (computed by the same expression). */
void orc_collide_aar(int nx, int ny, double tau1, double tau2, const uint8_t* region,
                     const double* ft, double* fnext) {
  ORC_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double c[9], feq[9], rho, ux, uy;
      for (int q = 0; q < 9; ++q) c[q] = ft[at(nx, ny, q, i, j)];
      cell_moments(c, &rho, &ux, &uy);
      orc_equilibrium(rho, ux, uy, feq);
      if (region[(size_t)j * nx + i]) {
        double fstar[9];
        orc_quasi_equilibrium(c, fstar);
        for (int q = 0; q < 9; ++q) {
          const double omega = -(c[q] - fstar[q]) / tau1 - (fstar[q] - feq[q]) / tau2;
          fnext[at(nx, ny, q, i, j)] = c[q] + omega;
        }
      } else {
        for (int q = 0; q < 9; ++q) {
          const double omega = -(c[q] - feq[q]) / tau1;
          fnext[at(nx, ny, q, i, j)] = c[q] + omega;
        }
      }
    }
}

void orc_moments(int nx, int ny, const double* f, double* rho, double* ux, double* uy) {
  ORC_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double c[9];
      for (int q = 0; q < 9; ++q) c[q] = f[at(nx, ny, q, i, j)];
      const size_t k = (size_t)j * nx + i;
      cell_moments(c, &rho[k], &ux[k], &uy[k]);
    }
}

/* phi(x) = (1 + x) ln(1 + x) - x.  For |x| < 1/16 its Maclaurin series
 * sum_{n>=2} (-1)^n x^n / (n (n - 1)) (from the series of ln(1 + x)),
 * summed to n = 18; otherwise the closed form with log1p. */
static double phi(double x) {
  if (fabs(x) < 0.0625) {
    double s = 0.0, p = x * x;
    for (int n = 2; n <= 18; ++n) {
      s += ((n % 2 == 0) ? 1.0 : -1.0) * p / (double)(n * (n - 1));
      p *= x;
    }
    return s;
  }
  return (1.0 + x) * log1p(x) - x;
}

static double frob2(double a, double b, double c, double d) {
  return sqrt(a * a + b * b + c * c + d * d);
}

/* Entropic estimate, Eqs. alpha-polynomial-1/-2, read literally: f^neq =
 * f - f^eq (as defined at the start of section "Refinement sensors") and the
 * current populations f in the denominators.  a_1 = 0 (equilibrium) gives
 * alpha := 2. */
double orc_alpha_poly(const double ft[9], double a[4]) {
  double rho, ux, uy, feq[9];
  cell_moments(ft, &rho, &ux, &uy);
  orc_equilibrium(rho, ux, uy, feq);
  for (int n = 1; n <= 4; ++n) {
    double s = 0.0;
    for (int q = 0; q < 9; ++q) {
      const double fneq = ft[q] - feq[q];
      s += pow(fneq, n + 1) / pow(ft[q], n);
    }
    const double sign = (n % 2 == 1) ? 1.0 : -1.0; /* (-1)^(n-1) */
    a[n - 1] = sign * s / (double)(n * (n + 1));
  }
  const double a1 = a[0], a2 = a[1], a3 = a[2], a4 = a[3];
  if (a1 == 0.0) return 2.0;
  return 2.0 - 4.0 * a2 / a1 + 16.0 * a2 * a2 / (a1 * a1) - 8.0 * a3 / a1 +
         80.0 * a2 * a3 / (a1 * a1) - 80.0 * a2 * a2 * a2 / (a1 * a1 * a1) - 16.0 * a4 / a1;
}

/* g(alpha) = H(f + alpha (f^eq - f)) - H(f) with H of Eq.
 * H-function-discrete, written without cancellation: with D = f^eq - f,
 * y = D/f, and sum D = 0, g = alpha sum D ln(f/(w rho)) + sum f phi(alpha y). */
static double mirror_gap(const double ft[9], const double feq[9], double rho, double alpha) {
  double g = 0.0;
  for (int q = 0; q < 9; ++q) {
    const double d = feq[q] - ft[q];
    g += alpha * d * log(ft[q] / (W[q] * rho)) + ft[q] * phi(alpha * d / ft[q]);
  }
  return g;
}

/* Positive root of Eq. H-mirr-equal by bisection (diagnostic only). */
double orc_alpha_exact(const double ft[9]) {
  double rho, ux, uy, feq[9];
  cell_moments(ft, &rho, &ux, &uy);
  orc_equilibrium(rho, ux, uy, feq);
  double amax = INFINITY;
  int moved = 0;
  for (int q = 0; q < 9; ++q) {
    if (ft[q] <= 0.0 || feq[q] <= 0.0) return NAN;
    const double d = feq[q] - ft[q];
    if (d != 0.0) moved = 1;
    if (d < 0.0) {
      const double lim = ft[q] / (-d);
      if (lim < amax) amax = lim;
    }
  }
  if (!moved) return 2.0;
  double lo = 1.0e-3, hi = 2.0;
  if (mirror_gap(ft, feq, rho, lo) >= 0.0) return NAN;
  while (mirror_gap(ft, feq, rho, hi) < 0.0) {
    if (hi >= 0.999999 * amax || hi > 1.0e6) return NAN;
    hi = fmin(2.0 * hi, 0.5 * (hi + amax));
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (mirror_gap(ft, feq, rho, mid) < 0.0)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* All sensors of Table 1 for a single distribution (the g-terms dropped,
 * section "Overview and further considerations": the sensors apply to a
 * single distribution function), on the pre-collision populations ft.
 *
 * Class-1 reading for the isothermal D2Q9 BGK model: its first-order stress
 * is P^neq = -rho c_s^2 tau (grad u + grad u^T) with no separate bulk part,
 * i.e. in the notation of Eq. tauNS-1: mu = rho c_s^2 tau, lambda = 0 and
 * eta = 2 mu / D + lambda = mu.
 *
 * Logarithmic sensors: f ln(f/f^eq) = f^eq phi(x) + f^neq with x = f^neq/f^eq,
 * and sum f^neq = 0 exactly (rho of f and of f^eq coincide, Eq.
 * eq_quadratur1), so the sums are evaluated term-by-term without the O(1)
 * cancellation of the printed form:
 *   KL       = |sum f^eq phi(x)|
 *   HR       = |sum f^neq L + sum f^eq phi(x)|,     L = ln(f^eq/(w rho))
 *   sigma_H  = (1/tau) (sum f^neq L + sum f^neq ln(1 + x))
 *   sigma_KL = (1/tau) sum f^neq ln(1 + x)
 * (the constant ln(rho) parts multiply sum f^neq = 0).  The printed forms
 * are kept in orc_cell_log_sensors_literal and checked against these.
 *
 * Non-positive populations (section "Overview and further considerations":
 * positivity is not guaranteed by Grad-Hermite equilibria): if any ft_q <= 0
 * or f^eq_q <= 0, Kn and the five entropy-based sensors are +Inf.        */
int orc_cell_sensors(const double ft[9], double tau, double out[ORC_NSENS]) {
  return orc_cell_sensors_model(ft, tau, 0, out);
}

int orc_cell_sensors_model(const double ft[9], double tau, int two_relax,
                           double out[ORC_NSENS]) {
  return orc_cell_sensors_set(ft, tau, two_relax, 1, out);
}

/* full = 0: only Kn, neq, qe and KL (the sensor set that the flags of a production run
 * use), by the same lines as the full evaluation; the other entries are NaN. */
int orc_cell_sensors_set(const double ft[9], double tau, int two_relax, int full,
                         double out[ORC_NSENS]) {
  double rho, ux, uy, feq[9], fneq[9];
  cell_moments(ft, &rho, &ux, &uy);
  orc_equilibrium(rho, ux, uy, feq);
  int nonpos = 0;
  for (int q = 0; q < 9; ++q) {
    fneq[q] = ft[q] - feq[q];
    if (ft[q] <= 0.0 || feq[q] <= 0.0) nonpos = 1;
  }

  for (int k = 0; k < ORC_NSENS; ++k) out[k] = NAN;
  if (full) {
  /* Non-equilibrium pressure tensor P^neq = sum v v f^neq. */
  double P[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int q = 0; q < 9; ++q) {
    const double v[2] = {(double)CX[q], (double)CY[q]};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) P[a][b] += v[a] * v[b] * fneq[q];
  }
  const double D = 2.0;
  const double mu = rho * CS2 * tau;
  const double lambda = 0.0;
  const double eta = 2.0 * mu / D + lambda;
  const double trP = P[0][0] + P[1][1];

  out[ORC_TAU_NS] = frob2(P[0][0], P[0][1], P[1][0], P[1][1]);
  out[ORC_C] = sqrt(D) * fabs(-trP / (2.0 * mu + D * lambda));
  {
    double M[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) M[a][b] = ((a == b ? trP / D : 0.0) - P[a][b]) / mu;
    out[ORC_S] = frob2(M[0][0], M[0][1], M[1][0], M[1][1]);
  }
  {
    double M[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        M[a][b] = ((a == b ? lambda / (D * eta) * trP : 0.0) - P[a][b]) / (2.0 * mu);
    out[ORC_E] = frob2(M[0][0], M[0][1], M[1][0], M[1][1]);
  }
  {
    /* (sum v f / sum f) . P^neq */
    double jx = 0.0, jy = 0.0, r = 0.0;
    for (int q = 0; q < 9; ++q) {
      r += ft[q];
      jx += CX[q] * ft[q];
      jy += CY[q] * ft[q];
    }
    const double u[2] = {jx / r, jy / r};
    double qh[2] = {0.0, 0.0};
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) qh[b] += u[a] * P[a][b];
    out[ORC_QH] = sqrt(qh[0] * qh[0] + qh[1] * qh[1]);
  }
  }
  {
    /* f*: the equilibrium itself for BGK, else the quasi-equilibrium of the
     * two-relaxation model (orc_quasi_equilibrium) */
    double fstar[9];
    if (two_relax)
      orc_quasi_equilibrium(ft, fstar);
    else
      for (int q = 0; q < 9; ++q) fstar[q] = feq[q];
    double kn = 0.0, neq = 0.0, qe = 0.0;
    for (int q = 0; q < 9; ++q) {
      kn += fabs(fneq[q] / feq[q]);
      neq += fabs(fneq[q]);
      qe += fabs(fstar[q] - feq[q]);
    }
    out[ORC_KN] = kn;
    out[ORC_NEQ] = neq;
    out[ORC_QE] = qe;
  }
  {
    double kl = 0.0;
    for (int q = 0; q < 9; ++q) {
      const double x = fneq[q] / feq[q];
      kl += feq[q] * phi(x);
    }
    out[ORC_KL] = fabs(kl);
    if (full) {
      double lin = 0.0, sig = 0.0;
      for (int q = 0; q < 9; ++q) {
        const double x = fneq[q] / feq[q];
        const double L = log(feq[q] / (W[q] * rho));
        lin += fneq[q] * L;
        sig += fneq[q] * log1p(x);
      }
      out[ORC_HR] = fabs(lin + kl);
      out[ORC_SIGMA_H] = (lin + sig) / tau;
      out[ORC_SIGMA_KL] = sig / tau;
    }
  }
  if (full) {
    /* |2 - alpha| of Eq. sensor-alpha-kin with alpha of Eq. alpha-polynomial-1;
     * the constant 2 cancels exactly, so the correction terms are summed directly */
    double a[4];
    orc_alpha_poly(ft, a);
    double e = 0.0;
    if (a[0] != 0.0) {
      const double a1 = a[0], a2 = a[1], a3 = a[2], a4 = a[3];
      e = 4.0 * a2 / a1 - 16.0 * a2 * a2 / (a1 * a1) + 8.0 * a3 / a1 -
          80.0 * a2 * a3 / (a1 * a1) + 80.0 * a2 * a2 * a2 / (a1 * a1 * a1) + 16.0 * a4 / a1;
    }
    out[ORC_ALPHA] = fabs(e);
  }
  if (nonpos) {
    out[ORC_KN] = INFINITY;
    out[ORC_KL] = INFINITY;
    if (full) {
      out[ORC_HR] = INFINITY;
      out[ORC_SIGMA_H] = INFINITY;
      out[ORC_SIGMA_KL] = INFINITY;
      out[ORC_ALPHA] = INFINITY;
    }
  }
  return nonpos;
}

/* Printed forms: Eq. Hneq-sensor, Eq. HKL-sensor, Eq. Dissip-H-sensor and
 * Eq. Dissip-HKL-sensor, with Omega_i = -(f_i - f^eq_i)/tau. */
void orc_cell_log_sensors_literal(const double ft[9], double tau, double out[4],
                                  double scale[4]) {
  double rho, ux, uy, feq[9];
  cell_moments(ft, &rho, &ux, &uy);
  orc_equilibrium(rho, ux, uy, feq);
  double hf = 0.0, hfeq = 0.0, kl = 0.0, sh = 0.0, skl = 0.0;
  double s_hr = 0.0, s_kl = 0.0, s_sh = 0.0, s_skl = 0.0;
  for (int q = 0; q < 9; ++q) {
    const double omega = -(ft[q] - feq[q]) / tau;
    const double t1 = ft[q] * log(ft[q] / W[q]);
    const double t2 = feq[q] * log(feq[q] / W[q]);
    const double t3 = ft[q] * log(ft[q] / feq[q]);
    const double t4 = omega * log(ft[q] / W[q]);
    const double t5 = omega * log(ft[q] / feq[q]);
    hf += t1;
    hfeq += t2;
    kl += t3;
    sh += t4;
    skl += t5;
    /* rounding scale: |term| plus |prefactor| (the log's argument is rounded
     * to one ulp, i.e. the log is off by ~eps absolute); for sigma_H also
     * the rounding of Omega (~eps f / tau) times |ln(f/w)| */
    s_hr += fabs(t1) + fabs(t2) + ft[q] + feq[q];
    s_kl += fabs(t3) + ft[q];
    s_sh += fabs(t4) + fabs(omega) + ft[q] / tau * fabs(log(ft[q] / W[q]));
    s_skl += fabs(t5) + fabs(omega);
  }
  out[0] = fabs(hf - hfeq);
  out[1] = fabs(kl);
  out[2] = -sh;
  out[3] = -skl;
  scale[0] = s_hr;
  scale[1] = s_kl;
  scale[2] = s_sh;
  scale[3] = s_skl;
}

void orc_sensor_fields(int nx, int ny, double tau, const double* f, int pull, double* out,
                       uint8_t* nonpos) {
  orc_sensor_fields_model(nx, ny, tau, 0, f, pull, out, nonpos);
}

void orc_sensor_fields_model(int nx, int ny, double tau, int two_relax, const double* f,
                             int pull, double* out, uint8_t* nonpos) {
  ORC_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double c[9], s[ORC_NSENS];
      for (int q = 0; q < 9; ++q) {
        const int si = pull ? wrap(i - CX[q], nx) : i;
        const int sj = pull ? wrap(j - CY[q], ny) : j;
        c[q] = f[at(nx, ny, q, si, sj)];
      }
      const int np = orc_cell_sensors_model(c, tau, two_relax, s);
      for (int k = 0; k < ORC_NSENS; ++k) out[at(nx, ny, k, i, j)] = s[k];
      if (nonpos) nonpos[(size_t)j * nx + i] = (uint8_t)np;
    }
}

/* Regrid step (1) of the SAMR cycle: tag cells whose sensor exceeds its
 * threshold (strict comparison); the AAR switch is a second criterion. */
void orc_flags(int nx, int ny, const double* eps_r, double thr_r, const double* eps_s,
               double thr_s, const uint8_t* nonpos, int tile, uint8_t* flags,
               int32_t* tiles, int64_t counts[3]) {
  const int ntx = (nx + tile - 1) / tile, nty = (ny + tile - 1) / tile;
  for (int k = 0; k < 2 * ntx * nty; ++k) tiles[k] = 0;
  counts[0] = counts[1] = counts[2] = 0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t c = (size_t)j * nx + i;
      const int r = eps_r[c] > thr_r;
      const int s = (thr_s >= 0.0) && (eps_s[c] > thr_s);
      const int p = nonpos ? nonpos[c] != 0 : 0;
      flags[c] = (uint8_t)(r | (s << 1) | (p << 7));
      const int t = (j / tile) * ntx + (i / tile);
      tiles[t] += r;
      tiles[ntx * nty + t] += s;
      counts[0] += r;
      counts[1] += s;
      counts[2] += p;
    }
}

/* Neumaier-compensated running sum, so the lattice totals are accurate to a
 * few ulps of the result whatever the lattice size (a naive running sum of
 * 9 nx ny terms drifts by ~sqrt(n) ulps of the total). */
static void kahan_add(double* s, double* c, double v) {
  const double t = *s + v;
  if (fabs(*s) >= fabs(v))
    *c += (*s - t) + v;
  else
    *c += (v - t) + *s;
  *s = t;
}

void orc_sums(int nx, int ny, const double* f, double sums[3]) {
  double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int q = 0; q < 9; ++q) {
        const double v = f[at(nx, ny, q, i, j)];
        kahan_add(&s[0], &c[0], v);
        kahan_add(&s[1], &c[1], CX[q] * v);
        kahan_add(&s[2], &c[2], CY[q] * v);
      }
  for (int k = 0; k < 3; ++k) sums[k] = s[k] + c[k];
}

void orc_mac_sensors(int nx, int ny, double tau, const double* rho, const double* ux,
                     const double* uy, double* out) {
  const size_t n = (size_t)nx * ny;
  ORC_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t c = (size_t)j * nx + i;
      const size_t ip = (size_t)j * nx + wrap(i + 1, nx), im = (size_t)j * nx + wrap(i - 1, nx);
      const size_t jp = (size_t)wrap(j + 1, ny) * nx + i, jm = (size_t)wrap(j - 1, ny) * nx + i;
      /* G[a][b] = d_a u_b */
      const double G[2][2] = {{0.5 * (ux[ip] - ux[im]), 0.5 * (uy[ip] - uy[im])},
                              {0.5 * (ux[jp] - ux[jm]), 0.5 * (uy[jp] - uy[jm])}};
      const double div = G[0][0] + G[1][1];
      const double mu = rho[c] * CS2 * tau;
      double sym[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) sym[a][b] = G[a][b] + G[b][a];
      out[c] = mu * frob2(sym[0][0], sym[0][1], sym[1][0], sym[1][1]);
      out[n + c] = sqrt(2.0) * fabs(div);
      out[2 * n + c] = frob2(sym[0][0] - div, sym[0][1], sym[1][0], sym[1][1] - div);
      out[3 * n + c] = 0.5 * frob2(sym[0][0], sym[0][1], sym[1][0], sym[1][1]);
    }
}

int64_t orc_run(int nx, int ny, double tau, double* f, double* work, int nsteps,
                int sensor_r, double thr_r, int sensor_s, double thr_s, int tile,
                double* rec_field, uint8_t* flags, int32_t* tiles, int64_t counts[3],
                double sums[3], int full) {
  const size_t n = (size_t)nx * ny;
  double* eps_s = (double*)malloc(sizeof(double) * n);
  uint8_t* np = (uint8_t*)malloc(n);
  for (int step = 0; step < nsteps; ++step) {
    orc_stream(nx, ny, f, work);
    ORC_ROWS
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double c[9], s[ORC_NSENS];
        for (int q = 0; q < 9; ++q) c[q] = work[at(nx, ny, q, i, j)];
        np[(size_t)j * nx + i] = (uint8_t)orc_cell_sensors_set(c, tau, 0, full, s);
        rec_field[(size_t)j * nx + i] = s[sensor_r];
        eps_s[(size_t)j * nx + i] = s[sensor_s];
      }
    orc_flags(nx, ny, rec_field, thr_r, eps_s, thr_s, np, tile, flags, tiles, counts);
    orc_sums(nx, ny, work, sums);
    orc_collide(nx, ny, tau, work, f);
  }
  free(eps_s);
  free(np);
  return counts[2];
}

/* ---------------------------------------------------------------- adjoint ----
 * Reverse-mode derivative of the sensor objective of orc_adjoint_kl (orc.h).
 * Everything below differentiates the definitions used above as written: the
 * Grad-Hermite equilibrium, the BGK collision, pull streaming, and the KL sensor
 * in its printed form eps_KL = |sum_i f_i ln(f_i / f^eq_i)| (Eq. HKL-sensor). */

/* Derivatives of the equilibrium with respect to the conserved moments rho and
 * j = rho u.  With u = j / rho the GH expansion of orc_equilibrium reads
 *   f^eq_i = w_i (rho + c_i.j / c_s^2 + ((c_i.j)^2 - c_s^2 |j|^2) / (2 c_s^4 rho)). */
static void feq_moment_derivs(double rho, double jx, double jy, double drho[9],
                              double djx[9], double djy[9]) {
  const double j2 = jx * jx + jy * jy;
  for (int q = 0; q < 9; ++q) {
    const double cj = CX[q] * jx + CY[q] * jy;
    drho[q] = W[q] * (1.0 - (cj * cj - CS2 * j2) / (2.0 * CS2 * CS2 * rho * rho));
    djx[q] = W[q] * (CX[q] / CS2 + (cj * CX[q] - CS2 * jx) / (CS2 * CS2 * rho));
    djy[q] = W[q] * (CY[q] / CS2 + (cj * CY[q] - CS2 * jy) / (CS2 * CS2 * rho));
  }
}

/* d f^eq_q / d f_p: f^eq depends on f through rho = sum f and j = sum c f. */
static double feq_dfp(const double drho[9], const double djx[9], const double djy[9], int q,
                      int p) {
  return drho[q] + CX[p] * djx[q] + CY[p] * djy[q];
}

/* Gradient g[9] of eps_KL(ft) = |K|, K = sum_q ft_q ln(ft_q / f^eq_q(ft)):
 *   dK/dft_p = ln(ft_p / f^eq_p) + 1 - sum_q (ft_q / f^eq_q) d f^eq_q / d ft_p,
 * times sign(K).  Cells with a non-positive population get NaN. */
static void cell_kl_grad(const double ft[9], double g[9]) {
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int q = 0; q < 9; ++q) {
    rho += ft[q];
    jx += CX[q] * ft[q];
    jy += CY[q] * ft[q];
  }
  double feq[9], drho[9], djx[9], djy[9];
  orc_equilibrium(rho, jx / rho, jy / rho, feq);
  feq_moment_derivs(rho, jx, jy, drho, djx, djy);
  int nonpos = 0;
  double K = 0.0;
  for (int q = 0; q < 9; ++q) {
    if (ft[q] <= 0.0 || feq[q] <= 0.0) nonpos = 1;
    K += feq[q] * phi(ft[q] / feq[q] - 1.0);  /* = sum ft ln(ft/feq), as in orc_cell_sensors */
  }
  const double sgn = K > 0.0 ? 1.0 : (K < 0.0 ? -1.0 : 0.0);
  for (int p = 0; p < 9; ++p) {
    if (nonpos) {
      g[p] = NAN;
      continue;
    }
    double s = 0.0;
    for (int q = 0; q < 9; ++q) s += (ft[q] / feq[q]) * feq_dfp(drho, djx, djy, q, p);
    g[p] = sgn * (log(ft[p] / feq[p]) + 1.0 - s);
  }
}

/* Transpose of orc_stream: lf_q(i, j) = lt_q(i + cx_q, j + cy_q). */
static void stream_transpose(int nx, int ny, const double* lt, double* lf) {
  for (int q = 0; q < 9; ++q)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        lf[at(nx, ny, q, i, j)] = lt[at(nx, ny, q, wrap(i + CX[q], nx), wrap(j + CY[q], ny))];
}

int orc_adjoint_kl(int nx, int ny, double tau, int nsteps, int store_every, const double* rho0,
                   const double* ux0, const double* uy0, const double* weight, double* J,
                   double* grad_rho0, double* grad_tau) {
  if (nsteps < 1 || store_every < 1) return -1;
  const size_t n = (size_t)nx * ny, S = 9 * n;
  /* f^0 .. f^{N-1}: every store_every-th state kept, the others recomputed per segment */
  const int nck = (nsteps - 1) / store_every + 1;
  double* ck = (double*)malloc(sizeof(double) * S * (size_t)nck);
  double* seg = (double*)malloc(sizeof(double) * S * (size_t)store_every);
  double* ft = (double*)malloc(sizeof(double) * S);
  double* lt = (double*)malloc(sizeof(double) * S);
  double* lf = (double*)malloc(sizeof(double) * S);
  if (!ck || !seg || !ft || !lt || !lf) {
    free(ck), free(seg), free(ft), free(lt), free(lf);
    return -1;
  }
  orc_init_equilibrium(nx, ny, rho0, ux0, uy0, ck);
  double* cur = ft; /* scratch while stepping forward */
  memcpy(cur, ck, sizeof(double) * S);
  for (int k = 1; k < nsteps; ++k) {
    orc_step(nx, ny, tau, cur, lt);
    memcpy(cur, lt, sizeof(double) * S);
    if (k % store_every == 0) memcpy(ck + S * (size_t)(k / store_every), cur, sizeof(double) * S);
  }
  /* cur = f^{N-1}.  Objective on its streamed image, and its gradient lt = dJ/dft^{N-1}. */
  double* fN = lf;
  memcpy(fN, cur, sizeof(double) * S);
  orc_stream(nx, ny, fN, ft);
  double js = 0.0, jc = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double c[9], s[ORC_NSENS], g[9];
      for (int q = 0; q < 9; ++q) c[q] = ft[at(nx, ny, q, i, j)];
      orc_cell_sensors(c, tau, s);
      cell_kl_grad(c, g);
      const double w = weight ? weight[(size_t)j * nx + i] : 1.0;
      kahan_add(&js, &jc, w * s[ORC_KL]);
      for (int q = 0; q < 9; ++q) lt[at(nx, ny, q, i, j)] = w * g[q];
    }
  *J = js + jc;
  /* Reverse sweep over f^{n+1} = collide(stream(f^n)), n = N-2 .. 0:
   * lf = dJ/df^{n+1} = stream^T(lt), then lt = dJ/dft^n = (d collide / d ft)^T lf and
   * dJ/dtau += sum lf . d collide/d tau = sum lf (ft - f^eq) / tau^2. */
  double gs = 0.0, gc = 0.0;
  for (int seg0 = ((nsteps - 2) / store_every) * store_every; nsteps >= 2 && seg0 >= 0;
       seg0 -= store_every) {
    /* states f^{seg0} .. f^{seg0 + store_every - 1} of this segment (those < N-1) */
    const int last = seg0 + store_every - 1 < nsteps - 2 ? seg0 + store_every - 1 : nsteps - 2;
    memcpy(seg, ck + S * (size_t)(seg0 / store_every), sizeof(double) * S);
    for (int k = seg0 + 1; k <= last; ++k)
      orc_step(nx, ny, tau, seg + S * (size_t)(k - 1 - seg0), seg + S * (size_t)(k - seg0));
    for (int k = last; k >= seg0; --k) {
      stream_transpose(nx, ny, lt, lf);
      orc_stream(nx, ny, seg + S * (size_t)(k - seg0), ft);
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double c[9], l[9], feq[9], drho[9], djx[9], djy[9];
          double rho = 0.0, jx = 0.0, jy = 0.0;
          for (int q = 0; q < 9; ++q) {
            c[q] = ft[at(nx, ny, q, i, j)];
            l[q] = lf[at(nx, ny, q, i, j)];
            rho += c[q];
            jx += CX[q] * c[q];
            jy += CY[q] * c[q];
          }
          orc_equilibrium(rho, jx / rho, jy / rho, feq);
          feq_moment_derivs(rho, jx, jy, drho, djx, djy);
          for (int q = 0; q < 9; ++q) kahan_add(&gs, &gc, l[q] * (c[q] - feq[q]) / (tau * tau));
          for (int p = 0; p < 9; ++p) {
            /* d fnext_q / d ft_p = delta_qp (1 - 1/tau) + (1/tau) d f^eq_q / d ft_p */
            double s = 0.0;
            for (int q = 0; q < 9; ++q) s += l[q] * feq_dfp(drho, djx, djy, q, p);
            lt[at(nx, ny, p, i, j)] = (1.0 - 1.0 / tau) * l[p] + s / tau;
          }
        }
    }
  }
  *grad_tau = gs + gc;
  /* dJ/df^0 = stream^T(lt); f^0 = f^eq(rho0, u0) is rho0 times f^eq(1, u0) at fixed u0 */
  stream_transpose(nx, ny, lt, lf);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t c = (size_t)j * nx + i;
      double e1[9];
      orc_equilibrium(1.0, ux0[c], uy0[c], e1);
      double s = 0.0;
      for (int q = 0; q < 9; ++q) s += lf[at(nx, ny, q, i, j)] * e1[q];
      grad_rho0[c] = s;
    }
  free(ck), free(seg), free(ft), free(lt), free(lf);
  return 0;
}

/* ------------------------------------------------------ FP16 deviation storage ----
 * The storage form of populations as FP16 deviations from the rest equilibrium (the
 * storage choice of the lattice library, not a formula of the paper):
 *   h_q = RN16((f_q - b_q) s_q),  b_q = RN32(w_q rho0),  s_q = 2^(k_q + K),
 *   k_q = 1, 3, 5 for w_q = 4/9, 1/9, 1/36 (s_q = 1 when unscaled),
 *   decoded f_q = RN32(b_q + h_q / s_q).
 * RN16 / RN32: round to the nearest binary16 / binary32 value, ties to even. */

/* Nearest IEEE binary16 value of x (ties to even), as a double; +-Inf beyond the
 * largest finite value 65504 (from 65520 up, the midpoint to 2^16). */
double orc_fp16_round(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  const double a = fabs(x);
  if (a >= 65520.0) return x > 0 ? INFINITY : -INFINITY;
  int e2;
  frexp(a, &e2);             /* a = m 2^e2, m in [0.5, 1): binade exponent e2 - 1 */
  int e = e2 - 1;
  if (e < -14) e = -14;      /* subnormal range: fixed spacing 2^-24 */
  const double quantum = ldexp(1.0, e - 10);
  const double r = rint(a / quantum) * quantum;  /* rint: nearest, ties to even */
  return x > 0 ? r : -r;
}

static void dev16_params(double rho0, int dev_exp, int unscaled, double b[9], double s[9]) {
  static const int K[9] = {1, 3, 3, 3, 3, 5, 5, 5, 5};
  for (int q = 0; q < 9; ++q) {
    b[q] = (double)(float)(W[q] * rho0);
    s[q] = unscaled ? 1.0 : ldexp(1.0, K[q] + dev_exp);
  }
}

void orc_dev16_encode(int nx, int ny, double rho0, int dev_exp, int unscaled, const double* f,
                      double* h) {
  double b[9], s[9];
  dev16_params(rho0, dev_exp, unscaled, b, s);
  for (int q = 0; q < 9; ++q)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t k = at(nx, ny, q, i, j);
        h[k] = orc_fp16_round((f[k] - b[q]) * s[q]);
      }
}

void orc_dev16_decode(int nx, int ny, double rho0, int dev_exp, int unscaled, const double* h,
                      double* f) {
  double b[9], s[9];
  dev16_params(rho0, dev_exp, unscaled, b, s);
  for (int q = 0; q < 9; ++q)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t k = at(nx, ny, q, i, j);
        f[k] = (double)(float)(b[q] + h[k] / s[q]);
      }
}
