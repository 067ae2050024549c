/*
 * orc.h -- plain FP64 CPU oracle for the fused D2Q9 stream + BGK collide + local
 * kinetic sensor step of "Local kinetic sensors for adaptive mesh and algorithm
 * refinement" (arXiv 2603.13618).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library under paper_2603_13618_gb300/.
 *
 * Layout: populations are structure-of-arrays f[q][j][i] (q = 0..8, j = row,
 * i = column, i fastest), dense (row pitch = nx), FP64.  Cell (i, j) sits at
 * x = i, y = j, lattice units dx = dt = 1.  Velocities (D2Q9):
 *   c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
 *   c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1),  weights 4/9, 1/9 x4, 1/36 x4.
 *
 * Parity status (see each function): every sensor except the entropic
 * estimate (ORC_ALPHA) is pinned by closed forms, invariants or hand-derived
 * special cases in tests/test_oracle_*.py.  ORC_ALPHA is "parity unpinned"
 * beyond its printed polynomial (section "Entropic estimate sensor", Eqs.
 * alpha-polynomial-1/-2): the polynomial does not reproduce the exact mirror
 * root of Eq. H-mirr-equal to first order, so nothing independent fixes it.
 * The discrete adjoint (orc_adjoint_kl) is pinned by central finite differences of
 * the objective evaluated with the forward functions alone (tests/test_oracle_adjoint.py).
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sensor indices (Table 1 of the paper, f-distribution only). */
enum {
  ORC_TAU_NS = 0,  /* Eq. sensor-TauNS-kin   |P^neq|_F                          */
  ORC_C = 1,       /* Eq. sensor-C-kin       sqrt(D)|tr P^neq|/(2mu + D lambda)  */
  ORC_S = 2,       /* Eq. sensor-S-kin       |(1/mu)(tr P/D I - P)|_F            */
  ORC_E = 3,       /* Eq. sensor-E-kin       |(1/2mu)(lambda/(D eta) tr P I - P)| */
  ORC_QH = 4,      /* Eq. sensor-qH-kin      |u . P^neq|_2                       */
  ORC_KN = 5,      /* Eq. sensor-Knudsen-kin_f  sum |f^neq/f^eq|                 */
  ORC_NEQ = 6,     /* Eq. sensor-neq-kin     sum |f^neq|                         */
  ORC_QE = 7,      /* Eq. Sensor-qe-kin      sum |f* - f^eq|  (0 for BGK)        */
  ORC_HR = 8,      /* Eq. Hneq-sensor        |H(f) - H(f^eq)|                    */
  ORC_KL = 9,      /* Eq. HKL-sensor         |sum f ln(f/f^eq)|                  */
  ORC_SIGMA_H = 10,  /* Eq. Dissip-H-sensor  -sum Omega ln(f/w)                  */
  ORC_SIGMA_KL = 11, /* Eq. Dissip-HKL-sensor -sum Omega ln(f/f^eq)              */
  ORC_ALPHA = 12,  /* Eq. sensor-alpha-kin   |2 - alpha| (polynomial)            */
  ORC_NSENS = 13
};

/* Threads of the row-parallel per-cell sweeps (init, stream, collide, moments, sensor
 * fields, the sensor pass of orc_run): 1 by default.  Every cell's arithmetic is
 * independent of the split, so results are identical at any count.  Reductions
 * (flags, tile counts, sums) and the adjoint stay serial.  orc_have_openmp() is 0
 * when the library was built without OpenMP (the count then stays 1). */
void orc_set_threads(int n);
int orc_get_threads(void);
int orc_have_openmp(void);

/* Equilibrium, Grad-Hermite expansion to order N = 2 at T_ref = c_s^2 = 1/3
 * (section "Discrete kinetic model", unnumbered GH expansion). */
void orc_equilibrium(double rho, double ux, double uy, double feq[9]);

/* f := f^eq(rho, u) everywhere: "ICs supplied by equilibrium populations"
 * (section "Evaluation of the local kinetic sensors").  Fields are [ny][nx]. */
void orc_init_equilibrium(int nx, int ny, const double* rho, const double* ux,
                          const double* uy, double* f);

/* Pull streaming with periodic wrap: ft_q(i,j) = f_q(i - cx_q, j - cy_q). */
void orc_stream(int nx, int ny, const double* f, double* ft);

/* BGK collision of an already-streamed state: f' = ft - (ft - f^eq)/tau
 * (Eq. new_collision_fi with f* = f^eq, tau1 = tau2 = tau).               */
void orc_collide(int nx, int ny, double tau, const double* ft, double* fnext);

/* One full lattice step: stream then collide. */
void orc_step(int nx, int ny, double tau, const double* f, double* fnext);

/* Two-relaxation model of adaptive algorithm refinement (section "Conclusions"),
 * single-distribution D2Q9 reading: the quasi-equilibrium keeps the odd part of the
 * non-equilibrium populations, f*_i = f^eq_i + (f^neq_i - f^neq_{-i})/2, of the
 * cell's populations ft[9] (orc_quasi_equilibrium); orc_collide_aar applies Eq.
 * new_collision_fi with it (tau1, tau2) where region[ny][nx] != 0 and BGK (tau1)
 * elsewhere, to an already-streamed state. */
void orc_quasi_equilibrium(const double ft[9], double fstar[9]);
void orc_collide_aar(int nx, int ny, double tau1, double tau2, const uint8_t* region,
                     const double* ft, double* fnext);

/* Moments (Eqs. eq_quadratur1-2) of a state: rho, ux, uy fields [ny][nx]. */
void orc_moments(int nx, int ny, const double* f, double* rho, double* ux, double* uy);

/* All ORC_NSENS sensors of one cell's populations ft[9] (the pre-collision
 * state the collision acts on).  Returns 1 if any ft_q <= 0 or f^eq_q <= 0
 * (then the logarithmic sensors and the Knudsen sensor are +Inf), else 0.  */
int orc_cell_sensors(const double ft[9], double tau, double out[ORC_NSENS]);
/* The same for a given collision model: two_relax = 0 is BGK (f* = f^eq, so
 * ORC_QE = 0), two_relax = 1 the two-relaxation model (ORC_QE = sum |f* - f^eq|
 * with the quasi-equilibrium of orc_quasi_equilibrium). */
int orc_cell_sensors_model(const double ft[9], double tau, int two_relax,
                           double out[ORC_NSENS]);
/* The same, with full = 0 evaluating only ORC_KN, ORC_NEQ, ORC_QE and ORC_KL (the
 * refine/switch set of a production run) by the same lines; the other entries are
 * NaN.  full = 1 is orc_cell_sensors_model. */
int orc_cell_sensors_set(const double ft[9], double tau, int two_relax, int full,
                         double out[ORC_NSENS]);

/* The four logarithmic sensors (HR, KL, SIGMA_H, SIGMA_KL) evaluated in their
 * literal printed form, for the consistency check of the cancellation-free
 * forms used by orc_cell_sensors.  out[4] = {HR, KL, SIGMA_H, SIGMA_KL};
 * scale[4] = the rounding scale of each literal sum: sum over terms of
 * |term| + |prefactor of the logarithm|. */
void orc_cell_log_sensors_literal(const double ft[9], double tau, double out[4],
                                  double scale[4]);

/* Raw polynomial coefficients a_1..a_4 of Eq. alpha-polynomial-2 and the
 * resulting alpha of Eq. alpha-polynomial-1 (alpha := 2 when a_1 == 0). */
double orc_alpha_poly(const double ft[9], double a[4]);

/* Exact positive root alpha of H(f + alpha (f^eq - f)) = H(f) (Eq.
 * H-mirr-equal) by bisection, for diagnostics.  Returns 2 at equilibrium and
 * NaN if f is not positive. */
double orc_alpha_exact(const double ft[9]);

/* Sensor fields of a state: if pull != 0 the state is streamed first (the
 * sensors of the step that would act on it), else evaluated as stored.
 * out is [ORC_NSENS][ny][nx]; nonpos is [ny][nx] (may be NULL). */
void orc_sensor_fields(int nx, int ny, double tau, const double* f, int pull,
                       double* out, uint8_t* nonpos);
void orc_sensor_fields_model(int nx, int ny, double tau, int two_relax, const double* f,
                             int pull, double* out, uint8_t* nonpos);

/* Tagging (regrid step 1): flag bit0 = refine (eps_r > thr_r), bit1 = switch
 * (thr_s >= 0 and eps_s > thr_s), bit7 = non-positive population.  Tile counts
 * tiles[2][nty][ntx] of refine and switch flags over tile x tile blocks
 * (ragged edge tiles are partial); counts[3] = {refine, switch, nonpos}.    */
void orc_flags(int nx, int ny, const double* eps_r, double thr_r, const double* eps_s,
               double thr_s, const uint8_t* nonpos, int tile, uint8_t* flags,
               int32_t* tiles, int64_t counts[3]);

/* Conservation sums {sum rho, sum rho ux, sum rho uy} of a state (pull != 0:
 * of its streamed image, which is the same multiset of populations). */
void orc_sums(int nx, int ny, const double* f, double sums[3]);

/* Macroscopic (class-1) counterparts by second-order central differences on
 * the periodic lattice (section "Evaluation of the local kinetic sensors"):
 * out[4][ny][nx] = {eps_mac.tauNS, eps_mac.C, eps_mac.S, eps_mac.E} with
 * mu = rho c_s^2 tau, lambda = 0 (Eqs. sensor-TauNS-mac, -C-mac, -S-mac, -E-mac). */
void orc_mac_sensors(int nx, int ny, double tau, const double* rho, const double* ux,
                     const double* uy, double* out);

/* Full fused reference run (used for the CPU timing baseline): nsteps of
 * stream, the sensors (all of them, or with full = 0 the set of
 * orc_cell_sensors_set), flags on sensor_r / sensor_s, sums, collide; work is
 * scratch of the size of f and the result ends in f.  rec_field receives the
 * sensor_r field of the last step.  Returns the last step's non-positive count. */
int64_t orc_run(int nx, int ny, double tau, double* f, double* work, int nsteps,
                int sensor_r, double thr_r, int sensor_s, double thr_s, int tile,
                double* rec_field, uint8_t* flags, int32_t* tiles, int64_t counts[3],
                double sums[3], int full);

/* Discrete adjoint of the sensor objective
 *   J = sum_x W(x) eps_KL(ft(x)),  ft = stream(f^{N-1}),
 *   f^0 = f^eq(rho0, u0),  f^{n+1} = collide(stream(f^n); tau),
 * i.e. the KL sensor (Eq. HKL-sensor) of step N (its pre-collision state, as for
 * every sensor here) summed over the lattice with weights W (NULL: W = 1).
 * Outputs J, grad_rho0[ny][nx] = dJ/drho0 (u0 fixed) and grad_tau = dJ/dtau, by a
 * reverse sweep through the steps (every store_every-th state kept, the others
 * recomputed from it).  Gradients are NaN where a population is non-positive.
 * Returns 0, or -1 (nsteps < 1, store_every < 1 or no memory). */
int orc_adjoint_kl(int nx, int ny, double tau, int nsteps, int store_every, const double* rho0,
                   const double* ux0, const double* uy0, const double* weight, double* J,
                   double* grad_rho0, double* grad_tau);

/* FP16 deviation storage of populations (the library's KSS_FP16DEV form):
 *   h_q = RN16((f_q - b_q) s_q),  b_q = RN32(w_q rho0),  s_q = 2^(k_q + K)
 *   (k_q = 1, 3, 5 for w_q = 4/9, 1/9, 1/36; s_q = 1 if unscaled),
 *   decoded f_q = RN32(b_q + h_q / s_q).
 * orc_fp16_round: the nearest binary16 value (ties to even, +-Inf from 65520 up).
 * Codes h are carried as doubles holding binary16 values; arrays are [9][ny][nx]. */
double orc_fp16_round(double x);
void orc_dev16_encode(int nx, int ny, double rho0, int dev_exp, int unscaled, const double* f,
                      double* h);
void orc_dev16_decode(int nx, int ny, double rho0, int dev_exp, int unscaled, const double* h,
                      double* f);

#ifdef __cplusplus
}
#endif
#endif
