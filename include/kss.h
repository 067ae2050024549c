/*
 * kss.h -- C ABI of the GB300 (sm_103a) fused D2Q9 stream + collide + local kinetic
 * sensor library ("kinetic sensor stepping").
 *
 * The library advances a periodic D2Q9 lattice-Boltzmann lattice with the BGK
 * collision and, on output steps, evaluates in the same pass the local kinetic
 * refinement sensors of arXiv 2603.13618 ("Local kinetic sensors for adaptive mesh
 * and algorithm refinement", Table 1, single distribution) at every cell, tags the
 * cells against sensor thresholds (regrid step 1 of the SAMR cycle, and the
 * adaptive-algorithm-refinement switch of the conclusions), counts the tags per
 * tile and forms the lattice's conservation sums.
 *
 * Conventions (all entry points):
 *   - Lattice units dx = dt = 1; D2Q9 velocities
 *       c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
 *       c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1),  weights 4/9, 1/9 x4, 1/36 x4,
 *     c_s^2 = 1/3; viscosity nu = c_s^2 (tau - 1/2).
 *   - Fields are dense row-major arrays of nx*ny doubles, element (i, j) at j*nx + i
 *     (x = i, y = j).  Populations are dense [9][ny][nx] doubles.  Every array at the
 *     boundary is FP64 whatever the storage precision; conversion happens on the GPU.
 *   - on_device = 0: the pointer is host memory (pageable or pinned) owned by the
 *     caller; the call copies and synchronises before returning.  (kss_set_fields and
 *     kss_set_populations read page-locked inputs directly over the host link, without
 *     a staging copy.)
 *     on_device = 1: the pointer is CUDA device memory of the current device, owned
 *     by the caller, which must keep it valid until the lattice's stream has passed
 *     the call (reads synchronise the stream before returning).
 *   - Return value: KSS_OK (0) on success, a negative KSS_ERR_* code on error, or the
 *     positive KSS_WARN_NONPOSITIVE from the calls that evaluate sensors when a cell
 *     had a non-positive population (its flag bit 7 is set and the count reported).
 *     A CUDA error is sticky: every later call on that lattice returns
 *     KSS_ERR_CUDA; kss_last_error() gives the message.
 *   - The library owns every device buffer of a lattice (two population buffers,
 *     sensor/flag outputs, per-block scratch); kss_destroy frees them.
 *   - A lattice is used from one host thread at a time.
 */
#ifndef KSS_H
#define KSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KSS_OK 0
#define KSS_ERR_ARG (-1)         /* invalid argument (size, pointer, id, threshold)   */
#define KSS_ERR_OOM (-2)         /* device or host allocation failed                  */
#define KSS_ERR_CUDA (-3)        /* a CUDA call failed (sticky)                       */
#define KSS_ERR_TIMEOUT (-4)     /* a bounded device wait ran out                     */
#define KSS_ERR_STATE (-5)       /* call not valid in the lattice's current state     */
#define KSS_ERR_UNSUPPORTED (-6) /* precision or option not built into this library  */
#define KSS_ERR_BOUNDS (-8)      /* a device bounds check failed: only in libraries built
                                    with -DKSS_DEBUG_BOUNDS=1, where every step block checks
                                    its coordinates, rows, deferred-cell slots and tile
                                    indices and skips an access that would leave its buffer
                                    (sticky, like KSS_ERR_TIMEOUT)                        */
#define KSS_WARN_NONPOSITIVE 1   /* sensors evaluated; some cell had f_q <= 0 or f^eq_q <= 0 */

/* Storage and arithmetic precision of a lattice:
 *   KSS_FP64, KSS_FP32  populations stored and collided in that precision;
 *   KSS_FP16DEV         populations stored as FP16 deviations from the rest equilibrium
 *                       of the reference density rho0 (kss_config.rho0):
 *                         h_q = RN_fp16((f_q - b_q) s_q),  b_q = RN_fp32(w_q rho0),
 *                         s_q = 2^(k_q + dev_exp), k_q = 1, 3, 5 for w_q = 4/9, 1/9, 1/36
 *                       (s_q w_q = (8/9) 2^dev_exp for every q; dev_unscaled = 1 takes
 *                       s_q = 1, the literal deviation), decoded as
 *                       f_q = RN_fp32(b_q + h_q / s_q) and collided in FP32.  Sensor
 *                       fields are FP32.  18 bytes per cell per buffer instead of 36. */
typedef enum { KSS_FP64 = 0, KSS_FP32 = 1, KSS_FP16DEV = 2 } kss_precision;

/* Sensor ids: Table 1 of the paper, f-distribution terms only (the model has no
 * second distribution g).  mu = rho c_s^2 tau, lambda = 0, eta = mu (the D2Q9 BGK
 * first-order stress P^neq = -rho c_s^2 tau (grad u + grad u^T)).  All sensors are
 * evaluated on the post-streaming, pre-collision populations f of the step. */
typedef enum {
  KSS_S_TAU_NS = 0,   /* Eq. sensor-TauNS-kin:  |P^neq|_F, P^neq = sum c c f^neq        */
  KSS_S_C = 1,        /* Eq. sensor-C-kin:      sqrt(2) |tr P^neq| / (2 mu)             */
  KSS_S_S = 2,        /* Eq. sensor-S-kin:      |(tr P^neq / 2 I - P^neq) / mu|_F       */
  KSS_S_E = 3,        /* Eq. sensor-E-kin:      |P^neq|_F / (2 mu)   (lambda = 0)       */
  KSS_S_QH = 4,       /* Eq. sensor-qH-kin:     |u . P^neq|_2                           */
  KSS_S_KN = 5,       /* Eq. sensor-Knudsen-kin_f: sum |f^neq / f^eq| (not averaged)    */
  KSS_S_NEQ = 6,      /* Eq. sensor-neq-kin:    sum |f^neq|                             */
  KSS_S_QE = 7,       /* Eq. Sensor-qe-kin:     sum |f* - f^eq|: 0 for BGK (tau2 = 0);  */
                      /*   with tau2 > 0 the two-relaxation quasi-equilibrium (below)   */
  KSS_S_HR = 8,       /* Eq. Hneq-sensor:       |H(f) - H(f^eq)|, H = sum f ln(f/w)     */
  KSS_S_KL = 9,       /* Eq. HKL-sensor:        |sum f ln(f / f^eq)|                    */
  KSS_S_SIGMA_H = 10, /* Eq. Dissip-H-sensor:   -sum Omega ln(f/w), Omega = -f^neq/tau  */
  KSS_S_SIGMA_KL = 11,/* Eq. Dissip-HKL-sensor: -sum Omega ln(f/f^eq)                   */
  KSS_S_ALPHA = 12,   /* Eqs. sensor-alpha-kin, alpha-polynomial-1/-2: |2 - alpha|      */
  KSS_S_COUNT = 13
} kss_sensor;

/* Non-positive populations (positivity is not guaranteed by Grad-Hermite equilibria,
 * section "Overview and further considerations"): in a cell with some f_q <= 0 or
 * f^eq_q <= 0 the sensors KN, HR, KL, SIGMA_H, SIGMA_KL and ALPHA are +Inf, flag
 * bit 7 is set and the cell is counted. */

/* Flag byte of a cell. */
#define KSS_FLAG_REFINE 0x01u   /* refine sensor > refine threshold (strict)         */
#define KSS_FLAG_SWITCH 0x02u   /* switch sensor > switch threshold (strict)         */
#define KSS_FLAG_NONPOS 0x80u   /* some population or equilibrium population <= 0    */

typedef struct {
  int32_t nx, ny;            /* lattice size, 1 <= nx, ny, nx*ny <= 2^31 - 1           */
  int32_t precision;         /* kss_precision                                          */
  double tau;                /* BGK relaxation time, > 0.5                             */
  int32_t refine_sensor;     /* kss_sensor tagged against refine_threshold            */
  double refine_threshold;   /* flag bit 0: eps > threshold                           */
  int32_t switch_sensor;     /* kss_sensor tagged against switch_threshold            */
  double switch_threshold;   /* flag bit 1: eps > threshold; < 0 disables the switch  */
  uint32_t record_mask;      /* bit s set: sensor s's field is stored on output steps */
  int32_t output_every;      /* steps n with n % output_every == 0 are output steps;  */
                             /* 0 = no output steps (plain stream + collide)          */
  int32_t tile;              /* tag-count tile edge: 8, 16, 32 or 64 cells             */
  void* stream;              /* cudaStream_t to run on; NULL = the CUDA default stream */
  int32_t own_stream;        /* 1: ignore `stream`, create a non-blocking stream owned */
                             /*    by the lattice (destroyed with it)                  */
  int32_t kernel;            /* step kernel: KSS_KERNEL_AUTO, _VECTOR or _TMA          */
  double rho0;               /* KSS_FP16DEV: reference density of the deviations, > 0  */
  int32_t dev_exp;           /* KSS_FP16DEV: scale exponent K (-24 .. 40)              */
  int32_t dev_unscaled;      /* KSS_FP16DEV: 1 = literal deviations (s_q = 1)          */
  double tau2;               /* adaptive algorithm refinement: 0 = BGK everywhere; > 0.5 */
                             /*   = the two-relaxation model (tau1 = tau, tau2) in the  */
                             /*   cells of the switched region (see kss_set_aar_region) */
} kss_config;

/* Step kernels (same results; they differ in how source rows reach the SM):
 *   KSS_KERNEL_VECTOR  16-byte vector loads into registers, warp-shuffle halos;
 *   KSS_KERNEL_TMA     bulk copies (cp.async.bulk) into a per-warp shared-memory ring,
 *                      persistent CTAs; used for plain and {Kn, KL, neq} steps of FP32 and
 *                      FP64 lattices, other cases fall back to the vector kernel;
 *   KSS_KERNEL_AUTO    the faster on GB300, which is the vector kernel at every size
 *                      measured. */
#define KSS_KERNEL_AUTO 0
#define KSS_KERNEL_VECTOR 1
#define KSS_KERNEL_TMA 2

typedef struct kss_lattice kss_lattice;  /* opaque */

/* Fill *cfg with defaults for an nx x ny lattice: tau 0.8, refine on KSS_S_KN at 1e-3,
 * switch on KSS_S_NEQ at 1e-4, record KSS_S_KL, output every step, tile 16, the CUDA
 * default stream, rho0 = 1, dev_exp = 12 (relative deviations up to about 15 stay in
 * FP16 range), dev_unscaled = 0, tau2 = 0 (BGK everywhere). */
int kss_config_default(kss_config* cfg, int32_t nx, int32_t ny, int32_t precision);

/* Create a lattice (device buffers allocated; populations zero until set). */
int kss_create(const kss_config* cfg, kss_lattice** out);
/* Free a lattice and its device buffers after its stream drains (NULL-safe). */
void kss_destroy(kss_lattice* lat);

/* Equilibrium initial condition (section "Evaluation of the local kinetic sensors":
 * initial conditions are supplied as equilibrium populations): f_q := f^eq_q(rho, u)
 * with the Grad-Hermite N = 2 equilibrium of section "Discrete kinetic model".
 * rho, ux, uy: nx*ny doubles each.  Resets the step counter to 0. */
int kss_set_fields(kss_lattice* lat, const double* rho, const double* ux, const double* uy,
                   int on_device);
/* The same from FP32 fields (nx*ny floats each), for callers whose fields are single
 * precision: half the bytes of kss_set_fields to move from the host.  A field value gives
 * exactly the populations of the same value passed to kss_set_fields.  Host arrays that
 * are page-locked are read in place over the host link; others go through the lattice's
 * staging buffer.  Errors as kss_set_fields (KSS_ERR_ARG for a NULL field). */
int kss_set_fields_f32(kss_lattice* lat, const float* rho, const float* ux, const float* uy,
                       int on_device);

/* Raw populations [9][ny][nx] (checkpoint / resume and tests).  Set resets the step
 * counter to 0; get returns the stored post-collision state f^n. */
int kss_set_populations(kss_lattice* lat, const double* f, int on_device);
int kss_get_populations(kss_lattice* lat, double* f, int on_device);

/* Advance nsteps >= 0 steps: pull streaming (periodic) + BGK collision
 * f' = f - (f - f^eq)/tau (Eq. new_collision_fi with f* = f^eq), fused on output steps
 * with the sensors, tagging, tile counts and sums.  Asynchronous on the lattice's
 * stream; errors of the launches are reported here or by the next call. */
int kss_step(kss_lattice* lat, int32_t nsteps);

/* rho, ux, uy of the stored state (Eqs. eq_quadratur1-2), nx*ny doubles each. */
int kss_read_moments(kss_lattice* lat, double* rho, double* ux, double* uy, int on_device);

/* Sensor field (nx*ny doubles) of the pre-collision populations of the most recent
 * step, or of the stored populations if no step was taken since the last set.  A
 * field recorded on that step is returned as stored; any other is evaluated on
 * demand from the population buffer the step read. */
int kss_read_sensor(kss_lattice* lat, int32_t sensor, double* out, int on_device);

/* Tags of the same state as kss_read_sensor: flags (nx*ny bytes, KSS_FLAG_*),
 * tile_counts (int32 [2][nty][ntx], nty = ceil(ny/tile), ntx = ceil(nx/tile): refine
 * then switch tags per tile; ragged edge tiles are partial) and counts[3] = {refine,
 * switch, non-positive}.  Any output pointer may be NULL.  on_device applies to flags
 * and tile_counts; counts is always host memory. */
int kss_read_flags(kss_lattice* lat, uint8_t* flags, int32_t* tile_counts, int64_t counts[3],
                   int on_device);

/* Conservation sums {sum rho, sum rho ux, sum rho uy} (FP64, fixed-order reduction:
 * bitwise reproducible for a given lattice and configuration) and counts[3] of the
 * same state, and the step index it belongs to.  Host pointers; any may be NULL. */
int kss_read_stats(kss_lattice* lat, double sums[3], int64_t counts[3], int64_t* step);

/* ---- Adaptive algorithm refinement (section "Conclusions": a sensor selects the cells
 * where the single-relaxation BGK model gives way to a two-relaxation model) ----------
 * With kss_config.tau2 > 0 the lattice keeps a switched region, one byte per cell.  The
 * collision of step n is Eq. new_collision_fi with tau1 = tau and tau2 in the cells of
 * the region and BGK elsewhere; its quasi-equilibrium keeps the odd part of the
 * non-equilibrium populations,
 *   f*_q = f^eq_q + (f^neq_q - f^neq_-q)/2   (-q: the opposite velocity),
 * so tau1 relaxes the even part of f^neq (the stress: nu = c_s^2 (tau - 1/2)) and tau2
 * the odd, third-order part; density and momentum are conserved.  KSS_S_QE is then
 * sum |f* - f^eq| = sum over the four pairs of |f^neq_q - f^neq_-q|, in every cell (the
 * quasi-equilibrium is a function of the state), and can serve as the switch sensor.
 * The region in force at step n is the switch flags (KSS_FLAG_SWITCH) of the most
 * recent output step before n; an output step replaces it with its own flags.  It is
 * empty after kss_create, kss_set_fields and kss_set_populations, and
 * kss_set_aar_region replaces it (nx*ny bytes, nonzero = two-relaxation; get returns
 * 0 / 1).  KSS_ERR_STATE on a lattice with tau2 = 0.  AAR steps run on the vector
 * kernel, one launch per step; in a batch, members with tau2 > 0 take the two-
 * relaxation collision in their regions and the others step as BGK (the batch then
 * runs one launch per step, no multi-step launch).  Because an output step rewrites the
 * region, a batch with such members needs one output_every for all members
 * (KSS_ERR_UNSUPPORTED from kss_batch_create otherwise) and, when it is above 1, the
 * members in phase: kss_batch_step returns KSS_ERR_STATE if their step counts differ
 * modulo output_every (after a member was set or stepped on its own). */
int kss_set_aar_region(kss_lattice* lat, const uint8_t* region, int on_device);
int kss_get_aar_region(kss_lattice* lat, uint8_t* region, int on_device);

/* ---- Domain decomposition into y-slabs (section "Adaptive refinement and parallel
 * processing": the lattice is shared out between processes) --------------------------
 * A lattice of NX x NY cells split into slabs of whole rows, one per process or device;
 * slab r owns rows [y_r, y_r + ny_r) and is a lattice of nx = NX, ny = ny_r created by
 * kss_slab_create.  Within a slab the step is the one of kss_step, except at its two
 * faces: pull streaming reads row -1 for the populations with c_y = +1 (q = 2, 5, 6) and
 * row ny for those with c_y = -1 (q = 4, 7, 8), which are halo rows the caller fills
 * before every step instead of wrapping periodically inside the slab.  Per step:
 *   kss_slab_edges      the rows leaving the slab: to_below = q 4, 7, 8 of row 0 (they
 *                       stream into the slab below), to_above = q 2, 5, 6 of row ny - 1;
 *   kss_slab_set_halos  from_below = the slab below's to_above, from_above = the slab
 *                       above's to_below (for one slab, its own rows: periodic);
 *   kss_step(lat, 1)    one step (a slab takes one step per call: KSS_ERR_ARG otherwise).
 * Buffers hold 3 rows of nx elements in the storage type (double, float, or the binary16
 * codes of KSS_FP16DEV), q in the order given, raw so that the exchange is exact; host
 * or device memory (on_device), owned by the caller.  kss_slab_edges synchronises for
 * host buffers.  The slab's sums and counts are those of its own rows; the lattice's are
 * their sums over the slabs (an all-reduce), its flags and sensor fields the slabs'
 * rows in order, and its tile counts too when every slab but the last has a multiple of
 * tile rows.  A slab steps on the vector kernel (no TMA kernel, no multi-step launch);
 * sensors read on demand after a step use the halo rows that step read, so read them
 * before the next kss_slab_set_halos. */
int kss_slab_create(const kss_config* cfg, kss_lattice** out);
int kss_slab_edges(kss_lattice* lat, void* to_below, void* to_above, int on_device);
int kss_slab_set_halos(kss_lattice* lat, const void* from_below, const void* from_above,
                       int on_device);

/* Test support for failure detection (no counterpart in the paper).  Every device-side
 * wait of the library (the multi-step launches' dependency waits, the TMA kernel's
 * barrier waits) gives up after a deadline, sets the lattice's error word and returns,
 * so that a lost dependency ends in an error instead of a hang.  This call runs that
 * bounded wait on the lattice's stream for a device word that nothing ever sets, with a
 * deadline of deadline_cycles (1 .. 1e9 clock cycles, about 0.5 s at most): the wait
 * runs out, and the next synchronising call on the lattice returns KSS_ERR_TIMEOUT
 * (sticky, as for a real expiry).  Nothing faults; the GPU context stays usable. */
int kss_testing_expire_wait(kss_lattice* lat, int64_t deadline_cycles);
/* The same for the TMA kernel's bounded mbarrier wait: an mbarrier whose phase never
 * completes (one of two arrivals, no copy ever issued to it), waited on with a deadline of
 * deadline_cycles (1 .. 1e9); the next synchronising call returns KSS_ERR_TIMEOUT. */
int kss_testing_expire_mbarrier(kss_lattice* lat, int64_t deadline_cycles);

/* Test support: host-side fault injection (no counterpart in the paper).  kind 0: the n-th
 * device allocation of the library from now (n >= 0, 0 = the next) fails as if the device
 * were out of memory, without calling the CUDA allocator; kind 1: the n-th kss_step call
 * from now fails as if its launch had failed (KSS_ERR_CUDA, sticky on that lattice)
 * before it launches anything.  One event at a time; it disarms when it fires, and n < 0
 * disarms it.  kss_testing_live_allocations: device allocations the library holds now
 * (a failed kss_create or kss_batch_create must release everything it took).
 * Returns KSS_OK, or KSS_ERR_ARG for another kind. */
int kss_testing_fail_after(int32_t kind, int64_t n);
int64_t kss_testing_live_allocations(void);

/* Steps taken since the last set. */
int kss_get_step(const kss_lattice* lat, int64_t* step);
/* Wait for the lattice's stream; reports KSS_ERR_TIMEOUT (sticky) if a bounded device
 * wait of an earlier step ran out. */
int kss_sync(kss_lattice* lat);

/* Static description of an error code, and the last error message of a lattice. */
const char* kss_strerror(int code);
const char* kss_last_error(const kss_lattice* lat);

/* Library version (major * 10000 + minor * 100 + patch). */
int kss_version(void);

/* ---- Batches: many independent lattices advanced by one launch per step -------------
 * Under structured adaptive mesh refinement the discrete model is solved uniformly on
 * every patch of every level (section "Static refinement"): many lattices of different
 * sizes, most of them too small to fill the GPU one launch at a time.  A batch owns n lattices of any sizes and advances all
 * of them with one launch of the fused step per time step: the lattices' CTA blocks form
 * one work list.  Each member gives exactly the results it would give alone with the
 * same CTA height (populations, sensors, flags, tile counts and counts bit for bit; the
 * conservation sums too when its CTA height is its default one).
 *
 * Members are ordinary kss_lattice handles (set fields, read outputs, even step one
 * alone); kss_destroy on a member does nothing, kss_batch_destroy frees them all.
 * All members share one precision and one stream (those of cfgs[0]; the batch's own
 * non-blocking stream if cfgs[0].own_stream).  Batched steps always use the vector
 * kernel.  A batched step is an output step (each member's own sensor set, flags, tile
 * counts and sums) for every member when it is one for any member by its own
 * output_every; the populations do not depend on which steps are output steps. */
typedef struct kss_batch kss_batch;  /* opaque */

typedef struct {
  int32_t rows;         /* CTA height in rows: 16, 32 or 64, a multiple of every member's */
                        /* tile; 0 = 32 (the single-lattice default; 64 with a tile of 64) */
  int32_t ctas_per_sm;  /* 0: one CTA per work item; k > 0: k CTAs per SM, each striding */
                        /* over the work items (persistent)                              */
  int32_t graph;        /* 1: kss_batch_step captures its launches once per (step count, */
                        /* output pattern) as a CUDA graph and replays it               */
  double ms_per_step;   /* kss_batch_autotune: measured time of one output step of the  */
                        /* whole batch with this choice; ignored by kss_batch_set_tuning */
  int32_t multi_step;   /* 1 (default): a kss_batch_step(n >= 2) call whose steps are all */
                        /* {Kn, KL, neq} output steps runs as ONE cooperative launch: each */
                        /* block of a step waits (bounded, KSS_ERR_TIMEOUT) only for its  */
                        /* lattice's neighbouring blocks of the previous step; same results */
                        /* bit for bit; ctas_per_sm and graph then do not apply            */
} kss_batch_tuning;

/* Create n >= 1 lattices from cfgs[0..n-1] (each validated as by kss_create).  Members
 * start with zero populations, like kss_create. */
int kss_batch_create(int32_t n, const kss_config* cfgs, kss_batch** out);
/* Free the batch and all its members after the stream drains (NULL-safe). */
void kss_batch_destroy(kss_batch* b);
/* Member k (0 <= k < n), owned by the batch; NULL if k is out of range. */
kss_lattice* kss_batch_member(kss_batch* b, int32_t k);
/* Advance every member nsteps >= 0 steps: one launch per step, or all of them in one
 * launch (kss_batch_tuning.multi_step); asynchronous on the batch's stream.  Returns a
 * member's sticky error if one has any; a bounded wait of a multi-step launch that ran
 * out shows as KSS_ERR_TIMEOUT on the members' next synchronising call. */
int kss_batch_step(kss_batch* b, int32_t nsteps);
/* Current work decomposition, and a new one (validated; KSS_ERR_ARG if rows is not a
 * multiple of every member's tile). */
int kss_batch_get_tuning(const kss_batch* b, kss_batch_tuning* t);
int kss_batch_set_tuning(kss_batch* b, const kss_batch_tuning* t);
/* Choose rows and ctas_per_sm by timing `steps` output steps of every candidate on the
 * members themselves, or take the choice from cache_path (a text file, one line per
 * key "device name|SMs|precision|log2 cells|log2 lattices"; NULL = no file) when it
 * holds one for this batch's key; a new measurement is appended to the file.  The timed
 * launches read each member's stored state and write its other buffer, so every member
 * must be at step 0 (just created or set): KSS_ERR_STATE otherwise.  The members' stored
 * states are unchanged; their outputs are evaluated again on the next read.  The choice
 * is applied (graph as before) and returned in *chosen (may be NULL). */
int kss_batch_autotune(kss_batch* b, const char* cache_path, int32_t steps,
                       kss_batch_tuning* chosen);
/* Last error message of the batch's own calls. */
const char* kss_batch_last_error(const kss_batch* b);

/* ---- Regridding on the flags: tile tagging and clustering into patches -----------------
 * Steps (1)-(2) of the regridding routine (section "Adaptive refinement and parallel
 * processing"): cells tagged by the refine sensor, a buffer of `buffer` cells around them
 * (the applications use 2, section "Application to adaptive mesh refinement"), and a
 * clustering of the tagged region into rectangular patches with a grid-efficiency
 * threshold (0.98 in the 2-D application).  Here the tagging tiles are the unit: a tile
 * is marked when a refine-flagged cell lies within `buffer` cells of it (periodic), and
 * the marked tiles are clustered by the signature method of Berger & Rigoutsos (the
 * clustering the paper cites), breadth first:
 *   1. signatures: marked tiles per column and per row of the box;
 *   2. an empty box is dropped, any other shrunk to the bounding box of its marks;
 *   3. accepted if marks >= efficiency * area, or if it is a single tile;
 *   4. else cut at the interior hole (zero signature) nearest the centre (x before y,
 *      lower index first on ties), the hole row / column in neither half;
 *   5. else at the strongest sign change of the signature Laplacian
 *      s[i-1] - 2 s[i] + s[i+1] (ties: nearest the centre, x before y, lower index);
 *   6. else the longer side (x if equal) is halved.
 * Boxes are reported level by level in list order (children lower half first): the
 * result is a deterministic function of the flags.  Boxes do not wrap the periodic seam.
 * Box coordinates are in tiles, half-open: cells [x0*tile, min(x1*tile, nx)). */
typedef struct {
  int32_t x0, y0, x1, y1;
} kss_box;

/* On the lattice's flags of its current step (evaluated first if that step had no
 * outputs).  tile_mask: [nty][ntx] bytes or NULL; boxes: up to max_boxes boxes or NULL;
 * *nboxes: the number of boxes (may exceed max_boxes: only max_boxes are written).
 * on_device applies to tile_mask and boxes.  buffer in [0, 1024], efficiency in [0, 1];
 * the tile grid is at most 8192 tiles per side (KSS_ERR_UNSUPPORTED beyond). */
int kss_regrid(kss_lattice* lat, int32_t buffer, double efficiency, uint8_t* tile_mask,
               kss_box* boxes, int32_t max_boxes, int32_t* nboxes, int on_device);

/* The same on caller flags (dense [ny][nx] bytes, bit 0 = refine), host or device by
 * on_device, on `stream` (NULL = the default stream); allocates its workspace per call. */
int kss_regrid_flags(const uint8_t* flags, int32_t nx, int32_t ny, int32_t tile, int32_t buffer,
                     double efficiency, uint8_t* tile_mask, kss_box* boxes, int32_t max_boxes,
                     int32_t* nboxes, int on_device, void* stream);

/* ---- Adjoint: gradients of a sensor objective -----------------------------------------
 * Gradient of the sensor-weighted objective
 *   J = sum_x W(x) eps_KL(x)    (Eq. HKL-sensor, the KL sensor of step nsteps, i.e. of
 *                                the pre-collision populations that step N acts on)
 * of a periodic lattice started from equilibrium populations f^eq(rho0, u0) (section
 * "Evaluation of the local kinetic sensors": equilibrium initial conditions), with
 * respect to the initial density field rho0 (u0 held fixed) and the relaxation time
 * tau, by the discrete adjoint of the stream + collide steps (reverse mode through the
 * exact discrete map; see adjoint_kernel.cuh).  The forward pass keeps every
 * checkpoint_every-th state; the backward pass recomputes each segment from its
 * checkpoint and runs the adjoint steps through it, so memory is
 * (nsteps / checkpoint_every + checkpoint_every + 4) population buffers.
 * The sensor-tuning use of such gradients is the data-driven outlook of the
 * conclusions ("Summary and conclusions"). */
typedef struct kss_adjoint kss_adjoint;  /* opaque */

typedef struct {
  int32_t nx, ny;            /* lattice size (as kss_config)                         */
  int32_t precision;         /* KSS_FP32 or KSS_FP64: storage and arithmetic         */
  int32_t nsteps;            /* N >= 1: J is evaluated on the sensors of step N      */
  int32_t checkpoint_every;  /* >= 1; states kept every this many steps              */
  void* stream;              /* cudaStream_t, NULL = the default stream              */
  int32_t own_stream;        /* 1: a stream created and owned by the object          */
} kss_adjoint_config;

int kss_adjoint_create(const kss_adjoint_config* cfg, kss_adjoint** out);
void kss_adjoint_destroy(kss_adjoint* adj);  /* NULL-safe */

/* Forward pass: rho0, ux0, uy0 (nx*ny doubles each) and the weights W (nx*ny doubles,
 * NULL = all 1), host or device memory by on_device; tau > 0.5.  Writes J (host) and
 * keeps the checkpoints for kss_adjoint_backward.  J is +Inf if some population or
 * equilibrium population of step N is non-positive. */
int kss_adjoint_forward(kss_adjoint* adj, const double* rho0, const double* ux0,
                        const double* uy0, const double* weight, double tau, int on_device,
                        double* J);

/* Backward pass of the last forward pass (once per forward pass): grad_rho0 = dJ/drho0
 * (nx*ny doubles, host or device by on_device; may be NULL) and *grad_tau = dJ/dtau
 * (host; may be NULL).  KSS_ERR_STATE without a forward pass since the last backward. */
int kss_adjoint_backward(kss_adjoint* adj, double* grad_rho0, double* grad_tau, int on_device);

const char* kss_adjoint_last_error(const kss_adjoint* adj);
/* How the reverse sweep runs (no counterpart in the paper): on = 1 (the default) takes
 * each segment's reverse steps in one cooperative launch whose blocks wait only on their
 * neighbours' previous step (bounded waits: KSS_ERR_TIMEOUT from kss_adjoint_backward if
 * one runs out); on = 0 one launch per reverse step.  The gradients are the same bit for
 * bit.  KSS_ERR_ARG for another value. */
int kss_adjoint_set_multistep(kss_adjoint* adj, int on);

/* ---- Allocation-free fused step (no counterpart in the paper) ----------------------
 * For callers that cannot call cudaMalloc: code that owns all device memory itself
 * (a pool or framework allocator whose buffers it hands in), or that must not allocate
 * while it runs.  One FP32 fused step -- pull streaming, BGK collision, the Kn / KL /
 * neq sensors, flags, tile counts and conservation sums, the same kernel as kss_step
 * with the {Kn, KL, neq} sensor set -- on buffers the caller provides.  The kernel's
 * scratch (per-CTA partial sums and counts, a CTA completion counter) lives in a fixed
 * array with static storage in this library's device code, of about 640 KiB, which
 * every GPU that loads the library holds until the process exits.  The call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Buffers (device memory of the current device, owned by the caller):
 *   f_in, f_out   populations [9][ny][pitch] floats, 16-byte aligned; the step reads
 *                 f_in and writes f_out, and the two ranges must not overlap (an
 *                 overlap, an in-place call included, is KSS_ERR_ARG); pitch >= nx, a
 *                 multiple of 32
 *   sensor_out    the record_sensor field [ny][pitch] floats (16-byte aligned), or NULL
 *   flags         [ny][pitch] bytes (KSS_FLAG_*), 4-byte aligned
 *   tile_counts   int32 [2][ceil(ny/tile)][ceil(nx/tile)] (refine, switch)
 *   sums, counts  double[3] {sum rho, sum rho ux, sum rho uy} and uint64[3]
 *                 {refine, switch, non-positive}
 * refine_sensor, switch_sensor and record_sensor must be KSS_S_KN, KSS_S_KL or
 * KSS_S_NEQ; switch_threshold < 0 disables the switch flag; tile is 8, 16, 32 or 64.
 * Asynchronous on `stream` (NULL = the default stream).
 *
 * Limit: the launch has ceil(nx/128) * ceil(ny/R) CTAs (R = 32 rows, 64 for tile 64) and
 * the scratch holds KSS_NOALLOC_MAX_BLOCKS of them (4096 x 4096 uses 4096, 8192 x 8192
 * uses 16384); larger problems are rejected with KSS_ERR_NOALLOC_CAPACITY before
 * anything is launched.
 * The first call on each device looks up the device address of the scratch array
 * (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture.  Every call shares the scratch array, which keeps the last call's
 * contents (the call clears the counter it needs at zero): calls that overlap on the GPU,
 * on any stream, race and give wrong sums and counts.
 * Returns KSS_OK, KSS_ERR_ARG, KSS_ERR_NOALLOC_CAPACITY or KSS_ERR_CUDA. */
#define KSS_NOALLOC_MAX_BLOCKS 16384
#define KSS_ERR_NOALLOC_CAPACITY (-7)
int kss_step_f32_noalloc(const float* f_in, float* f_out, int32_t nx, int32_t ny, int32_t pitch,
                         double tau, int32_t refine_sensor, double refine_threshold,
                         int32_t switch_sensor, double switch_threshold, int32_t tile,
                         int32_t record_sensor, float* sensor_out, uint8_t* flags,
                         int32_t* tile_counts, double* sums, unsigned long long* counts,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KSS_H */
