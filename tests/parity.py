"""Tolerances and comparison helpers of the GPU-vs-oracle parity tests.

Tolerance model (derived from the arithmetic; u = unit round-off of the storage type,
2^-24 for FP32 and 2^-53 for FP64, n = steps taken):

* populations / moments: the state drifts from the oracle's by independent rounding
  of the collision each step, a few u relative per step, as a random walk:
  |df| <= c u sqrt(n + 1) f.  FP64 uses c = 64; FP32 moments must meet the stated
  1e-5 after 100 steps.
* sensors: each f^neq_q = f_q - f^eq_q carries an absolute error of a few u f_q (the
  rounding of f^eq, and of an FP32 initial state) plus the state drift, which a
  sensor's definition carries to its value in proportion to the natural scale of its
  terms (sensor_scale): Kn sums 9 terms |x_q| whose errors are ~u; KL and sigma_KL sum
  x_q f^neq_q (~u neq, ~2 u neq / tau); neq and tau_ns sum ~u f_q (~u rho); C, S, E divide
  by mu (3 / tau); q_H and the linear term of HR and sigma_H carry |u| (rho |u|).  The
  floor is c(n) u scale_s with c(n) = C_EVAL + C_DRIFT sqrt(n + 1), on top of a relative
  tolerance (FP64 1e-10, FP32 1e-3).  C_EVAL and C_DRIFT were set from the measured
  errors of every comparison of the GPU suite (REPORT; the largest coefficient any
  sensor needed was 9.3 at n = 100 and 5.4 at n <= 7, against c(n) = 18 ... 36).
* alpha: when the pre-collision state ft is known, the floor is instead a first-order
  propagation of those input errors through the printed polynomial (alpha_error): its
  ratios r_n = a_n / a_1 amplify the errors of the sums a_n, and the polynomial
  |4 r2 - 16 r2^2 + 8 r3 - 80 r2 r3 + 80 r2^3 + 16 r4| cancels far from equilibrium.
* flags: identical except at cells whose oracle sensor lies within 1e-4 of the
  threshold (absolute band); tile counts and global counts are then compared as
  exact integers after removing the band cells' contributions.
"""
from __future__ import annotations

import math

import numpy as np

SENSORS = ("tau_ns", "c", "s", "e", "qh", "kn", "neq", "qe", "hr", "kl", "sigma_h",
           "sigma_kl", "alpha")
UNIT_ROUNDOFF = {"fp64": 2.0**-53, "fp32": 2.0**-24}
RTOL = {"fp64": 1e-10, "fp32": 1e-3}
FLAG_BAND = 1e-4


def alpha_error(ft, prec, nsteps):
    """First-order bound on the rounding error of the entropic estimate |2 - alpha| of
    the pre-collision populations ft [9, ny, nx] (FP64), in the storage precision.

    Input errors: f^neq_q = f_q - f^eq_q with |d f^neq_q| <= 8 u (|f_q| + |f^eq_q|) s,
    |d f_q| <= u |f_q| s, s = sqrt(n + 1) (the state drift); each term
    t_nq = f^neq_q^(n+1) / f_q^n then carries
    (n+1) |y_q|^n |d f^neq_q| + n |t_nq| |d f_q| / |f_q| + 2n u |t_nq|, y_q = f^neq_q / f_q,
    a_n = c_n sum_q t_nq adds 9 u sum_q |t_nq|, r_n = a_n / a_1 carries
    (|d a_n| + |r_n| |d a_1|) / |a_1|, and the polynomial
    |dP/dr2| |d r2| + |dP/dr3| |d r3| + 16 |d r4| plus 8 u times its terms' magnitudes."""
    u = UNIT_ROUNDOFF[prec]
    sdrift = math.sqrt(nsteps + 1)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)[:, None, None]
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)[:, None, None]
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    with np.errstate(all="ignore"):
        rho = ft.sum(axis=0)
        ux = (cx * ft).sum(axis=0) / rho
        uy = (cy * ft).sum(axis=0) / rho
        cu = cx * ux + cy * uy
        feq = w * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))
        fneq = ft - feq
        y = fneq / ft
        dfneq = 8 * u * (np.abs(ft) + np.abs(feq)) * sdrift
        df = u * np.abs(ft) * sdrift
        c = {1: 0.5, 2: -1 / 6, 3: 1 / 12, 4: -1 / 20}
        a, da = {}, {}
        for n in (1, 2, 3, 4):
            t = fneq ** (n + 1) / ft ** n
            dt = ((n + 1) * np.abs(y) ** n * dfneq + n * np.abs(t) * df / np.abs(ft)
                  + 2 * n * u * np.abs(t))
            a[n] = c[n] * t.sum(axis=0)
            da[n] = abs(c[n]) * (dt.sum(axis=0) + 9 * u * np.abs(t).sum(axis=0))
        r = {n: a[n] / a[1] for n in (2, 3, 4)}
        dr = {n: (da[n] + np.abs(r[n]) * da[1]) / np.abs(a[1]) + u * np.abs(r[n])
              for n in (2, 3, 4)}
        r2, r3, r4 = r[2], r[3], r[4]
        terms = (np.abs(4 * r2) + 16 * r2 * r2 + np.abs(8 * r3) + np.abs(80 * r2 * r3)
                 + np.abs(80 * r2 ** 3) + np.abs(16 * r4))
        err = (np.abs(4 - 32 * r2 - 80 * r3 + 240 * r2 * r2) * dr[2]
               + np.abs(8 - 80 * r2) * dr[3] + 16 * dr[4] + 8 * u * terms)
    return np.where(np.isfinite(err), err, 0.0)


# Error floor of the sensors: atol = c(n) u scale_s with c(n) = C_EVAL + C_DRIFT sqrt(n + 1).
# C_EVAL covers the rounding of one evaluation (f^eq_q and f^neq_q carry a few u f^eq_q;
# an FP32 initial state rounds every population once), C_DRIFT the random walk of the
# state's rounding over n collisions.  The constants are set from the measured errors
# (REPORT below records, for every comparison, the c that it needed).
C_EVAL = {"fp64": 16.0, "fp32": 16.0}
C_DRIFT = {"fp64": 2.0, "fp32": 2.0}

# Every comparison adds a record here: the largest error and the floor coefficient c the
# cells needed beyond the relative tolerance (tests/conftest.py prints a summary).
REPORT = []


def neq_field(ft):
    """sum_q |f^neq_q| of the populations ft [9, ny, nx] (FP64), the natural scale of
    the KL-type sensors: their terms are x_q f^neq_q with x_q = f^neq_q / f^eq_q."""
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)[:, None, None]
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)[:, None, None]
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    with np.errstate(all="ignore"):
        rho = ft.sum(axis=0)
        ux = (cx * ft).sum(axis=0) / rho
        uy = (cy * ft).sum(axis=0) / rho
        cu = cx * ux + cy * uy
        feq = w * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))
        out = np.abs(ft - feq).sum(axis=0)
    return np.where(np.isfinite(out), out, 0.0)


def sensor_scale(name, rho, ux, uy, kn, tau, neq=None, two_relax=False):
    """Natural scale of each sensor's rounding error, per cell (a first-order propagation
    of an error of order u f_q in every f^neq_q through the sensor's definition):
        tau_ns, neq: sum_q f_q = rho     C, S, E: rho / mu = 3 / tau     qh: rho |u|
        Kn: 9 terms |x_q| with |dx_q| ~ u     KL, sigma_KL: sum |x_q| f^eq_q u ~ neq u
        HR, sigma_H: the linear term sum f^neq L_q (L_q ~ 3 c.u) adds rho |u|
        sigma_KL, sigma_H: d(f^neq ln(1 + x)) ~ 2 x d f^neq, so 2 neq / tau
        alpha: 1     qe: 0 for BGK, rho for the two-relaxation model."""
    speed = np.sqrt(ux * ux + uy * uy)
    if neq is None:  # no populations at hand: f^eq_q <= rho / 2 bounds neq by rho Kn / 2
        neq = 0.5 * rho * np.where(np.isfinite(kn), kn, 0.0)
    return {
        "tau_ns": rho, "neq": rho, "c": 3.0 / tau + 0 * rho, "s": 3.0 / tau + 0 * rho,
        "e": 3.0 / tau + 0 * rho, "qh": rho * speed, "kn": 9.0 + 0 * rho, "kl": neq,
        "hr": rho * speed + neq, "sigma_h": (rho * speed + 2.0 * neq) / tau,
        "sigma_kl": 2.0 * neq / tau, "alpha": 1.0 + 0 * rho,
        "qe": rho if two_relax else 0 * rho,
    }[name]


def floor_coefficient(prec, nsteps):
    return C_EVAL[prec] + C_DRIFT[prec] * math.sqrt(nsteps + 1)


def sensor_atol(name, prec, nsteps, rho, ux, uy, kn, tau, two_relax=False, neq=None):
    u = UNIT_ROUNDOFF[prec]
    scale = sensor_scale(name, rho, ux, uy, kn, tau, neq, two_relax)
    return floor_coefficient(prec, nsteps) * u * scale


def sensor_tolerance(name, want, prec, nsteps, rho, ux, uy, kn, tau, ft=None,
                     two_relax=False, neq=None):
    """The per-cell tolerance |got - want| <= tol that assert_sensor_close applies."""
    w = np.where(np.isinf(want), 0.0, want)
    if neq is None and ft is not None:
        neq = neq_field(ft)
    scale = sensor_scale(name, rho, ux, uy, kn, tau, neq, two_relax)
    atol = floor_coefficient(prec, nsteps) * UNIT_ROUNDOFF[prec] * scale
    if name == "alpha" and ft is not None:
        atol = np.maximum(atol, 4.0 * alpha_error(ft, prec, nsteps))
    return RTOL[prec] * np.abs(w) + atol


def assert_sensor_close(name, got, want, prec, nsteps, rho, ux, uy, kn, tau, ft=None,
                        two_relax=False, neq=None, where=""):
    both_inf = np.isinf(got) & np.isinf(want)
    assert np.array_equal(np.isinf(got), np.isinf(want)), f"{name}: +Inf pattern differs"
    g, w = np.where(both_inf, 0.0, got), np.where(both_inf, 0.0, want)
    if neq is None and ft is not None:
        neq = neq_field(ft)
    u = UNIT_ROUNDOFF[prec]
    scale = sensor_scale(name, rho, ux, uy, kn, tau, neq, two_relax)
    atol = floor_coefficient(prec, nsteps) * u * scale
    if name == "alpha" and ft is not None:
        atol = np.maximum(atol, 4.0 * alpha_error(ft, prec, nsteps))
    tol = RTOL[prec] * np.abs(w) + atol
    err = np.abs(g - w)
    with np.errstate(all="ignore"):
        beyond = np.maximum(err - RTOL[prec] * np.abs(w), 0.0)
        need = np.where(scale > 0, beyond / (u * scale), np.where(beyond > 0, np.inf, 0.0))
    if name != "alpha":
        with np.errstate(all="ignore"):
            large = np.abs(w) >= 1e3 * floor_coefficient(prec, nsteps) * u * scale
            rel_large = float(np.max(np.where(large, err / np.abs(w), 0.0), initial=0.0))
        with np.errstate(all="ignore"):
            ratio = np.where(tol > 0, err / tol, np.where(err > 0, np.inf, 0.0))
        alt = {}
        for rt in (1e-4, 2e-4, 5e-4):
            with np.errstate(all="ignore"):
                b = np.maximum(err - rt * np.abs(w), 0.0)
                nd = np.where(scale > 0, b / (u * scale), np.where(b > 0, np.inf, 0.0))
            alt[str(rt)] = float(np.max(nd, initial=0.0))
        REPORT.append({"sensor": name, "prec": prec, "nsteps": int(nsteps), "where": where,
                       "c_needed_at_rtol": alt,
                       "cells": int(err.size), "max_err": float(np.max(err, initial=0.0)),
                       "max_tol_ratio": float(np.max(ratio, initial=0.0)),
                       "c_needed": float(np.max(need, initial=0.0)),
                       "c_floor": floor_coefficient(prec, nsteps),
                       "rel_err_large_values": rel_large})
    bad = err > tol
    assert not bad.any(), (f"{name} ({prec}): {int(bad.sum())} cells out of tolerance, "
                           f"worst err {err.max():.3e} vs tol {tol[np.unravel_index(err.argmax(), err.shape)]:.3e}")
    return float(np.max(err / np.maximum(np.abs(w), 1e-300), initial=0.0))


def band_mask(eps_r, thr_r, eps_s, thr_s):
    m = np.abs(eps_r - thr_r) <= FLAG_BAND
    if thr_s >= 0:
        m |= np.abs(eps_s - thr_s) <= FLAG_BAND
    return m


def assert_flags_match(flags, tiles, counts, ref_flags, ref_tiles, ref_counts, band, tile):
    """Flags identical outside the threshold band; counts exact up to the band cells."""
    diff = (flags != ref_flags) & ~band
    assert not diff.any(), f"{int(diff.sum())} flags differ outside the threshold band"
    nb = int(band.sum())
    if nb == 0:
        np.testing.assert_array_equal(tiles, ref_tiles)
        np.testing.assert_array_equal(counts, ref_counts)
        return 0
    # every tile count differs from the oracle's by at most its band cells
    ny, nx = flags.shape
    nty, ntx = tiles.shape[1:]
    bt = np.zeros((nty, ntx), dtype=np.int64)
    jj, ii = np.nonzero(band)
    np.add.at(bt, (jj // tile, ii // tile), 1)
    assert np.all(np.abs(tiles[0] - ref_tiles[0]) <= bt)
    assert np.all(np.abs(tiles[1] - ref_tiles[1]) <= bt)
    # and equals the recount of the GPU's own flags exactly
    ty = np.repeat((np.arange(ny) // tile)[:, None], nx, axis=1)
    tx = np.repeat((np.arange(nx) // tile)[None, :], ny, axis=0)
    rc = np.zeros((2, nty, ntx), dtype=np.int64)
    np.add.at(rc[0], (ty, tx), (flags & 1).astype(np.int64))
    np.add.at(rc[1], (ty, tx), ((flags >> 1) & 1).astype(np.int64))
    np.testing.assert_array_equal(tiles, rc)
    assert counts[0] == int(np.sum(flags & 1)) and counts[1] == int(np.sum((flags >> 1) & 1))
    assert counts[2] == int(np.sum(flags >> 7))
    return nb
