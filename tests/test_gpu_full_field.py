"""The headline workload compared in full: every cell of the 4096^2 FP32 lattice, in the
benchmark's launch configuration, against the FP64 oracle run on the whole lattice.

Workload and launch: 4096^2 periodic, smooth perturbations on the 2:1 density step (seed
2603), Kn refine 1e-3, neq switch 1e-4, output every step, 16 x 16 tiles, the library's
automatic kernel choice.  At this size the library takes 64-row CTAs; kss_step(1) is one
launch of the fused step kernel and kss_step(2) one cooperative two-step launch of the
multi-step kernel (the benchmark's timed kernel).  After 1 and 2 steps from
kss_set_fields: populations, moments, the Kn, KL and neq fields of the last step, flags,
tile counts, counts and the conservation sums, at tau = 0.6 (the benchmark's) and 1.0.
The comparison helpers then get planted mistakes in host copies of the GPU's results
(never in the kernel) and must reject them.

The oracle runs its row sweeps on all host cores (bit-identical to one thread).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

N = 4096
THR_R, THR_S, TILE = 1e-3, 1e-4, 16
U32 = parity.UNIT_ROUNDOFF["fp32"]


@pytest.fixture(scope="module")
def kss():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_13618_gb300 import kss

    kss.load()
    return kss


@pytest.fixture(scope="module")
def threads():
    n = oracle.set_threads(oracle.host_cores())
    yield n
    oracle.set_threads(1)


@pytest.fixture(scope="module")
def fields():
    return inputs.smooth_jump(N, N, seed=2603, kmax=8)


def _planted_sensor_errors_are_caught(name, got, want, args, rng):
    """Errors of 1.5 times the cell's own tolerance, at five cells of a host copy of the
    GPU's field, fail the comparison (in either direction)."""
    tol = parity.sensor_tolerance(name, want, *args)
    finite = np.flatnonzero(np.isfinite(want))
    for sign in (1.0, -1.0):
        bad = got.copy()
        idx = rng.choice(finite, 5, replace=False)
        bad.flat[idx] = want.flat[idx] + sign * 1.5 * tol.flat[idx]
        with pytest.raises(AssertionError):
            parity.assert_sensor_close(name, bad, want, *args)
    parity.REPORT.pop()  # (the planted comparisons recorded themselves; drop them)
    parity.REPORT.pop()


@pytest.mark.parametrize("tau", [0.6, 1.0])
def test_every_cell_after_one_and_two_steps(kss, threads, fields, tau):
    rho, ux, uy = fields
    rng = np.random.default_rng(int(tau * 1000))
    f_prev = oracle.init_equilibrium(rho, ux, uy)
    for nsteps in (1, 2):
        if nsteps == 2:
            f_prev = oracle.step(f_prev, tau)
        lat = kss.Lattice(N, N, precision="fp32", tau=tau, refine_sensor="kn",
                          refine_threshold=THR_R, switch_sensor="neq",
                          switch_threshold=THR_S, record=("kl", "kn", "neq"),
                          output_every=1, tile=TILE)
        lat.set_fields(rho, ux, uy)
        lat.step(nsteps)
        got_f = lat.get_populations()
        got_m = lat.read_moments()
        got_s = {s: lat.read_sensor(s) for s in ("kn", "kl", "neq")}
        flags, tiles, counts = lat.read_flags()
        sums, counts2, step = lat.read_stats()
        lat.close()
        assert step == nsteps
        np.testing.assert_array_equal(counts2, counts)

        # oracle: sensors of the step (pre-collision state), then the step itself
        sens, nonpos = oracle.sensor_fields(f_prev, tau, pull=True)
        ft = oracle.stream(f_prev)
        r, u, v = oracle.moments(ft)
        fin = oracle.collide(ft, tau)
        where = f"4096^2 tau {tau} after {nsteps}"

        # populations and moments: every cell
        rel = np.abs(got_f - fin) / fin
        parity.REPORT.append({"sensor": "populations", "prec": "fp32", "nsteps": nsteps,
                              "where": where, "cells": int(rel.size),
                              "max_err": float(rel.max()),
                              "max_tol_ratio": float(rel.max() / (64 * U32 * math.sqrt(nsteps + 1))),
                              "c_needed": float(rel.max() / U32), "c_floor": 64 * math.sqrt(nsteps + 1),
                              "rel_err_large_values": float(rel.max())})
        assert rel.max() <= 64 * U32 * math.sqrt(nsteps + 1), rel.max()
        rr, ru, rv = oracle.moments(fin)
        assert np.max(np.abs(got_m[0] - rr) / rr) <= 1e-5
        umax = 0.1 / math.sqrt(3.0)
        assert np.max(np.abs(got_m[1] - ru)) <= 1e-5 * umax
        assert np.max(np.abs(got_m[2] - rv)) <= 1e-5 * umax
        del got_f, fin, rel

        # the three sensor fields of the step: every cell
        kn_ref = sens[oracle.SENSOR_ID["kn"]]
        neq = parity.neq_field(ft)
        for name, field in got_s.items():
            want = sens[oracle.SENSOR_ID[name]]
            args = ("fp32", nsteps, r, u, v, kn_ref, tau)
            parity.assert_sensor_close(name, field, want, *args, neq=neq, where=where)
            _planted_sensor_errors_are_caught(name, field, want, args + (None, False, neq), rng)

        # flags outside the 1e-4 band, tile counts and counts: every cell and tile
        es = sens[oracle.SENSOR_ID["neq"]]
        rf, rt, rc = oracle.flags(kn_ref, THR_R, es, THR_S, nonpos, TILE)
        band = parity.band_mask(kn_ref, THR_R, es, THR_S)
        parity.assert_flags_match(flags, tiles, counts, rf, rt, rc, band, TILE)
        assert 0 < counts[0] < N * N and 0 < counts[1] < N * N  # both flags take both values
        # planted: one flag flipped outside the band, one tile count off by one
        jj, ii = np.nonzero(~band)
        k = rng.integers(len(jj))
        bad = flags.copy()
        bad[jj[k], ii[k]] ^= 1
        with pytest.raises(AssertionError):
            parity.assert_flags_match(bad, tiles, counts, rf, rt, rc, band, TILE)
        bad_t = tiles.copy()
        bad_t[0, rng.integers(tiles.shape[1]), rng.integers(tiles.shape[2])] += 1
        with pytest.raises(AssertionError):
            parity.assert_flags_match(flags, bad_t, counts, rf, rt, rc, band, TILE)

        # conservation sums of the step's pre-collision state: the FP32 state differs from
        # the oracle's by at most a few roundings per population per step (worst case,
        # linear in the steps); the summation itself is exact to double-float precision
        want = oracle.sums(ft)
        tol = 8 * U32 * (nsteps + 1) * want[0]
        parity.REPORT.append({"sensor": "sums", "prec": "fp32", "nsteps": nsteps,
                              "where": where, "cells": 3,
                              "max_err": float(np.max(np.abs(sums - want))),
                              "max_tol_ratio": float(np.max(np.abs(sums - want)) / tol),
                              "c_needed": float(np.max(np.abs(sums - want)) / (U32 * want[0])),
                              "c_floor": 8 * (nsteps + 1), "rel_err_large_values": 0.0})
        assert np.all(np.abs(sums - want) <= tol), (sums, want)
