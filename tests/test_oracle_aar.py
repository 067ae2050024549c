"""Pins of the oracle's adaptive-algorithm-refinement part: the two-relaxation collision
(Eq. new_collision_fi with the quasi-equilibrium f*_i = f^eq_i + (f^neq_i - f^neq_{-i})/2
in flagged cells, BGK elsewhere) and the quasi-equilibrium sensor (Eq. Sensor-qe-kin).

What fixes them independently of the oracle's code:

* limits: an empty region, or tau2 = tau1, is the BGK collision;
* relaxation eigenmodes in closed form: on a uniform lattice (streaming is the identity)
  a non-equilibrium part that is even under c -> -c decays by (1 - 1/tau1) per step, an
  odd one by (1 - 1/tau2) -- Hermite modes of D2Q9 built here from the weights;
* eps_qe of such a state is the odd part's sum of magnitudes, 0 for an even one, and 0
  for the BGK model whatever the state;
* mass and momentum are conserved over hundreds of steps;
* hydrodynamics: the shear wave decays with nu = c_s^2 (tau1 - 1/2) whatever tau2
  (tau2 relaxes only the odd, non-hydrodynamic moments);
* the region schedule of run_aar (flags of the most recent output step before the
  step) against the explicit composition of single steps.
"""
import math

import numpy as np
import pytest

from paper_2603_13618_gb300 import inputs

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0

# Hermite modes w_q H(c_q) with zero mass and momentum
EVEN = {"xy": W * CX * CY, "xx-yy": W * (CX**2 - CY**2),
        "xxyy": W * (CX**2 - CS2) * (CY**2 - CS2)}
ODD = {"xxy": W * (CX**2 - CS2) * CY, "xyy": W * CX * (CY**2 - CS2)}


def _uniform(f9, nx=5, ny=3):
    return np.broadcast_to(np.asarray(f9)[:, None, None], (9, ny, nx)).copy()


def test_modes_have_no_mass_or_momentum():
    for h in list(EVEN.values()) + list(ODD.values()):
        assert abs(h.sum()) < 1e-16
        assert abs((CX * h).sum()) < 1e-16 and abs((CY * h).sum()) < 1e-16


def test_empty_region_and_equal_times_are_bgk(orc):
    rng = np.random.default_rng(3)
    r, u, v = inputs.random_smooth(23, 17, seed=4, kmax=3, drho_amp=0.05, mach=0.15)
    ft = orc.stream(orc.step(orc.init_equilibrium(r, u, v), 0.7, 5))
    empty = np.zeros((17, 23), dtype=np.uint8)
    np.testing.assert_array_equal(orc.collide_aar(ft, 0.7, 1.9, empty), orc.collide(ft, 0.7))
    region = (rng.random((17, 23)) < 0.5).astype(np.uint8)
    np.testing.assert_allclose(orc.collide_aar(ft, 0.7, 0.7, region), orc.collide(ft, 0.7),
                               rtol=4e-16, atol=1e-17)
    # and a non-trivial region changes the result where it is set, only there
    g = orc.collide_aar(ft, 0.7, 1.9, region)
    b = orc.collide(ft, 0.7)
    same = np.all(g == b, axis=0)
    assert np.all(same[region == 0])
    assert not np.any(same[region == 1])


@pytest.mark.parametrize("tau1,tau2", [(0.8, 1.3), (0.55, 0.9), (1.7, 0.6)])
def test_relaxation_eigenmodes(orc, tau1, tau2):
    feq = orc.equilibrium(1.1, 0.05, -0.03)
    d = 1e-3
    everywhere = np.ones((3, 5), dtype=np.uint8)
    for name, h in list(EVEN.items()) + list(ODD.items()):
        f = _uniform(feq + d * h)
        g = orc.collide_aar(f, tau1, tau2, everywhere)
        factor = (1 - 1 / tau1) if name in EVEN else (1 - 1 / tau2)
        np.testing.assert_allclose(g[:, 0, 0] - feq, factor * d * h, rtol=0, atol=4e-16,
                                   err_msg=name)
        # BGK cells: every mode by (1 - 1/tau1)
        g0 = orc.collide_aar(f, tau1, tau2, 0 * everywhere)
        np.testing.assert_allclose(g0[:, 0, 0] - feq, (1 - 1 / tau1) * d * h, rtol=0,
                                   atol=4e-16, err_msg=name)
    # a mixture: each part at its own rate
    he, ho = EVEN["xy"] + 0.5 * EVEN["xxyy"], ODD["xxy"] - 2 * ODD["xyy"]
    g = orc.collide_aar(_uniform(feq + d * (he + ho)), tau1, tau2, everywhere)
    want = (1 - 1 / tau1) * d * he + (1 - 1 / tau2) * d * ho
    np.testing.assert_allclose(g[:, 0, 0] - feq, want, rtol=0, atol=4e-16)


def test_quasi_equilibrium_and_qe_sensor_closed_form(orc):
    feq = orc.equilibrium(0.9, -0.04, 0.07)
    d = 2e-3
    he, ho = EVEN["xx-yy"] - EVEN["xy"], 3 * ODD["xyy"] + ODD["xxy"]
    ft = feq + d * (he + ho)
    np.testing.assert_allclose(orc.quasi_equilibrium(ft), feq + d * ho, rtol=0, atol=2e-16)
    s_trt, _ = orc.cell_sensors(ft, 0.8, two_relax=True)
    s_bgk, _ = orc.cell_sensors(ft, 0.8)
    qe = orc.SENSOR_ID["qe"]
    assert s_trt[qe] == pytest.approx(d * np.abs(ho).sum(), rel=1e-12)
    assert s_bgk[qe] == 0.0
    s_even, _ = orc.cell_sensors(feq + d * he, 0.8, two_relax=True)
    assert s_even[qe] <= 16 * np.finfo(float).eps * ft.max()  # rounding of f - f^eq only
    # the other sensors do not depend on the model
    keep = [k for k in range(orc.NSENS) if k != qe]
    np.testing.assert_array_equal(s_trt[keep], s_bgk[keep])


def test_conservation(orc):
    nx, ny = 32, 24
    r, u, v = inputs.random_smooth(nx, ny, seed=9, kmax=4, drho_amp=0.05, mach=0.15)
    f = orc.init_equilibrium(r, u, v)
    region = (np.random.default_rng(9).random((ny, nx)) < 0.5).astype(np.uint8)
    s0 = orc.sums(f)
    eps = np.finfo(np.float64).eps
    for t in range(1, 301):
        f = orc.step_aar(f, 0.7, 1.4, region)
        if t % 50 == 0:
            s = orc.sums(f)
            bound = 4.0 * eps * t * s0[0]
            assert np.all(np.abs(s - s0) <= bound), (t, s - s0)


@pytest.mark.parametrize("tau2", [0.55, 1.3, 3.0])
def test_shear_wave_viscosity_is_set_by_tau1(orc, tau2):
    nx, ny, tau1, steps = 4, 128, 0.8, 1000
    rho, ux, uy = inputs.shear_wave(nx, ny, 0.01)
    f = orc.init_equilibrium(rho, ux, uy)
    everywhere = np.ones((ny, nx), dtype=np.uint8)
    k = 2 * math.pi / ny
    y = np.arange(ny)
    ts, amps = [], []
    fb = f.copy()
    for t in range(0, steps + 1, 50):
        if t:
            for _ in range(50):
                f = orc.step_aar(f, tau1, tau2, everywhere)
            fb = orc.step(fb, tau1, 50)
        if t >= 100:
            _, u, _ = orc.moments(f)
            ts.append(t)
            amps.append(2.0 / ny * np.sum(u.mean(axis=1) * np.sin(k * y)))
    nu = -np.polyfit(ts, np.log(amps), 1)[0] / k**2
    assert abs(nu / (CS2 * (tau1 - 0.5)) - 1.0) < 5e-3, nu
    # the model did act: the state differs from the BGK run
    assert np.max(np.abs(f - fb)) > 0


@pytest.mark.parametrize("every", [1, 2])
def test_region_schedule(orc, every):
    """run_aar against single steps composed by hand: the collision of step n uses the
    switch flags of the most recent output step before n (none before the first).  The
    switch is the quasi-equilibrium sensor of the model, as the paper suggests for AAR."""
    nx, ny, tau, tau2, n = 20, 14, 0.75, 1.6, 5
    r, u, v = inputs.random_smooth(nx, ny, seed=2, kmax=3, drho_amp=0.03, mach=0.12)
    f0 = orc.step(orc.init_equilibrium(r, u, v), tau, 3)
    thr = 7e-4
    res = orc.run_aar(f0, tau, tau2, n, output_every=every, switch=("qe", thr))
    f = f0.copy()
    region = np.zeros((ny, nx), dtype=np.uint8)
    for step in range(1, n + 1):
        ft = orc.stream(f)
        new = None
        if step % every == 0:
            sens, _ = orc.sensor_fields(ft, tau, pull=False, two_relax=True)
            new = (sens[orc.SENSOR_ID["qe"]] > thr).astype(np.uint8)
        f = orc.collide_aar(ft, tau, tau2, region)
        if new is not None:
            region = new
    assert 0 < region.sum() < nx * ny  # the threshold splits the lattice
    np.testing.assert_array_equal(res["f"], f)
    np.testing.assert_array_equal(res["region"], region)
    np.testing.assert_array_equal((res["flags"] & 2) != 0, region != 0)
