"""Pins of the oracle's lattice part (stream, equilibrium, collide, sums) against what
the paper and the mathematics fix -- never against the oracle itself.

* equilibrium moments of the Grad-Hermite N = 2 expansion (section "Discrete kinetic
  model"): rho, rho u and the second moment rho c_s^2 I + rho u u are reproduced
  exactly by the quadrature (Eqs. eq_quadratur1-2);
* the uniform rest state is a fixed point of stream + collide;
* streaming is a pure permutation that moves population q by c_q;
* brute force on 8 x 8: an independent push-scheme, array-of-structures step with
  an explicit neighbour table gives the same states;
* conservation of mass and momentum (Eqs. eq_con_fstar1-2) over 2000 steps;
* hydrodynamics: the decaying shear wave has nu = c_s^2 (tau - 1/2).
"""
import math

import numpy as np
import pytest

from paper_2603_13618_gb300 import inputs

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def test_equilibrium_moments(orc):
    rng = np.random.default_rng(7)
    for _ in range(50):
        rho = rng.uniform(0.5, 2.0)
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        feq = orc.equilibrium(rho, ux, uy)
        assert abs(feq.sum() - rho) <= 1e-14 * rho
        assert abs((CX * feq).sum() - rho * ux) <= 1e-15
        assert abs((CY * feq).sum() - rho * uy) <= 1e-15
        # second moment of the N = 2 Hermite equilibrium: rho c_s^2 I + rho u u
        cs2 = 1.0 / 3.0
        pxx, pxy, pyy = (CX * CX * feq).sum(), (CX * CY * feq).sum(), (CY * CY * feq).sum()
        assert abs(pxx - (rho * cs2 + rho * ux * ux)) <= 1e-14
        assert abs(pyy - (rho * cs2 + rho * uy * uy)) <= 1e-14
        assert abs(pxy - rho * ux * uy) <= 1e-15
        assert np.all(feq > 0)


def test_rest_state_is_fixed_point(orc):
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rho0 = 1.25
    f = np.broadcast_to((w * rho0)[:, None, None], (9, 6, 10)).copy()
    feq = orc.equilibrium(rho0, 0.0, 0.0)
    np.testing.assert_array_equal(feq, w * rho0)
    g = orc.step(f, 0.7, nsteps=3)
    np.testing.assert_array_equal(g, f)


def test_stream_moves_population_q_by_cq(orc):
    nx, ny = 7, 5
    for q in range(9):
        f = np.zeros((9, ny, nx))
        f[q, 2, 3] = 1.0
        ft = orc.stream(f)
        want = np.zeros_like(f)
        want[q, (2 + CY[q]) % ny, (3 + CX[q]) % nx] = 1.0
        np.testing.assert_array_equal(ft, want)
    # a permutation of every plane: sorted values unchanged, with wrap
    rng = np.random.default_rng(3)
    f = rng.random((9, ny, nx))
    ft = orc.stream(f)
    for q in range(9):
        np.testing.assert_array_equal(np.sort(ft[q].ravel()), np.sort(f[q].ravel()))


# ---- brute force: push scheme on an array of structures, explicit neighbour table ----

def _push_collide(cells, tau):
    """Collide every cell of an AoS lattice cells[j][i][q] (plain Python)."""
    w = [4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36]
    out = []
    for row in cells:
        orow = []
        for f in row:
            rho = sum(f)
            ux = sum(CX[q] * f[q] for q in range(9)) / rho
            uy = sum(CY[q] * f[q] for q in range(9)) / rho
            usq = ux * ux + uy * uy
            g = []
            for q in range(9):
                cu = CX[q] * ux + CY[q] * uy
                feq = w[q] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq)
                g.append(f[q] + (feq - f[q]) / tau)
            orow.append(g)
        out.append(orow)
    return out


def _push_stream(cells):
    ny, nx = len(cells), len(cells[0])
    nbr = {(i, j, q): ((i + CX[q]) % nx, (j + CY[q]) % ny)
           for j in range(ny) for i in range(nx) for q in range(9)}
    out = [[[0.0] * 9 for _ in range(nx)] for _ in range(ny)]
    for j in range(ny):
        for i in range(nx):
            for q in range(9):
                ti, tj = nbr[(i, j, q)]
                out[tj][ti][q] = cells[j][i][q]
    return out


def test_brute_force_push_scheme_8x8(orc):
    nx = ny = 8
    tau = 0.63
    rng = np.random.default_rng(11)
    f0 = orc.init_equilibrium(1.0 + 0.05 * rng.standard_normal((ny, nx)),
                              0.05 * rng.standard_normal((ny, nx)),
                              0.05 * rng.standard_normal((ny, nx)))
    f0 = f0 * (1.0 + 0.02 * rng.standard_normal(f0.shape))  # leave equilibrium
    n = 6
    # pull: f_n = (C S)^n f0 ;  push: (S C)^(n-1) acting on S f0, then one more C
    pull = orc.step(f0, tau, nsteps=n)
    cells = [[list(f0[:, j, i]) for i in range(nx)] for j in range(ny)]
    cells = _push_stream(cells)
    for _ in range(n - 1):
        cells = _push_stream(_push_collide(cells, tau))
    cells = _push_collide(cells, tau)
    push = np.array(cells).transpose(2, 0, 1)
    np.testing.assert_allclose(pull, push, rtol=1e-14, atol=1e-16)


# ---- shear wave: conservation and nu = c_s^2 (tau - 1/2) ----

@pytest.fixture(scope="module")
def shear_run(orc):
    nx = ny = 128
    tau = 0.8
    rho, ux, uy = inputs.shear_wave(nx, ny, 0.01)
    f = orc.init_equilibrium(rho, ux, uy)
    snaps = {0: f}
    for t in range(50, 2001, 50):
        f = orc.step(f, tau, nsteps=50)
        snaps[t] = f
    return {"tau": tau, "nx": nx, "ny": ny, "snaps": snaps}


def test_conservation_2000_steps(orc, shear_run):
    """Mass and momentum are collision invariants (Eqs. eq_con_fstar1-2) and streaming
    is a permutation, so the totals change by round-off only: at most a few ulps of
    each cell's density per step (the bound is linear in t because the shear wave is
    uniform along x, so the rounding of its 128 columns is coherent)."""
    s0 = orc.sums(shear_run["snaps"][0])
    eps = np.finfo(np.float64).eps
    for t, f in shear_run["snaps"].items():
        s = orc.sums(f)
        bound = 4.0 * eps * max(t, 1) * s0[0]
        assert abs(s[0] - s0[0]) <= bound, t
        assert abs(s[1] - s0[1]) <= bound, t
        assert abs(s[2] - s0[2]) <= bound, t
    # and far below the physical scale after the full run
    assert abs(orc.sums(shear_run["snaps"][2000])[0] / s0[0] - 1.0) < 1e-12


def test_shear_wave_viscosity(orc, shear_run):
    ny, tau = shear_run["ny"], shear_run["tau"]
    k = 2 * math.pi / ny
    y = np.arange(ny)
    ts, amps = [], []
    for t, f in sorted(shear_run["snaps"].items()):
        _, ux, _ = orc.moments(f)
        a = 2.0 / ny * np.sum(ux.mean(axis=1) * np.sin(k * y))
        if t >= 100:
            ts.append(t)
            amps.append(a)
    slope = np.polyfit(ts, np.log(amps), 1)[0]
    nu = -slope / k**2
    nu_theory = (tau - 0.5) / 3.0
    assert abs(nu / nu_theory - 1.0) < 5e-3, (nu, nu_theory)
    # closed-form amplitude ratio over the whole run: A(2000)/A(0) = exp(-nu k^2 2000)
    _, ux0, _ = orc.moments(shear_run["snaps"][0])
    _, ux1, _ = orc.moments(shear_run["snaps"][2000])
    r = np.sum(ux1.mean(axis=1) * np.sin(k * y)) / np.sum(ux0.mean(axis=1) * np.sin(k * y))
    assert abs(r / math.exp(-nu_theory * k * k * 2000) - 1.0) < 5e-3


def test_sums_brute_force(orc):
    rng = np.random.default_rng(5)
    f = rng.random((9, 13, 17))
    s = orc.sums(f)
    np.testing.assert_allclose(s, [f.sum(), (CX[:, None, None] * f).sum(),
                                   (CY[:, None, None] * f).sum()], rtol=1e-13, atol=1e-13)


def test_row_parallel_sweeps_are_bitwise_serial(orc):
    """The oracle's per-cell sweeps split over threads give the single-thread results bit
    for bit (no arithmetic depends on the split; reductions stay serial)."""
    rho, ux, uy = inputs.smooth_jump(96, 70, seed=61, kmax=6)
    out = []
    for th in (1, 4):
        orc.set_threads(th)
        try:
            f = orc.init_equilibrium(rho, ux, uy)
            g = orc.step(f, 0.7, 3)
            s, n = orc.sensor_fields(g, 0.7, pull=True)
            m = orc.moments(g)
            run = orc.run(g, 0.7, 2, orc.SENSOR_ID["kn"], 1e-3,
                             orc.SENSOR_ID["neq"], 1e-4, 16)
        finally:
            orc.set_threads(1)
        out.append((f, g, s, n, *m, run))
    for a, b in zip(*out):
        if isinstance(a, dict):
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
        else:
            np.testing.assert_array_equal(a, b)
