"""Pins of the oracle's discrete adjoint (oracle.adjoint_kl) against what fixes it
independently: central finite differences of the objective computed by plain forward
steps and the sensor fields (oracle.objective_kl, which shares no code with the
reverse sweep), invariances, and special cases.

Objective: J = sum_x W(x) eps_KL(x) of step N (the KL sensor, Eq. HKL-sensor, on the
pre-collision populations of step N), as a function of the initial density rho0 (the
initial populations are f^eq(rho0, u0), u0 fixed) and of tau.
"""
import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs


def _fields(nx, ny, seed, mach=0.1, drho=0.05):
    return inputs.random_smooth(nx, ny, seed=seed, kmax=2, drho_amp=drho, mach=mach)


def _fd(fun, x, h):
    return (fun(x + h) - fun(x - h)) / (2 * h)


def test_full_density_gradient_matches_central_differences():
    nx, ny, tau, N = 8, 6, 0.8, 5
    r, u, v = _fields(nx, ny, seed=1)
    J, g, _ = oracle.adjoint_kl(r, u, v, tau, N)
    assert J == pytest.approx(oracle.objective_kl(r, u, v, tau, N), rel=1e-13)
    h = 1e-6
    fd = np.empty_like(g)
    for j in range(ny):
        for i in range(nx):
            e = np.zeros_like(r)
            e[j, i] = 1.0
            fd[j, i] = _fd(lambda t: oracle.objective_kl(r + t * e, u, v, tau, N), 0.0, h)
    scale = np.max(np.abs(g))
    assert scale > 0
    assert np.max(np.abs(g - fd)) <= 1e-6 * scale


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.4])
def test_tau_derivative_matches_central_differences(tau):
    r, u, v = _fields(10, 7, seed=2)
    N = 6
    _, _, gt = oracle.adjoint_kl(r, u, v, tau, N)
    fd = _fd(lambda t: oracle.objective_kl(r, u, v, t, N), tau, 1e-6)
    assert gt == pytest.approx(fd, rel=1e-6)


def test_weighted_objective_and_one_step():
    """N = 1: J depends on rho0 through the initial equilibrium and one streaming only
    (no collision in the chain); random weights W."""
    nx, ny, tau = 7, 9, 0.7
    r, u, v = _fields(nx, ny, seed=3, mach=0.15)
    w = np.random.default_rng(5).uniform(0.2, 2.0, size=(ny, nx))
    for N in (1, 4):
        J, g, gt = oracle.adjoint_kl(r, u, v, tau, N, weight=w)
        assert J == pytest.approx(oracle.objective_kl(r, u, v, tau, N, weight=w), rel=1e-13)
        d = np.random.default_rng(6).standard_normal((ny, nx))
        fd = _fd(lambda t: oracle.objective_kl(r + t * d, u, v, tau, N, weight=w), 0.0, 1e-6)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6)
        if N == 1:
            assert gt == 0.0  # no collision acts before the sensor of step 1


def test_segmented_recomputation_is_exact():
    r, u, v = _fields(12, 10, seed=4)
    ref = oracle.adjoint_kl(r, u, v, 0.9, 11, store_every=1)
    for se in (2, 3, 5, 10, 11, 20):
        J, g, gt = oracle.adjoint_kl(r, u, v, 0.9, 11, store_every=se)
        assert J == ref[0] and gt == ref[2]
        np.testing.assert_array_equal(g, ref[1])


def test_periodic_shift_moves_the_gradient():
    r, u, v = _fields(9, 8, seed=7)
    J, g, gt = oracle.adjoint_kl(r, u, v, 0.75, 6)
    sh = lambda a: np.roll(np.roll(a, 3, axis=1), -2, axis=0)
    J2, g2, gt2 = oracle.adjoint_kl(sh(r), sh(u), sh(v), 0.75, 6)
    assert J2 == pytest.approx(J, rel=1e-12) and gt2 == pytest.approx(gt, rel=1e-10)
    np.testing.assert_allclose(g2, sh(g), rtol=1e-10, atol=1e-12 * np.max(np.abs(g)))


def test_uniform_state_has_zero_objective_and_gradient():
    """A uniform state is a fixed point at equilibrium: eps_KL = 0 everywhere at every
    step, a minimum of J (J >= 0), so every derivative vanishes."""
    ny, nx = 6, 5
    r = np.full((ny, nx), 1.3)
    u = np.full((ny, nx), 0.04)
    v = np.full((ny, nx), -0.02)
    J, g, gt = oracle.adjoint_kl(r, u, v, 0.8, 7)
    assert J <= 1e-20
    assert np.max(np.abs(g)) <= 1e-15 and abs(gt) <= 1e-15


def test_directional_derivative_larger_lattice_richardson():
    """32 x 24 lattice, 15 steps: <grad J, d> against central differences at h and h/2
    (their Richardson combination removes the O(h^2) term)."""
    nx, ny, tau, N = 32, 24, 0.6, 15
    r, u, v = _fields(nx, ny, seed=8, mach=0.1, drho=0.02)
    J, g, gt = oracle.adjoint_kl(r, u, v, tau, N, store_every=4)
    d = np.random.default_rng(9).standard_normal((ny, nx))
    f = lambda t: oracle.objective_kl(r + t * d, u, v, tau, N)
    h = 1e-4
    d1, d2 = _fd(f, 0.0, h), _fd(f, 0.0, h / 2)
    rich = (4 * d2 - d1) / 3
    assert np.sum(g * d) == pytest.approx(rich, rel=1e-7)
