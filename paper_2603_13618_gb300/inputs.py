"""Seeded synthetic lattice inputs (density and velocity fields, float64).

This module holds input generation only -- none of the lattice-Boltzmann or sensor
arithmetic.  It is the one piece shared by the CUDA path's tests and benchmark and
by the CPU oracle's tests: both receive the same float64 (rho, ux, uy) arrays and
build their equilibrium populations from them independently.

Workloads (all in lattice units, c_s = 1/sqrt(3)):

* ``shear_wave``: the decaying shear wave rho = 1, u_x = u0 sin(2 pi y / ny),
  u_y = 0 (128 x 128, u0 = 0.01 for the FP64 correctness case).
* ``batch_specs``: the batched workload of many uneven lattices: for lattice k,
  a square size drawn from {64, 128, 256, 512, 1024}, tau ~ U[0.51, 1.5] and a Mach
  number ~ U[0.01, 0.15], all from one SplitMix64 stream; its fields are
  ``random_smooth`` (kmax 8) scaled to that Mach number.
* ``random_region``: a prescribed two-relaxation region (random cells, nonzero bytes)
  for the adaptive-algorithm-refinement tests.
* ``smooth_jump``: a density step rho_L / rho_R = 2 at x = nx/2 (and at the
  periodic seam x = 0) times (1 + drho), with drho, u_x, u_y random smooth fields:
  sums of Fourier modes with integer wavevectors (kx, ky) in [-kmax, kmax]^2
  (not both 0), Gaussian amplitudes divided by (1 + kx^2 + ky^2) and uniform
  phases, drawn from SplitMix64 keyed on (seed, field, mode).  The fields are
  scaled so that max|drho| = drho_amp and max|u| = mach * c_s over the full
  lattice.  This stands in for the paper's Sod / 2D-Riemann discontinuities,
  which an isothermal D2Q9 lattice cannot carry at their printed ratios.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

CS = 1.0 / math.sqrt(3.0)
_M64 = (1 << 64) - 1


def splitmix64(state: int):
    """One SplitMix64 step (Steele, Lea & Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def _uniforms(seed: int, field: int, mode: int, n: int):
    st = (seed * 0x100000001B3 + field * 0x1000193 + mode * 0x9E37 + 0x2603) & _M64
    out = []
    for _ in range(n):
        st, z = splitmix64(st)
        out.append(((z >> 11) + 0.5) / float(1 << 53))  # in (0, 1)
    return out


@lru_cache(maxsize=64)
def _coeffs(seed: int, field: int, kmax: int) -> np.ndarray:
    """Complex coefficient grid C[ky + kmax, kx + kmax] of one smooth field."""
    n = 2 * kmax + 1
    c = np.zeros((n, n), dtype=np.complex128)
    mode = 0
    for ky in range(-kmax, kmax + 1):
        for kx in range(-kmax, kmax + 1):
            if kx == 0 and ky == 0:
                continue
            u1, u2, u3 = _uniforms(seed, field, mode, 3)
            g = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
            a = g / (1.0 + kx * kx + ky * ky)
            c[ky + kmax, kx + kmax] = a * complex(math.cos(2 * math.pi * u3),
                                                  math.sin(2 * math.pi * u3))
            mode += 1
    return c


def _synth(seed: int, field: int, kmax: int, nx: int, ny: int, xs, ys) -> np.ndarray:
    """Unscaled field sum_m a_m cos(2 pi (kx x / nx + ky y / ny) + phase_m) at (ys x xs)."""
    k = np.arange(-kmax, kmax + 1, dtype=np.float64)
    ex = np.exp(2j * np.pi * np.outer(k, np.asarray(xs, dtype=np.float64)) / nx)
    ey = np.exp(2j * np.pi * np.outer(np.asarray(ys, dtype=np.float64), k) / ny)
    return np.real(ey @ _coeffs(seed, field, kmax) @ ex)


@lru_cache(maxsize=16)
def _scales(nx: int, ny: int, seed: int, kmax: int, drho_amp: float, mach: float):
    """Scale factors (s_rho, s_u) that normalise the fields over the full lattice."""
    xs, ys = np.arange(nx), np.arange(ny)
    d = _synth(seed, 0, kmax, nx, ny, xs, ys)
    s_rho = drho_amp / np.max(np.abs(d))
    ux = _synth(seed, 1, kmax, nx, ny, xs, ys)
    uy = _synth(seed, 2, kmax, nx, ny, xs, ys)
    s_u = mach * CS / np.max(np.sqrt(ux * ux + uy * uy))
    return float(s_rho), float(s_u)


def smooth_jump(nx: int, ny: int, seed: int = 2603, kmax: int = 8, drho_amp: float = 1e-2,
                mach: float = 0.1, jump: float = 2.0, x0: int = 0, y0: int = 0,
                wx: int | None = None, wy: int | None = None):
    """(rho, ux, uy) [wy, wx] of the smooth-perturbation + density-step workload.

    The lattice is nx x ny (periodic); the returned window starts at global cell
    (x0, y0) and wraps periodically, so a patch around any cell can be generated
    without the full lattice (the normalisation is always the full lattice's).
    """
    wx = nx if wx is None else wx
    wy = ny if wy is None else wy
    xs = (x0 + np.arange(wx)) % nx
    ys = (y0 + np.arange(wy)) % ny
    s_rho, s_u = _scales(nx, ny, seed, kmax, drho_amp, mach)
    drho = s_rho * _synth(seed, 0, kmax, nx, ny, xs, ys)
    ux = s_u * _synth(seed, 1, kmax, nx, ny, xs, ys)
    uy = s_u * _synth(seed, 2, kmax, nx, ny, xs, ys)
    base = np.where(xs < nx // 2, jump, 1.0)[None, :]
    rho = base * (1.0 + drho)
    return (np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.ascontiguousarray(uy))


def shear_wave(nx: int = 128, ny: int = 128, u0: float = 0.01, rho0: float = 1.0):
    """(rho, ux, uy) [ny, nx] of the decaying shear wave u_x = u0 sin(2 pi y / ny)."""
    y = np.arange(ny, dtype=np.float64)[:, None]
    rho = np.full((ny, nx), rho0)
    ux = np.broadcast_to(u0 * np.sin(2.0 * np.pi * y / ny), (ny, nx)).copy()
    uy = np.zeros((ny, nx))
    return rho, ux, uy


def random_smooth(nx: int, ny: int, seed: int, kmax: int = 4, drho_amp: float = 1e-2,
                  mach: float = 0.1):
    """Smooth random fields without the density step (rho = 1 + drho)."""
    return smooth_jump(nx, ny, seed=seed, kmax=kmax, drho_amp=drho_amp, mach=mach,
                       jump=1.0)


def batch_specs(n: int = 64, seed: int = 13618, sizes=(64, 128, 256, 512, 1024),
                tau_range=(0.51, 1.5), mach_range=(0.01, 0.15)):
    """[(size, tau, mach, field_seed)] of n square periodic lattices, drawn from one
    SplitMix64 stream started at `seed` (three outputs per lattice)."""
    st = seed & _M64
    out = []
    for k in range(n):
        st, z1 = splitmix64(st)
        st, z2 = splitmix64(st)
        st, z3 = splitmix64(st)
        u2 = ((z2 >> 11) + 0.5) / float(1 << 53)
        u3 = ((z3 >> 11) + 0.5) / float(1 << 53)
        size = sizes[z1 % len(sizes)]
        tau = tau_range[0] + (tau_range[1] - tau_range[0]) * u2
        mach = mach_range[0] + (mach_range[1] - mach_range[0]) * u3
        out.append((size, tau, mach, seed * 1000 + k))
    return out


def batch_fields(size: int, mach: float, field_seed: int):
    """(rho, ux, uy) of one lattice of the batched workload."""
    return random_smooth(size, size, seed=field_seed, kmax=8, mach=mach)


def random_region(nx: int, ny: int, seed: int, frac: float = 0.4) -> np.ndarray:
    """A prescribed adaptive-algorithm-refinement region, uint8 [ny, nx]: each cell
    switched with probability frac (numpy PCG64 keyed on seed), switched cells holding
    an arbitrary nonzero byte (any nonzero byte marks a switched cell)."""
    rng = np.random.default_rng(seed)
    on = rng.random((ny, nx)) < frac
    return np.where(on, rng.integers(1, 256, size=(ny, nx)), 0).astype(np.uint8)
