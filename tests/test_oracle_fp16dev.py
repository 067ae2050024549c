"""Pins of the oracle's FP16 deviation codec: its binary16 rounding against numpy's
float16 conversion (round to nearest, ties to even), and the codec's identities."""
import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs


def test_fp16_rounding_matches_numpy_float16():
    rng = np.random.default_rng(3)
    xs = np.concatenate([
        rng.standard_normal(4000) * 10.0 ** rng.integers(-9, 5, 4000),  # all binades
        rng.uniform(-70000, 70000, 500),                                  # overflow edge
        np.float16(rng.standard_normal(500)).astype(np.float64),          # exact values
    ])
    # exact midpoints between neighbouring binary16 values (ties to even)
    h = np.float16(rng.uniform(-1000, 1000, 500))
    nxt = np.nextafter(h, np.float16(np.inf))
    mids = (h.astype(np.float64) + nxt.astype(np.float64)) / 2
    # subnormal midpoints and the overflow threshold
    sub = (np.arange(1, 60) + 0.5) * 2.0 ** -24
    special = np.array([65504.0, 65519.999, 65520.0, -65520.0, 2.0 ** -25, 3 * 2.0 ** -26,
                        2.0 ** -14, 0.0])
    for x in np.concatenate([xs, mids, sub, -sub, special]):
        with np.errstate(over="ignore"):
            want = float(np.float16(x))
        got = oracle.fp16_round(x)
        assert got == want or (np.isinf(want) and got == want), (x, got, want)


def test_codec_roundtrip_and_scales():
    r, u, v = inputs.random_smooth(24, 16, seed=4, kmax=3, drho_amp=0.02, mach=0.1)
    f = oracle.init_equilibrium(r, u, v)
    for K in (0, 8, 12, 16):
        h = oracle.dev16_encode(f, rho0=1.0, dev_exp=K)
        # codes are binary16 values
        np.testing.assert_array_equal(h, np.float16(h).astype(np.float64))
        g = oracle.dev16_decode(h, rho0=1.0, dev_exp=K)
        # values are binary32 values
        np.testing.assert_array_equal(g, g.astype(np.float32).astype(np.float64))
        # error: half a binary16 quantum of the code, plus one binary32 rounding
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        s = 2.0 ** (np.array([1, 3, 3, 3, 3, 5, 5, 5, 5]) + K)
        e16 = np.maximum(np.floor(np.log2(np.maximum(np.abs(h), 2.0 ** -14))), -14)
        quantum = 2.0 ** (e16 - 10) / s[:, None, None]
        bound = 0.5 * quantum + 2.0 ** -24 * np.abs(f)
        assert np.all(np.abs(g - f) <= bound * (1 + 1e-12))
        # s_q w_q = (8/9) 2^K for every q
        np.testing.assert_allclose(s * w, (8 / 9) * 2.0 ** K, rtol=0, atol=0)
    # the rest state of the reference density (b_q = RN32(w_q rho0)) codes to zero
    b = np.float32(np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4) * 1.3).astype(np.float64)
    rest = np.broadcast_to(b[:, None, None], (9, 3, 2)).copy()
    np.testing.assert_array_equal(oracle.dev16_encode(rest, rho0=1.3, dev_exp=12), 0.0 * rest)


def test_unscaled_form_loses_small_deviations_to_subnormals():
    """The codes' own error, h/s - (f - b): with s_q = 2^(k_q + K) every deviation keeps
    binary16's relative precision 2^-11; unscaled (s_q = 1), deviations below 2^-14
    (6.1e-5) are subnormal binary16 values with a fixed spacing of 2^-24."""
    r, u, v = inputs.random_smooth(24, 16, seed=5, kmax=3, drho_amp=1e-3, mach=1e-3 * 3 ** 0.5)
    f = oracle.init_equilibrium(r, u, v)
    b = np.float32(np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)).astype(np.float64)
    dev = f - b[:, None, None]
    s = 2.0 ** (np.array([1, 3, 3, 3, 3, 5, 5, 5, 5]) + 20)
    hu = oracle.dev16_encode(f, dev_exp=0, unscaled=True)
    hs = oracle.dev16_encode(f, dev_exp=20)
    eu = np.abs(hu - dev)
    es = np.abs(hs / s[:, None, None] - dev)
    small = np.abs(dev) < 2.0 ** -14
    assert np.mean(small) > 0.5
    assert np.all(es <= 2.0 ** -11 * np.abs(dev))
    assert np.all(eu <= 2.0 ** -25 + 2.0 ** -11 * np.abs(dev))
    rel_u = eu[small] / np.abs(dev[small])
    assert np.max(rel_u) > 2.0 ** -8  # far coarser than 2^-11
