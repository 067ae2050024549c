"""Pins of the oracle against values the paper prints (fixtures under tests/golden/).

The entropic estimate (Eqs. alpha-polynomial-1/-2, section "Entropic estimate sensor"):
the oracle's alpha and its a_n against the printed coefficients, prefactors and powers,
and the alpha sensor (Eq. sensor-alpha-kin, single distribution) against |2 - alpha| of
the printed polynomial.  A changed coefficient, a dropped term, a wrong power or a wrong
sign of an a_n in the oracle fails here.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
ALPHA = 12


@pytest.fixture(scope="module")
def orc():
    import oracle

    return oracle


@pytest.fixture(scope="module")
def gold():
    with open(os.path.join(GOLDEN, "alpha_polynomial.json")) as fh:
        return json.load(fh)


def _states(orc, count, seed, amp):
    """Positive populations: a moving equilibrium with a relative perturbation of size amp
    (the state's own moments then differ from the base ones, as in a real cell)."""
    rng = np.random.default_rng(seed)
    for _ in range(count):
        rho = 1.0 + 0.05 * rng.standard_normal()
        ux, uy = 0.05 * rng.standard_normal(2)
        yield orc.equilibrium(rho, ux, uy) * (1.0 + amp * rng.standard_normal(9))


def _fneq(orc, f):
    rho = f.sum()
    feq = orc.equilibrium(rho, float(CX @ f) / rho, float(CY @ f) / rho)
    return f - feq


def _poly(gold, a):
    return sum(t["coef"] * np.prod([a[k] ** float(e) for k, e in enumerate(t["exponents"])])
               for t in gold["alpha_terms"])


@pytest.mark.parametrize("amp", [1e-2, 3e-2])
def test_a_n_follow_the_printed_prefactors_and_powers(orc, gold, amp):
    for f in _states(orc, 40, seed=int(amp * 1e4), amp=amp):
        d = _fneq(orc, f)
        _, a = orc.alpha_poly(f)
        for row in gold["a_n"]:
            want = float(Fraction(row["prefactor"])) * np.sum(
                d ** row["fneq_power"] / f ** row["f_power"])
            n = row["n"]
            assert a[n - 1] == pytest.approx(want, rel=1e-9, abs=1e-300), (n, a[n - 1], want)


@pytest.mark.parametrize("amp", [1e-2, 3e-2])
def test_alpha_is_the_printed_polynomial_of_its_a_n(orc, gold, amp):
    for f in _states(orc, 40, seed=7 + int(amp * 1e4), amp=amp):
        alpha, a = orc.alpha_poly(f)
        want = _poly(gold, a)
        # compare the departures from 2 (the constant is exact on both sides)
        assert alpha - 2.0 == pytest.approx(want - 2.0, rel=1e-9), (alpha, want)


def test_alpha_sensor_is_the_departure_of_the_printed_polynomial(orc, gold):
    for f in _states(orc, 40, seed=99, amp=2e-2):
        s, nonpos = orc.cell_sensors(f, 0.8)
        assert not nonpos
        _, a = orc.alpha_poly(f)
        assert s[ALPHA] == pytest.approx(abs(2.0 - _poly(gold, a)), rel=1e-9)


def test_equilibrium_gives_alpha_two(orc, gold):
    # (f^neq of equilibrium populations is round-off only: the moments are recomputed)
    f = orc.equilibrium(1.1, 0.03, -0.02)
    alpha, a = orc.alpha_poly(f)
    assert alpha == pytest.approx(2.0, abs=1e-12)
    assert [t["coef"] for t in gold["alpha_terms"] if not any(t["exponents"])] == [2]
