"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in a copy of
oracle/orc.c (a wrong coefficient, a flipped sign or direction, a swapped index or
operand, a dropped term, a different rounding rule), compiles it into a temporary library,
and runs one existing pin against that library: the pin must fail.  The unchanged source,
built the same way, passes the same pins (the control case).  Everything runs on the CPU.
"""
import json
import os

import pytest

import oracle
from tests import test_oracle_aar as t_aar
from tests import test_oracle_adjoint as t_adj
from tests import test_oracle_fp16dev as t_f16
from tests import test_oracle_golden as t_gold
from tests import test_oracle_lattice as t_lat
from tests import test_oracle_sensors as t_sen

SRC = os.path.join(os.path.dirname(oracle.__file__), "orc.c")


def _gold():
    with open(os.path.join(t_gold.GOLDEN, "alpha_polynomial.json")) as fh:
        return json.load(fh)


PINS = {
    "equilibrium_moments": lambda: t_lat.test_equilibrium_moments(oracle),
    "stream_by_cq": lambda: t_lat.test_stream_moves_population_q_by_cq(oracle),
    "push_scheme_8x8": lambda: t_lat.test_brute_force_push_scheme_8x8(oracle),
    "sums": lambda: t_lat.test_sums_brute_force(oracle),
    "hand_modes": lambda: t_sen.test_hand_derived_modes(oracle, 1.3, 0.6),
    "printed_log_forms": lambda: t_sen.test_log_sensors_match_printed_forms(oracle),
    "flags_tiles": lambda: t_sen.test_flags_and_tiles_brute_force(oracle),
    "fp16_numpy": lambda: t_f16.test_fp16_rounding_matches_numpy_float16(),
    "adjoint_tau_fd": lambda: t_adj.test_tau_derivative_matches_central_differences(0.8),
    "adjoint_rho_fd": lambda: t_adj.test_full_density_gradient_matches_central_differences(),
    "aar_eigenmodes": lambda: t_aar.test_relaxation_eigenmodes(oracle, 0.8, 1.3),
    "alpha_printed": lambda: t_gold.test_alpha_is_the_printed_polynomial_of_its_a_n(
        oracle, _gold(), 1e-2),
    "codec_scales": lambda: t_f16.test_codec_roundtrip_and_scales(),
    "symmetries": lambda: t_sen.test_lattice_symmetries(oracle),
}

# (planted mistake, text in orc.c, replacement, pin that must catch it)
MUTANTS = [
    ("equilibrium second-order term halved",
     "h2 / (2.0 * CS2 * CS2)", "h2 / (4.0 * CS2 * CS2)", "equilibrium_moments"),
    ("streaming pushes instead of pulls",
     "ft[at(nx, ny, q, i, j)] = f[at(nx, ny, q, wrap(i - CX[q], nx), wrap(j - CY[q], ny))];",
     "ft[at(nx, ny, q, i, j)] = f[at(nx, ny, q, wrap(i + CX[q], nx), wrap(j + CY[q], ny))];",
     "stream_by_cq"),
    ("relaxation time taken as tau - 1/2",
     "const double omega = -(c[q] - feq[q]) / tau;",
     "const double omega = -(c[q] - feq[q]) / (tau - 0.5);", "push_scheme_8x8"),
    ("x and y momenta swapped in the moments",
     "    jx += CX[q] * ft[q];\n    jy += CY[q] * ft[q];\n  }\n  *rho = r;",
     "    jx += CY[q] * ft[q];\n    jy += CX[q] * ft[q];\n  }\n  *rho = r;", "push_scheme_8x8"),
    ("Kn normalised by f instead of f^eq",
     "kn += fabs(fneq[q] / feq[q]);", "kn += fabs(fneq[q] / ft[q]);", "hand_modes"),
    ("absolute value dropped from the neq sensor",
     "neq += fabs(fneq[q]);", "neq += fneq[q];", "hand_modes"),
    ("KL weighted by f instead of f^eq",
     "kl += feq[q] * phi(x);", "kl += ft[q] * phi(x);", "printed_log_forms"),
    ("tile index transposed",
     "const int t = (j / tile) * ntx + (i / tile);",
     "const int t = (i / tile) * nty + (j / tile);", "flags_tiles"),
    ("binary16 rounding ties away from zero",
     "rint(a / quantum)", "floor(a / quantum + 0.5)", "fp16_numpy"),
    ("sign of the dtau partial flipped",
     "kahan_add(&gs, &gc, l[q] * (c[q] - feq[q]) / (tau * tau));",
     "kahan_add(&gs, &gc, -l[q] * (c[q] - feq[q]) / (tau * tau));", "adjoint_tau_fd"),
    ("1/tau dropped from the equilibrium part of the collision Jacobian",
     "lt[at(nx, ny, p, i, j)] = (1.0 - 1.0 / tau) * l[p] + s / tau;",
     "lt[at(nx, ny, p, i, j)] = (1.0 - 1.0 / tau) * l[p] + s;", "adjoint_rho_fd"),
    ("quasi-equilibrium keeps the even part instead of the odd part",
     "const double odd = 0.5 * ((ft[q] - feq[q]) - (ft[OPP[q]] - feq[OPP[q]]));",
     "const double odd = 0.5 * ((ft[q] - feq[q]) + (ft[OPP[q]] - feq[OPP[q]]));",
     "aar_eigenmodes"),
    ("tau1 and tau2 swapped in the two-relaxation collision",
     "const double omega = -(c[q] - fstar[q]) / tau1 - (fstar[q] - feq[q]) / tau2;",
     "const double omega = -(c[q] - fstar[q]) / tau2 - (fstar[q] - feq[q]) / tau1;",
     "aar_eigenmodes"),
    ("a coefficient of the entropic-estimate polynomial changed",
     "- 8.0 * a3 / a1 +", "- 4.0 * a3 / a1 +", "alpha_printed"),
    ("trace part of the S sensor not divided by D",
     "M[a][b] = ((a == b ? trP / D : 0.0) - P[a][b]) / mu;",
     "M[a][b] = ((a == b ? trP : 0.0) - P[a][b]) / mu;", "hand_modes"),
    ("factor sqrt(D) dropped from the C sensor",
     "out[ORC_C] = sqrt(D) * fabs(-trP / (2.0 * mu + D * lambda));",
     "out[ORC_C] = fabs(-trP / (2.0 * mu + D * lambda));", "hand_modes"),
    ("indices of u . P^neq swapped in the q_H sensor",
     "qh[b] += u[a] * P[a][b];", "qh[b] += u[b] * P[a][b];", "symmetries"),
    ("sigma_KL weighted by f^eq instead of f^neq",
     "sig += fneq[q] * log1p(x);", "sig += feq[q] * log1p(x);", "printed_log_forms"),
    ("sign of the linear term of HR flipped",
     "lin += fneq[q] * L;", "lin -= fneq[q] * L;", "printed_log_forms"),
    ("binary16 deviation scale of one diagonal population wrong",
     "static const int K[9] = {1, 3, 3, 3, 3, 5, 5, 5, 5};",
     "static const int K[9] = {1, 3, 3, 3, 3, 5, 5, 5, 3};", "codec_scales"),
]


def _build(tmp_path, text, name):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    return oracle.load_library(oracle.build(src=str(src), out=str(tmp_path / f"{name}.so")))


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


def test_control_unchanged_source_passes_every_pin(tmp_path, source, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _build(tmp_path, source, "control"))
    for pin in PINS.values():
        pin()


@pytest.mark.parametrize("what,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, source, monkeypatch, what, old, new, pin):
    assert source.count(old) == 1, f"the text to mutate must occur once: {old!r}"
    monkeypatch.setattr(oracle, "_lib", _build(tmp_path, source.replace(old, new), "mutant"))
    with pytest.raises(AssertionError):
        PINS[pin]()


# ---- the regrid oracle (plain Python): mutants are loaded from a mutated copy of
# oracle/regrid.py in place of the module the pins use
from tests import test_oracle_regrid as t_reg  # noqa: E402

REGRID_SRC = os.path.join(os.path.dirname(oracle.__file__), "regrid.py")

REGRID_PINS = {
    "rolled_dilation": lambda: t_reg.test_tile_mask_against_rolled_dilation(),
    "blobs": lambda: t_reg.test_empty_full_and_separated_blobs(),
    "hole_centre": lambda: t_reg.test_hole_nearest_the_centre_wins(),
    "l_shape": lambda: t_reg.test_l_shape_splits_at_the_inflection(),
}

REGRID_MUTANTS = [
    ("buffer one cell short below and left",
     "np.arange(ty * tile - buffer, min((ty + 1) * tile, ny) + buffer) % ny",
     "np.arange(ty * tile - buffer + 1, min((ty + 1) * tile, ny) + buffer) % ny",
     "rolled_dilation"),
    ("efficiency test made strict",
     "if total >= efficiency * (w * h) or (w == 1 and h == 1):",
     "if total > efficiency * (w * h) or (w == 1 and h == 1):", "hole_centre"),
    ("hole distance measured from the wrong centre",
     "return abs(2 * i - (lo + hi - 1))", "return abs(2 * i - (lo + hi - 3))", "hole_centre"),
    ("inflection test on equal signs",
     "if d[k] * d[k + 1] < 0:", "if d[k] * d[k + 1] > 0:", "l_shape"),
]


def _load_regrid(tmp_path, text, name):
    import importlib.util

    path = tmp_path / f"{name}.py"
    path.write_text(text)
    spec = importlib.util.spec_from_file_location(f"regrid_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_regrid_control_unchanged_source_passes_every_pin(tmp_path, monkeypatch):
    with open(REGRID_SRC) as fh:
        monkeypatch.setattr(t_reg, "regrid", _load_regrid(tmp_path, fh.read(), "control"))
    for pin in REGRID_PINS.values():
        pin()


@pytest.mark.parametrize("what,old,new,pin", REGRID_MUTANTS, ids=[m[0] for m in REGRID_MUTANTS])
def test_planted_regrid_mistake_is_caught(tmp_path, monkeypatch, what, old, new, pin):
    with open(REGRID_SRC) as fh:
        text = fh.read()
    assert text.count(old) == 1, f"the text to mutate must occur once: {old!r}"
    monkeypatch.setattr(t_reg, "regrid", _load_regrid(tmp_path, text.replace(old, new), "mut"))
    with pytest.raises(AssertionError):
        REGRID_PINS[pin]()
