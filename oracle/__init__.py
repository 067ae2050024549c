"""Plain FP64 CPU oracle for the fused D2Q9 stream + collide + kinetic-sensor step.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The oracle is the
C library ``orc.c`` (plain scalar double-precision loops, one function per definition
of arXiv 2603.13618), loaded here with ctypes; it shares no code with the CUDA
library in ``paper_2603_13618_gb300``.

Arrays are numpy float64: populations ``f[9, ny, nx]``, fields ``[ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")

NSENS = 13
SENSOR_NAMES = ("tau_ns", "c", "s", "e", "qh", "kn", "neq", "qe", "hr", "kl",
                "sigma_h", "sigma_kl", "alpha")
SENSOR_ID = {n: k for k, n in enumerate(SENSOR_NAMES)}


def build(verbose: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile orc.c (or another copy of it, `src`) into _build/liborc.so (or `out`) with
    gcc (plain -O2, no fast-math)."""
    out = out or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    src = src or os.path.join(_HERE, "orc.c")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-Wall", "-Wextra", "-I", _HERE, "-o", out, src, "-lm"]
    # the row-parallel sweeps use OpenMP where the compiler has it (one thread unless
    # set_threads asks for more); without it the same source builds serial
    omp = cmd[:-1] + ["-fopenmp", "-lm"]
    if verbose:
        print(" ".join(omp))
    if subprocess.run(omp, capture_output=True).returncode != 0:
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
    return out


_lib = None


def load_library(path: str) -> ctypes.CDLL:
    """A compiled oracle library at `path`, with the ctypes signatures of its functions."""
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    ci, cd = ctypes.c_int, ctypes.c_double
    sig = {
        "orc_equilibrium": (None, [cd, cd, cd, dp]),
        "orc_init_equilibrium": (None, [ci, ci, dp, dp, dp, dp]),
        "orc_stream": (None, [ci, ci, dp, dp]),
        "orc_collide": (None, [ci, ci, cd, dp, dp]),
        "orc_step": (None, [ci, ci, cd, dp, dp]),
        "orc_moments": (None, [ci, ci, dp, dp, dp, dp]),
        "orc_cell_sensors": (ci, [dp, cd, dp]),
        "orc_cell_sensors_model": (ci, [dp, cd, ci, dp]),
        "orc_quasi_equilibrium": (None, [dp, dp]),
        "orc_collide_aar": (None, [ci, ci, cd, cd, u8p, dp, dp]),
        "orc_sensor_fields_model": (None, [ci, ci, cd, ci, dp, ci, dp, u8p]),
        "orc_cell_log_sensors_literal": (None, [dp, cd, dp, dp]),
        "orc_alpha_poly": (cd, [dp, dp]),
        "orc_alpha_exact": (cd, [dp]),
        "orc_sensor_fields": (None, [ci, ci, cd, dp, ci, dp, u8p]),
        "orc_flags": (None, [ci, ci, dp, cd, dp, cd, u8p, ci, u8p, i32p, i64p]),
        "orc_sums": (None, [ci, ci, dp, dp]),
        "orc_mac_sensors": (None, [ci, ci, cd, dp, dp, dp, dp]),
        "orc_run": (ctypes.c_int64, [ci, ci, cd, dp, dp, ci, ci, cd, ci, cd, ci,
                                      dp, u8p, i32p, i64p, dp, ci]),
        "orc_cell_sensors_set": (ci, [dp, cd, ci, ci, dp]),
        "orc_adjoint_kl": (ci, [ci, ci, cd, ci, ci, dp, dp, dp, dp, dp, dp, dp]),
        "orc_fp16_round": (cd, [cd]),
        "orc_dev16_encode": (None, [ci, ci, cd, ci, ci, dp, dp]),
        "orc_dev16_decode": (None, [ci, ci, cd, ci, ci, dp, dp]),
        "orc_set_threads": (None, [ci]),
        "orc_get_threads": (ci, []),
        "orc_have_openmp": (ci, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        src = os.path.join(_HERE, "orc.c")
        if (not os.path.exists(_LIB_PATH)
                or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src)):
            build()
        _lib = load_library(_LIB_PATH)
    return _lib


def _p(a: np.ndarray, ct=ctypes.c_double):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> int:
    """Split the row sweeps of later calls over n threads (1 = the serial oracle; results
    are the same bit for bit at any count).  Returns the count in force, which stays 1
    when the library was built without OpenMP."""
    L = lib()
    L.orc_set_threads(int(n) if L.orc_have_openmp() else 1)
    return L.orc_get_threads()


def get_threads() -> int:
    return lib().orc_get_threads()


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.empty(9)
    lib().orc_equilibrium(rho, ux, uy, _p(out))
    return out


def init_equilibrium(rho, ux, uy) -> np.ndarray:
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    ny, nx = rho.shape
    f = np.empty((9, ny, nx))
    lib().orc_init_equilibrium(nx, ny, _p(rho), _p(ux), _p(uy), _p(f))
    return f


def stream(f) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    lib().orc_stream(f.shape[2], f.shape[1], _p(f), _p(out))
    return out


def collide(ft, tau: float) -> np.ndarray:
    ft = _f64(ft)
    out = np.empty_like(ft)
    lib().orc_collide(ft.shape[2], ft.shape[1], tau, _p(ft), _p(out))
    return out


def step(f, tau: float, nsteps: int = 1) -> np.ndarray:
    f = _f64(f).copy()
    g = np.empty_like(f)
    for _ in range(nsteps):
        lib().orc_step(f.shape[2], f.shape[1], tau, _p(f), _p(g))
        f, g = g, f
    return f


def moments(f):
    f = _f64(f)
    ny, nx = f.shape[1:]
    rho, ux, uy = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
    lib().orc_moments(nx, ny, _p(f), _p(rho), _p(ux), _p(uy))
    return rho, ux, uy


def cell_sensors(ft, tau: float, two_relax: bool = False, full: bool = True):
    """All sensors of one cell's populations ft[9]; two_relax: the collision model is
    the two-relaxation one (its quasi-equilibrium enters eps_qe), else BGK.  full=False:
    only Kn, neq, qe and KL (the others NaN)."""
    ft = _f64(ft)
    out = np.empty(NSENS)
    if full:
        nonpos = lib().orc_cell_sensors_model(_p(ft), tau, int(two_relax), _p(out))
    else:
        nonpos = lib().orc_cell_sensors_set(_p(ft), tau, int(two_relax), 0, _p(out))
    return out, bool(nonpos)


def quasi_equilibrium(ft) -> np.ndarray:
    """f* of the two-relaxation model for one cell's populations ft[9] (orc.h)."""
    ft = _f64(ft)
    out = np.empty(9)
    lib().orc_quasi_equilibrium(_p(ft), _p(out))
    return out


def collide_aar(ft, tau1: float, tau2: float, region) -> np.ndarray:
    """Eq. new_collision_fi with the two-relaxation quasi-equilibrium where region != 0,
    BGK elsewhere, of an already-streamed state ft[9, ny, nx]."""
    ft = _f64(ft)
    region = np.ascontiguousarray(region, dtype=np.uint8)
    assert region.shape == ft.shape[1:]
    out = np.empty_like(ft)
    lib().orc_collide_aar(ft.shape[2], ft.shape[1], tau1, tau2, _p(region, ctypes.c_uint8),
                          _p(ft), _p(out))
    return out


def step_aar(f, tau1: float, tau2: float, region) -> np.ndarray:
    """One step (pull streaming, then collide_aar)."""
    return collide_aar(stream(f), tau1, tau2, region)


def cell_log_sensors_literal(ft, tau: float):
    ft = _f64(ft)
    out, scale = np.empty(4), np.empty(4)
    lib().orc_cell_log_sensors_literal(_p(ft), tau, _p(out), _p(scale))
    return out, scale


def alpha_poly(ft):
    ft = _f64(ft)
    a = np.empty(4)
    alpha = lib().orc_alpha_poly(_p(ft), _p(a))
    return alpha, a


def alpha_exact(ft) -> float:
    return lib().orc_alpha_exact(_p(_f64(ft)))


def sensor_fields(f, tau: float, pull: bool = True, two_relax: bool = False):
    """All sensors of the state (streamed first when pull=True): ([13, ny, nx], nonpos).
    two_relax: eps_qe of the two-relaxation model (else of BGK, identically 0)."""
    f = _f64(f)
    ny, nx = f.shape[1:]
    out = np.empty((NSENS, ny, nx))
    nonpos = np.empty((ny, nx), dtype=np.uint8)
    lib().orc_sensor_fields_model(nx, ny, tau, int(two_relax), _p(f), int(pull), _p(out),
                                  _p(nonpos, ctypes.c_uint8))
    return out, nonpos


def flags(eps_r, thr_r: float, eps_s, thr_s: float, nonpos, tile: int):
    eps_r, eps_s = _f64(eps_r), _f64(eps_s)
    nonpos = np.ascontiguousarray(nonpos, dtype=np.uint8)
    ny, nx = eps_r.shape
    ntx, nty = -(-nx // tile), -(-ny // tile)
    fl = np.empty((ny, nx), dtype=np.uint8)
    tiles = np.empty((2, nty, ntx), dtype=np.int32)
    counts = np.empty(3, dtype=np.int64)
    lib().orc_flags(nx, ny, _p(eps_r), thr_r, _p(eps_s), thr_s,
                    _p(nonpos, ctypes.c_uint8), tile, _p(fl, ctypes.c_uint8),
                    _p(tiles, ctypes.c_int32), _p(counts, ctypes.c_int64))
    return fl, tiles, counts


def sums(f) -> np.ndarray:
    f = _f64(f)
    out = np.empty(3)
    lib().orc_sums(f.shape[2], f.shape[1], _p(f), _p(out))
    return out


def mac_sensors(rho, ux, uy, tau: float) -> np.ndarray:
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    ny, nx = rho.shape
    out = np.empty((4, ny, nx))
    lib().orc_mac_sensors(nx, ny, tau, _p(rho), _p(ux), _p(uy), _p(out))
    return out


def run(f, tau: float, nsteps: int, sensor_r: int, thr_r: float, sensor_s: int,
        thr_s: float, tile: int = 16, full: bool = True):
    """nsteps fused reference steps in place on a copy of f; returns a dict.  full=False
    evaluates only the {Kn, KL, neq} set (flags on one of them)."""
    f = _f64(f).copy()
    ny, nx = f.shape[1:]
    work = np.empty_like(f)
    rec = np.empty((ny, nx))
    fl = np.empty((ny, nx), dtype=np.uint8)
    ntx, nty = -(-nx // tile), -(-ny // tile)
    tiles = np.empty((2, nty, ntx), dtype=np.int32)
    counts = np.empty(3, dtype=np.int64)
    sm = np.empty(3)
    lib().orc_run(nx, ny, tau, _p(f), _p(work), nsteps, sensor_r, thr_r, sensor_s,
                  thr_s, tile, _p(rec), _p(fl, ctypes.c_uint8),
                  _p(tiles, ctypes.c_int32), _p(counts, ctypes.c_int64), _p(sm), int(full))
    return {"f": f, "eps_r": rec, "flags": fl, "tiles": tiles, "counts": counts,
            "sums": sm}


def run_aar(f, tau: float, tau2: float, nsteps: int, output_every: int = 1,
            refine=("kn", 1e-3), switch=("neq", 1e-4), tile: int = 16, region=None):
    """nsteps steps of adaptive algorithm refinement from the state f.

    Step n: stream; on output steps (n % output_every == 0) all sensors of the
    streamed state (eps_qe of the two-relaxation model), the flags and the sums;
    collide with the two-relaxation model in the region in force (that of the most
    recent output step before n: its switch flags; `region` (default: empty) before
    the first one); after an output step the region is its switch flags.
    Returns a dict: f, region, switch_margin (the smallest |eps_s - thr_s| of any cell
    at any output step: how far every switch decision was from the threshold), and of
    the last output step (None if there was none) sensors, flags, tiles, counts, sums."""
    f = _f64(f).copy()
    ny, nx = f.shape[1:]
    reg = (np.zeros((ny, nx), dtype=np.uint8) if region is None
           else (np.asarray(region) != 0).astype(np.uint8))
    rs, rt = SENSOR_ID.get(refine[0], refine[0]), refine[1]
    ss, st = SENSOR_ID.get(switch[0], switch[0]), switch[1]
    last = dict(sensors=None, flags=None, tiles=None, counts=None, sums=None)
    margin = float("inf")
    for n in range(1, nsteps + 1):
        ft = stream(f)
        out = output_every > 0 and n % output_every == 0
        if out:
            sens, nonpos = sensor_fields(ft, tau, pull=False, two_relax=True)
            fl, tl, cnt = flags(sens[rs], rt, sens[ss], st, nonpos, tile)
            margin = min(margin, float(np.min(np.abs(sens[ss] - st))))
            last = dict(sensors=sens, flags=fl, tiles=tl, counts=cnt, sums=sums(ft))
        f = collide_aar(ft, tau, tau2, reg)
        if out:
            reg = ((last["flags"] & 0x02) != 0).astype(np.uint8)
    return dict(f=f, region=reg, switch_margin=margin, **last)


def adjoint_kl(rho0, ux0, uy0, tau: float, nsteps: int, weight=None, store_every: int = 1):
    """(J, dJ/drho0 [ny, nx], dJ/dtau) of J = sum W eps_KL at step nsteps (orc.h)."""
    rho0, ux0, uy0 = _f64(rho0), _f64(ux0), _f64(uy0)
    ny, nx = rho0.shape
    w = None if weight is None else _f64(weight)
    J, gt = ctypes.c_double(), ctypes.c_double()
    g = np.empty((ny, nx))
    rc = lib().orc_adjoint_kl(nx, ny, tau, nsteps, store_every, _p(rho0), _p(ux0), _p(uy0),
                              None if w is None else _p(w), ctypes.byref(J), _p(g),
                              ctypes.byref(gt))
    if rc != 0:
        raise MemoryError("orc_adjoint_kl failed")
    return J.value, g, gt.value


def objective_kl(rho0, ux0, uy0, tau: float, nsteps: int, weight=None) -> float:
    """J = sum W eps_KL of step nsteps by plain forward steps and the sensor fields
    (no adjoint code involved)."""
    f = init_equilibrium(rho0, ux0, uy0)
    f = step(f, tau, nsteps - 1)
    kl = sensor_fields(f, tau, pull=True)[0][SENSOR_ID["kl"]]
    w = 1.0 if weight is None else _f64(weight)
    return float(np.sum(w * kl))


def fp16_round(x: float) -> float:
    return lib().orc_fp16_round(float(x))


def dev16_encode(f, rho0: float = 1.0, dev_exp: int = 12, unscaled: bool = False):
    """FP16 deviation codes (binary16 values as float64) of populations f[9, ny, nx]."""
    f = _f64(f)
    h = np.empty_like(f)
    lib().orc_dev16_encode(f.shape[2], f.shape[1], rho0, dev_exp, int(unscaled), _p(f), _p(h))
    return h


def dev16_decode(h, rho0: float = 1.0, dev_exp: int = 12, unscaled: bool = False):
    """Populations f[9, ny, nx] (float64 holding binary32 values) of FP16 deviation codes."""
    h = _f64(h)
    f = np.empty_like(h)
    lib().orc_dev16_decode(h.shape[2], h.shape[1], rho0, dev_exp, int(unscaled), _p(h), _p(f))
    return f
