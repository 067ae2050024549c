"""GPU: FP16 deviation storage (precision "fp16dev": populations stored as binary16
deviations from the rest equilibrium, collided in FP32) against the oracle.

The storage rounds every population once per step, so the reference is the oracle's
own FP16 deviation codec (oracle.dev16_encode / dev16_decode, pinned against numpy's
float16 rounding): from a state that both sides store exactly, one step agrees within
one binary16 quantum of the code plus a few FP32 roundings of the value; sensors,
flags and sums of a stored state follow the FP32 tolerances; error against the
unrounded FP64 oracle is measured and bounded.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

K = 12          # scale exponent: s_q w_q = (8/9) 2^12
SHIFT = np.array([1, 3, 3, 3, 3, 5, 5, 5, 5])
ALL = tuple(range(13))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_13618_gb300 import kss

    kss.load()
    yield


def _kss():
    from paper_2603_13618_gb300 import kss

    return kss


def _quantum(h, k=K):
    """Value of one binary16 step of each code h (as a population difference)."""
    e = np.maximum(np.floor(np.log2(np.maximum(np.abs(h), 2.0 ** -14))), -14)
    return 2.0 ** (e - 10) / 2.0 ** (SHIFT + k)[:, None, None]


def _stored_state(nx, ny, seed, tau, steps=15):
    """An oracle state rounded to the FP16 deviation form; codes below 1 are set to 0 so
    that the FP32 decode and re-encode of the library reproduce every code exactly."""
    r, u, v = inputs.random_smooth(nx, ny, seed=seed, kmax=4, drho_amp=0.02, mach=0.1)
    f = oracle.step(oracle.init_equilibrium(r, u, v), tau, steps)
    h = oracle.dev16_encode(f, rho0=1.0, dev_exp=K)
    h[np.abs(h) < 1.0] = 0.0
    return oracle.dev16_decode(h, rho0=1.0, dev_exp=K)


@pytest.mark.parametrize("nx,ny,tile", [(37, 21, 16), (130, 67, 8), (5, 1, 8), (200, 9, 32)])
def test_stored_state_round_trip_and_its_sensors(nx, ny, tile):
    kss = _kss()
    tau = 0.7
    X = _stored_state(nx, ny, seed=nx + ny, tau=tau)
    lat = kss.Lattice(nx, ny, precision="fp16dev", tau=tau, tile=tile, dev_exp=K)
    lat.set_populations(X)
    np.testing.assert_array_equal(lat.get_populations(), X)
    ref, nonpos = oracle.sensor_fields(X, tau, pull=False)
    r, u, v = oracle.moments(X)
    for sid in ALL:
        name = parity.SENSORS[sid]
        parity.assert_sensor_close(name, lat.read_sensor(name), ref[sid], "fp32", 0, r, u, v,
                                   ref[oracle.SENSOR_ID["kn"]], tau, ft=X)
    lat.close()


# (517 x 40: three 256-column blocks of the eight-cell step, an odd row end at the periodic
# seam and in lane 0 of the last block; 300 x 33: the row-end lane's upper four cells lie
# past the row end)
@pytest.mark.parametrize("nx,ny,tile,tau", [(37, 21, 16, 0.7), (130, 67, 8, 0.55),
                                            (1, 5, 8, 0.9), (256, 96, 16, 1.2),
                                            (517, 40, 16, 0.8), (300, 33, 8, 0.6)])
def test_one_step_against_the_oracle_codec(nx, ny, tile, tau):
    kss = _kss()
    X = _stored_state(nx, ny, seed=3 * nx + ny, tau=tau)
    lat = kss.Lattice(nx, ny, precision="fp16dev", tau=tau, tile=tile, dev_exp=K,
                      record=("kl", "kn", "neq"))
    lat.set_populations(X)
    lat.step(1)
    got = lat.get_populations()
    fo = oracle.step(X, tau)
    ho = oracle.dev16_encode(fo, rho0=1.0, dev_exp=K)
    want = oracle.dev16_decode(ho, rho0=1.0, dev_exp=K)
    bound = _quantum(ho) + 8 * 2.0 ** -24 * np.abs(want)
    assert np.all(np.abs(got - want) <= bound)
    assert np.mean(got == want) > 0.95  # codes differ only where FP32 rounding decides
    # sensors, flags and sums of the step: the FP32 arithmetic on exactly stored inputs
    ref, nonpos = oracle.sensor_fields(X, tau, pull=True)
    ft = oracle.stream(X)
    r, u, v = oracle.moments(ft)
    kn = ref[oracle.SENSOR_ID["kn"]]
    for name in ("kn", "kl", "neq", "tau_ns", "alpha"):
        sid = oracle.SENSOR_ID[name]
        parity.assert_sensor_close(name, lat.read_sensor(name), ref[sid], "fp32", 0, r, u, v, kn,
                                   tau, ft=ft)
    rf, rt, rcnt = oracle.flags(kn, 1e-3, ref[oracle.SENSOR_ID["neq"]], 1e-4, nonpos, tile)
    flags, tiles, counts = lat.read_flags()
    band = parity.band_mask(kn, 1e-3, ref[oracle.SENSOR_ID["neq"]], 1e-4)
    parity.assert_flags_match(flags, tiles, counts, rf, rt, rcnt, band, tile)
    sums, _, _ = lat.read_stats()
    want_s = oracle.sums(ft)
    assert np.all(np.abs(sums - want_s) <= 64 * parity.UNIT_ROUNDOFF["fp32"] * want_s[0])
    lat.close()


def test_trajectory_follows_the_oracle_codec():
    """30 steps: the library and the oracle both round to FP16 deviations every step;
    their codes part only where the FP32 arithmetic of the library decides a rounding
    differently, one quantum at a time."""
    kss = _kss()
    nx, ny, tau, n = 96, 80, 0.8, 30
    X = _stored_state(nx, ny, seed=21, tau=tau)
    lat = kss.Lattice(nx, ny, precision="fp16dev", tau=tau, dev_exp=K, output_every=0)
    lat.set_populations(X)
    lat.step(n)
    got = lat.get_populations()
    f = X
    for _ in range(n):
        f = oracle.dev16_decode(oracle.dev16_encode(oracle.step(f, tau), rho0=1.0, dev_exp=K),
                                rho0=1.0, dev_exp=K)
    # a differing rounding moves mass and momentum, which the next steps spread to the
    # neighbouring cells and to every population of them: measure the differences in
    # the coarsest code step of each population plane
    q = _quantum(oracle.dev16_encode(f, rho0=1.0, dev_exp=K))
    qmax = q.reshape(9, -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(got - f) / qmax) <= 8
    assert np.mean(got == f) > 0.5
    r1, _, _ = lat.read_moments()
    r2, _, _ = oracle.moments(f)
    assert np.max(np.abs(r1 - r2)) <= 8 * float(np.sum(qmax))
    lat.close()


@pytest.mark.parametrize("N", [1024, 8192])
def test_error_against_fp64_on_a_window(N):
    """The precision workload's inputs (smooth perturbations of amplitude 1e-3 in density
    and velocity) on an N^2 lattice (8192^2: the benchmark's size and launch
    configuration), 100 steps: FP16 deviations (K = 20) against the unrounded FP64 oracle
    on the central 128^2 window (the oracle runs the window's domain of dependence,
    328^2).  Two roundings act each step: the FP32 collision (the parity suite's
    population bound, 64 u sqrt(n + 1) relative with u = 2^-24) and the storage, which
    rounds every population's deviation d_q = f_q - w_q rho0 to binary16 (unit round-off
    2^-11 of the code), moving a cell's density and momentum by at most 2^-11 sum_q |d_q|
    per step, independent from step to step (a random walk): error <=
    64 u sqrt(n + 1) max rho + sqrt(n) 2^-11 max_cell sum_q |d_q|.  At this amplitude the
    deviations are small and the FP32 term dominates.  At 1024^2 the Kn sensor (about
    1e-5) is resolved above that noise; at 8192^2 (gradients 8 times smaller) it is not,
    and only the FP32 sensor tolerance applies."""
    kss = _kss()
    n, W, k = 100, 128, 20
    amp = 1e-3
    gen = dict(seed=8192, kmax=8, drho_amp=amp, mach=amp / inputs.CS, jump=1.0)
    rho, ux, uy = inputs.smooth_jump(N, N, **gen)
    lat = kss.Lattice(N, N, precision="fp16dev", tau=0.6, dev_exp=k, record=("kn", "kl"))
    lat.set_fields(rho, ux, uy)
    lat.step(n)
    x0 = N // 2 - W // 2
    r, u, v = lat.read_moments()
    kn = lat.read_sensor("kn")
    halo = n
    wr, wu, wv = inputs.smooth_jump(N, N, x0=x0 - halo, y0=x0 - halo, wx=W + 2 * halo,
                                    wy=W + 2 * halo, **gen)
    f = oracle.init_equilibrium(wr, wu, wv)
    f = oracle.step(f, 0.6, n - 1)
    sens, _ = oracle.sensor_fields(f, 0.6, pull=True)
    f = oracle.step(f, 0.6)
    rr, ru, rv = oracle.moments(f)
    c = slice(halo, halo + W)
    win = (slice(x0, x0 + W), slice(x0, x0 + W))
    err_rho = np.max(np.abs(r[win] - rr[c, c]))
    err_u = np.max(np.abs(u[win] - ru[c, c]))
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    dev = float(np.max(np.sum(np.abs(f[:, c, c] - w), axis=0)))
    bound = (64 * 2.0**-24 * math.sqrt(n + 1) * float(np.max(rr[c, c]))
             + math.sqrt(n) * 2.0**-11 * dev)
    assert err_rho <= bound, (err_rho, bound)
    assert err_u <= bound, (err_u, bound)
    kn_ref = sens[oracle.SENSOR_ID["kn"]][c, c]
    err_kn = np.max(np.abs(kn[win] - kn_ref))
    if N == 1024:  # Kn (about 1e-5) stands above the storage noise
        assert err_kn <= 0.2 * np.max(kn_ref) + 1e-6
    else:  # the gradients scale as 1/N: Kn (about 5e-6) is below the FP32 noise floor,
        # so only the suite's FP32 sensor tolerance applies (64 u sqrt(n + 1) times Kn's
        # scale, 9)
        assert err_kn <= 64 * 2.0**-24 * math.sqrt(n + 1) * 9
    lat.close()


def test_batched_fp16_members_equal_single_lattices():
    kss = _kss()
    specs = [dict(nx=37, ny=21, tau=0.7), dict(nx=130, ny=67, tau=1.0, tile=8),
             dict(nx=64, ny=64, tau=0.55)]
    b = kss.Batch(specs, precision="fp16dev", dev_exp=K)
    singles = []
    for k, sp in enumerate(specs):
        fld = inputs.random_smooth(sp["nx"], sp["ny"], seed=k, kmax=3)
        b[k].set_fields(*fld)
        lat = kss.Lattice(precision="fp16dev", dev_exp=K, **sp)
        lat.set_fields(*fld)
        singles.append(lat)
    b.step(6)
    for lat in singles:
        lat.step(6)
    for k in range(len(specs)):
        np.testing.assert_array_equal(b[k].get_populations(), singles[k].get_populations())
        np.testing.assert_array_equal(b[k].read_flags()[0], singles[k].read_flags()[0])
        np.testing.assert_array_equal(b[k].read_sensor("kl"), singles[k].read_sensor("kl"))
        singles[k].close()
    b.close()


@pytest.fixture(scope="module")
def _all_cores():
    n = oracle.set_threads(oracle.host_cores())
    yield n
    oracle.set_threads(1)


def test_full_field_4096_one_step(_all_cores):
    """The benchmark's FP16 launch geometry (4096^2 and up take 64-row CTAs, with the row
    prefetch of the codes): one step from an exactly stored state, every cell against the
    oracle's step and FP16 codec -- populations within a quantum, the recorded Kn, KL and
    neq fields, flags outside the threshold band, tile counts, counts and sums."""
    kss = _kss()
    n, tau, tile = 4096, 0.6, 16
    r0, u0, v0 = inputs.random_smooth(n, n, seed=2603, kmax=8, drho_amp=0.02, mach=0.1)
    f = oracle.step(oracle.init_equilibrium(r0, u0, v0), tau, 3)
    h = oracle.dev16_encode(f, rho0=1.0, dev_exp=K)
    h[np.abs(h) < 1.0] = 0.0
    X = oracle.dev16_decode(h, rho0=1.0, dev_exp=K)
    del f, h, r0, u0, v0
    lat = kss.Lattice(n, n, precision="fp16dev", tau=tau, tile=tile, dev_exp=K,
                      refine_sensor="kn", refine_threshold=1e-3, switch_sensor="neq",
                      switch_threshold=1e-4, record=("kl", "kn", "neq"), output_every=1)
    lat.set_populations(X)
    lat.step(1)
    got = lat.get_populations()
    sens_got = {s: lat.read_sensor(s) for s in ("kn", "kl", "neq")}
    flags, tiles, counts = lat.read_flags()
    sums, _, _ = lat.read_stats()
    lat.close()
    ho = oracle.dev16_encode(oracle.step(X, tau), rho0=1.0, dev_exp=K)
    want = oracle.dev16_decode(ho, rho0=1.0, dev_exp=K)
    assert np.all(np.abs(got - want) <= _quantum(ho) + 8 * 2.0 ** -24 * np.abs(want))
    assert np.mean(got == want) > 0.95
    del got, want, ho
    ref, nonpos = oracle.sensor_fields(X, tau, pull=True)
    ft = oracle.stream(X)
    r, u, v = oracle.moments(ft)
    kn = ref[oracle.SENSOR_ID["kn"]]
    neq = parity.neq_field(ft)
    for name, field in sens_got.items():
        parity.assert_sensor_close(name, field, ref[oracle.SENSOR_ID[name]], "fp32", 0, r, u, v,
                                   kn, tau, neq=neq, where="fp16dev 4096^2 one step")
    es = ref[oracle.SENSOR_ID["neq"]]
    rf, rt, rcnt = oracle.flags(kn, 1e-3, es, 1e-4, nonpos, tile)
    band = parity.band_mask(kn, 1e-3, es, 1e-4)
    parity.assert_flags_match(flags, tiles, counts, rf, rt, rcnt, band, tile)
    want_s = oracle.sums(ft)
    assert np.all(np.abs(sums - want_s) <= 64 * parity.UNIT_ROUNDOFF["fp32"] * want_s[0])
