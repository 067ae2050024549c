"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, element
by element, on seeded synthetic inputs.  Tolerances: see tests/parity.py."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

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


def _oracle_run(rho, ux, uy, tau, nsteps):
    """(state before the last step, final state) of the oracle."""
    f = oracle.init_equilibrium(rho, ux, uy)
    prev = f
    for _ in range(nsteps):
        prev = f
        f = oracle.step(f, tau)
    return prev, f


def _check_step_outputs(lat, prec, prev, tau, nsteps, thr_r, thr_s, tile, sensors=ALL,
                        refine="kn", switch="neq"):
    """Sensors, flags, tiles, counts and sums of the last step vs the oracle."""
    ref, nonpos = oracle.sensor_fields(prev, tau, pull=nsteps > 0)
    ft = oracle.stream(prev) if nsteps > 0 else prev
    r, u, v = oracle.moments(ft)
    kn = ref[oracle.SENSOR_ID["kn"]]
    for sid in sensors:
        name = parity.SENSORS[sid]
        got = lat.read_sensor(name)
        parity.assert_sensor_close(name, got, ref[sid], prec, nsteps, r, u, v, kn, tau, ft=ft)
    er, es = ref[oracle.SENSOR_ID[refine]], ref[oracle.SENSOR_ID[switch]]
    rf, rt, rcnt = oracle.flags(er, thr_r, es, thr_s, nonpos, tile)
    flags, tiles, counts = lat.read_flags()
    band = parity.band_mask(er, thr_r, es, thr_s)
    parity.assert_flags_match(flags, tiles, counts, rf, rt, rcnt, band, tile)
    sums, c2, step = lat.read_stats()
    np.testing.assert_array_equal(c2, counts)
    assert step == nsteps
    want = oracle.sums(ft)
    scale = want[0]
    tol = 64 * parity.UNIT_ROUNDOFF[prec] * math.sqrt(nsteps + 1) * scale
    assert np.all(np.abs(sums - want) <= tol), (sums, want)


@pytest.mark.parametrize("nx,ny,tile,tau", [(37, 21, 16, 0.7), (64, 64, 8, 0.55),
                                            (130, 67, 32, 1.0), (1, 5, 8, 0.8),
                                            (5, 1, 8, 0.8), (200, 9, 64, 0.6),
                                            (3, 3, 16, 0.9)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", ["vector", "tma"])
def test_ragged_lattices(kernel, prec, nx, ny, tile, tau):
    kss = _kss()
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=nx * 1000 + ny, kmax=3)
    nsteps = 7
    prev, fin = _oracle_run(rho, ux, uy, tau, nsteps)
    thr_r, thr_s = 2e-3, 3e-4
    lat = kss.Lattice(nx, ny, precision=prec, tau=tau, refine_threshold=thr_r,
                      switch_threshold=thr_s, record=("kl", "kn", "neq"), tile=tile,
                      kernel=kernel)
    lat.set_fields(rho, ux, uy)
    lat.step(nsteps)
    got = lat.get_populations()
    u = parity.UNIT_ROUNDOFF[prec]
    assert np.max(np.abs(got - fin) / fin) <= 64 * u * math.sqrt(nsteps + 1)
    r, vx, vy = lat.read_moments()
    rr, ru, rv = oracle.moments(fin)
    assert np.max(np.abs(r - rr) / rr) <= 64 * u * math.sqrt(nsteps + 1)
    _check_step_outputs(lat, prec, prev, tau, nsteps, thr_r, thr_s, tile)
    lat.close()


@pytest.mark.parametrize("kernel", ["vector", "tma"])
def test_cfg1_shear_wave_fp64_2000_steps(kernel):
    """128^2 FP64 shear wave, tau = 0.8, 2000 steps, sensors and flags every 10 steps."""
    kss = _kss()
    nx = ny = 128
    tau, thr = 0.8, 1e-3
    rho, ux, uy = inputs.shear_wave(nx, ny, 0.01)
    lat = kss.Lattice(nx, ny, precision="fp64", tau=tau, refine_sensor="kn",
                      refine_threshold=thr, switch_sensor="neq", switch_threshold=1e-4,
                      record=("kn", "kl"), output_every=10, tile=16, kernel=kernel)
    lat.set_fields(rho, ux, uy)
    f = oracle.init_equilibrium(rho, ux, uy)
    done = 0
    checkpoints = (10, 50, 500, 1000, 2000)
    for t in checkpoints:
        f_prev = oracle.step(f, tau, t - 1 - done) if t - 1 > done else f
        f = oracle.step(f_prev, tau, 1)
        lat.step(t - done)
        done = t
        got = lat.get_populations()
        assert np.max(np.abs(got - f) / f) <= 1e-12
        r, vx, vy = lat.read_moments()
        rr, ru, rv = oracle.moments(f)
        assert np.max(np.abs(r - rr) / rr) <= 1e-12
        assert np.max(np.abs(vx - ru)) <= 1e-12 * np.max(np.abs(ru))
        _check_step_outputs(lat, "fp64", f_prev, tau, t, thr, 1e-4, 16,
                            sensors=(oracle.SENSOR_ID["kn"], oracle.SENSOR_ID["kl"],
                                     oracle.SENSOR_ID["neq"]))
    lat.close()


@pytest.mark.parametrize("tau,kernel", [(0.51, "vector"), (0.6, "vector"), (0.8, "vector"),
                                        (1.0, "vector"), (0.51, "tma"), (0.6, "tma"),
                                        (1.0, "tma")])
def test_fp32_smooth_jump_100_steps(tau, kernel):
    """FP32 moments within 1e-5 (relative) of the FP64 oracle after 100 steps, on the
    density-jump workload at a size the oracle finishes in seconds."""
    kss = _kss()
    nx, ny, nsteps = 192, 160, 100
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=2603, kmax=8)
    prev, fin = _oracle_run(rho, ux, uy, tau, nsteps)
    lat = kss.Lattice(nx, ny, precision="fp32", tau=tau, record=("kl",), kernel=kernel)
    lat.set_fields(rho, ux, uy)
    lat.step(nsteps)
    r, vx, vy = lat.read_moments()
    rr, ru, rv = oracle.moments(fin)
    assert np.max(np.abs(r - rr) / rr) <= 1e-5
    umax = np.max(np.hypot(ru, rv))
    assert np.max(np.abs(r * vx - rr * ru)) <= 1e-5 * np.max(rr) * umax
    assert np.max(np.abs(r * vy - rr * rv)) <= 1e-5 * np.max(rr) * umax
    _check_step_outputs(lat, "fp32", prev, tau, nsteps, 1e-3, 1e-4, 16)
    lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sensors_on_the_same_state(prec):
    """Sensor arithmetic alone: an oracle state, rounded to the storage precision by
    numpy, is set on the lattice and evaluated by both sides without a step."""
    kss = _kss()
    nx, ny, tau = 96, 80, 0.65
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=44, kmax=6)
    state = oracle.step(oracle.init_equilibrium(rho, ux, uy), tau, 20)
    if prec == "fp32":
        state = state.astype(np.float32).astype(np.float64)
    lat = kss.Lattice(nx, ny, precision=prec, tau=tau, record=())
    lat.set_populations(state)             # no step since set: sensors of the stored state
    np.testing.assert_array_equal(lat.get_populations(), state)
    ref, nonpos = oracle.sensor_fields(state, tau, pull=False)
    r, u, v = oracle.moments(state)
    for sid in ALL:
        name = parity.SENSORS[sid]
        parity.assert_sensor_close(name, lat.read_sensor(name), ref[sid], prec, 0, r, u, v,
                                   ref[oracle.SENSOR_ID["kn"]], tau, ft=state)
    lat.close()


def test_zero_at_equilibrium_and_rest_state():
    kss = _kss()
    rho, ux, uy = inputs.random_smooth(40, 24, seed=3)
    for prec in ("fp64", "fp32"):
        lat = kss.Lattice(40, 24, precision=prec, tau=0.9)
        lat.set_fields(rho, ux, uy)
        for name in ("kn", "kl", "neq", "tau_ns", "alpha"):
            assert np.max(np.abs(lat.read_sensor(name))) <= (1e-13 if prec == "fp64" else 2e-5)
        fl, tiles, counts = lat.read_flags()
        assert not fl.any() and not tiles.any() and not counts.any()
        lat.close()
    # uniform rest state: a fixed point, bit for bit
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = np.ascontiguousarray(np.broadcast_to((1.25 * w)[:, None, None], (9, 8, 12)))
    lat = kss.Lattice(12, 8, precision="fp64", tau=0.7)
    lat.set_populations(f)
    lat.step(5)
    np.testing.assert_array_equal(lat.get_populations(), f)
    lat.close()


def test_nonpositive_convention():
    kss = _kss()
    nx, ny, tau = 24, 16, 0.8
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = np.ascontiguousarray(np.broadcast_to(w[:, None, None], (9, ny, nx))).copy()
    f[5, 3, 4] = -1e-3
    f[0, 3, 4] += 1e-3 + 1 / 36
    for prec in ("fp64", "fp32"):
        lat = kss.Lattice(nx, ny, precision=prec, tau=tau)
        lat.set_populations(f)
        kn = lat.read_sensor("kn")
        assert lat.last_status == kss.KSS_WARN_NONPOSITIVE
        assert kn[3, 4] == math.inf and np.isfinite(np.delete(kn.ravel(), 3 * nx + 4)).all()
        for name in ("hr", "kl", "sigma_h", "sigma_kl", "alpha"):
            assert lat.read_sensor(name)[3, 4] == math.inf
        assert np.isfinite(lat.read_sensor("neq")).all()
        fl, tiles, counts = lat.read_flags()
        assert fl[3, 4] == kss.FLAG_NONPOS | kss.FLAG_REFINE | kss.FLAG_SWITCH
        assert counts[2] == 1 and counts[0] == 1
        lat.close()


def test_conservation_and_reproducibility_fp64():
    kss = _kss()
    nx, ny, tau = 256, 200, 0.6
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=9, kmax=8)
    sums = []
    for _ in range(2):
        lat = kss.Lattice(nx, ny, precision="fp64", tau=tau, output_every=50)
        lat.set_fields(rho, ux, uy)
        s0 = lat.read_stats()[0]
        lat.step(500)
        s1, _, step = lat.read_stats()
        assert step == 500
        assert np.all(np.abs(s1 - s0) <= 4 * 2.0**-52 * 500 * s0[0])
        sums.append(s1)
        lat.close()
    np.testing.assert_array_equal(sums[0], sums[1])  # fixed-order reductions


def test_device_pointer_paths():
    import torch

    kss = _kss()
    nx, ny, tau = 80, 48, 0.75
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=12, kmax=4)
    prev, fin = _oracle_run(rho, ux, uy, tau, 3)
    lat = kss.Lattice(nx, ny, precision="fp64", tau=tau)
    lat.set_fields(*(torch.from_numpy(a).cuda() for a in (rho, ux, uy)))
    lat.step(3)
    f_dev = lat.get_populations(device=True)
    assert f_dev.is_cuda
    np.testing.assert_allclose(f_dev.cpu().numpy(), fin, rtol=1e-13)
    kl = lat.read_sensor("kl", device=True).cpu().numpy()
    np.testing.assert_allclose(kl, lat.read_sensor("kl"), rtol=0, atol=0)
    fl_d, t_d, c_d = lat.read_flags(device=True)
    fl_h, t_h, c_h = lat.read_flags()
    np.testing.assert_array_equal(fl_d.cpu().numpy(), fl_h)
    np.testing.assert_array_equal(t_d.cpu().numpy(), t_h)
    # populations round trip through device memory, then identical continuation
    lat.set_populations(f_dev)
    lat.step(2)
    np.testing.assert_allclose(lat.get_populations(), oracle.step(fin, tau, 2), rtol=1e-13)
    lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
def test_reading_other_sensors_keeps_the_step_outputs(prec):
    """A sensor the step did not record is evaluated on demand (for alpha: the all-sensor
    pass, which sums in another order and takes another KL series); the flags, tile
    counts, counts and sums of the step must stay exactly those the step produced."""
    kss = _kss()
    nx, ny = 150, 70
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=17, kmax=6)
    lat = kss.Lattice(nx, ny, precision=prec, tau=0.62, record=("kl",))
    lat.set_fields(rho, ux, uy)
    lat.step(5)
    before = (lat.read_flags(), lat.read_stats())
    for name in ("alpha", "sigma_h", "kn", "qe"):
        lat.read_sensor(name)
    after = (lat.read_flags(), lat.read_stats())
    for x, y in zip(before[0], after[0]):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(before[1], after[1]):
        np.testing.assert_array_equal(x, y)
    lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
def test_pinned_host_inputs(prec):
    """Page-locked host inputs are read by the initialisation kernels directly; pageable
    ones (or a mix) go through the staging copy.  Both give the same state bit for bit."""
    import torch

    kss = _kss()
    nx, ny = 70, 45
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=31, kmax=4)
    pinned = [torch.from_numpy(a).pin_memory() for a in (rho, ux, uy)]
    states = []
    for fields in ((rho, ux, uy), pinned, (pinned[0], ux, pinned[2])):
        lat = kss.Lattice(nx, ny, precision=prec, tau=0.7)
        lat.set_fields(*fields)
        states.append(lat.get_populations())
        lat.close()
    np.testing.assert_array_equal(states[1], states[0])
    np.testing.assert_array_equal(states[2], states[0])
    f = oracle.step(oracle.init_equilibrium(rho, ux, uy), 0.7, 2)
    out = []
    for arr in (f, torch.from_numpy(f).pin_memory()):
        lat = kss.Lattice(nx, ny, precision=prec, tau=0.7)
        lat.set_populations(arr)
        lat.step(1)
        out.append(lat.get_populations())
        lat.close()
    np.testing.assert_array_equal(out[1], out[0])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
def test_fp32_fields(prec):
    """kss_set_fields_f32: FP32 fields from pageable host, page-locked host and device memory
    give the state of the same values passed as FP64, bit for bit, and so do three fused
    steps from it (populations, flags, tile counts, counts, sums, the recorded field); on
    an FP32 lattice the oracle's equilibrium of those values is within the FP32 rounding."""
    import torch

    kss = _kss()
    nx, ny = 300, 77
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=37, kmax=6)
    f32 = [a.astype(np.float32) for a in (rho, ux, uy)]
    f64 = [a.astype(np.float64) for a in f32]
    lats = []
    for fields in (f64, f32, [torch.from_numpy(a).pin_memory() for a in f32],
                   [torch.from_numpy(a).cuda() for a in f32]):
        lat = kss.Lattice(nx, ny, precision=prec, tau=0.7, record=("kl",))
        lat.set_fields(*fields)
        lats.append(lat)
    torch.cuda.synchronize()
    ref = lats[0]
    want = ref.get_populations()
    for lat in lats[1:]:
        np.testing.assert_array_equal(lat.get_populations(), want)
    if prec == "fp32":
        feq = oracle.init_equilibrium(*f64)
        assert np.max(np.abs(want - feq)) <= 8 * parity.UNIT_ROUNDOFF["fp32"] * np.max(feq)
    for lat in lats:
        lat.step(3)
    fr, tr, cr = ref.read_flags()
    for lat in lats[1:]:
        np.testing.assert_array_equal(lat.get_populations(), ref.get_populations())
        fl, tl, cl = lat.read_flags()
        np.testing.assert_array_equal(fl, fr)
        np.testing.assert_array_equal(tl, tr)
        np.testing.assert_array_equal(cl, cr)
        np.testing.assert_array_equal(lat.read_stats()[0], ref.read_stats()[0])
        np.testing.assert_array_equal(lat.read_sensor("kl"), ref.read_sensor("kl"))
    for lat in lats:
        lat.close()


def test_plain_steps_and_output_cadence():
    """output_every = 0 runs plain stream + collide; reads then evaluate on demand."""
    kss = _kss()
    nx, ny, tau = 64, 40, 0.7
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=21, kmax=4)
    prev, fin = _oracle_run(rho, ux, uy, tau, 9)
    for every in (0, 4):
        lat = kss.Lattice(nx, ny, precision="fp64", tau=tau, output_every=every,
                          record=("kl",))
        lat.set_fields(rho, ux, uy)
        lat.step(9)
        np.testing.assert_allclose(lat.get_populations(), fin, rtol=1e-13)
        _check_step_outputs(lat, "fp64", prev, tau, 9, 1e-3, 1e-4, 16)
        lat.close()


def test_switch_disabled_and_other_sensors_drive_flags():
    kss = _kss()
    nx, ny, tau = 72, 56, 0.6
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=5, kmax=5)
    prev, _ = _oracle_run(rho, ux, uy, tau, 6)
    lat = kss.Lattice(nx, ny, precision="fp64", tau=tau, refine_sensor="alpha",
                      refine_threshold=1e-4, switch_sensor="kl", switch_threshold=-1.0,
                      record=("sigma_h", "tau_ns"))
    lat.set_fields(rho, ux, uy)
    lat.step(6)
    _check_step_outputs(lat, "fp64", prev, tau, 6, 1e-4, -1.0, 16, refine="alpha",
                        switch="kl")
    fl, tiles, counts = lat.read_flags()
    assert not (fl & 2).any() and counts[1] == 0
    lat.close()


def test_library_owned_stream():
    kss = _kss()
    nx, ny, tau = 50, 30, 0.8
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=2, kmax=3)
    prev, fin = _oracle_run(rho, ux, uy, tau, 4)
    lat = kss.Lattice(nx, ny, precision="fp32", tau=tau, stream="own")
    lat.set_fields(rho, ux, uy)
    lat.step(4)
    np.testing.assert_allclose(lat.get_populations(), fin, rtol=64 * 2.0**-24 * math.sqrt(5))
    _check_step_outputs(lat, "fp32", prev, tau, 4, 1e-3, 1e-4, 16)
    lat.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_vector_and_tma_kernels_agree(prec):
    """Both step kernels run the same per-cell arithmetic: same states, fields, flags."""
    kss = _kss()
    nx, ny, tau = 517, 263, 0.6
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=8, kmax=8)
    out = {}
    for kernel in ("vector", "tma"):
        lat = kss.Lattice(nx, ny, precision=prec, tau=tau, record=("kl", "kn"), kernel=kernel,
                          output_every=3)
        lat.set_fields(rho, ux, uy)
        lat.step(30)
        out[kernel] = (lat.get_populations(), lat.read_sensor("kl"), lat.read_sensor("kn"),
                       *lat.read_flags(), lat.read_stats()[0], lat.read_moments())
        lat.close()
    a, b = out["vector"], out["tma"]
    rt = 64 * parity.UNIT_ROUNDOFF[prec] * math.sqrt(31)
    np.testing.assert_allclose(a[0], b[0], rtol=rt)
    r, u, v = a[7]
    for k, name in ((1, "kl"), (2, "kn")):
        parity.assert_sensor_close(name, b[k], a[k], prec, 30, r, u, v, a[2], tau)
    # the tag counts agree exactly wherever the flags do (both kernels' counts are
    # recounts of their own flags, checked against the oracle elsewhere)
    same = np.array_equal(a[3], b[3])
    if same:
        np.testing.assert_array_equal(a[4], b[4])
        np.testing.assert_array_equal(a[5], b[5])
    else:
        assert np.mean(a[3] != b[3]) < 1e-3
    # conservation sums: the states differ by round-off, bounded as in the oracle parity
    np.testing.assert_allclose(a[6], b[6], rtol=0, atol=rt * a[6][0])


def _cone_window(nx, ny, x0, y0, w, nsteps, tau):
    """Oracle state of the w x w window at global (x0, y0) after nsteps and the window's
    step-nsteps sensors, from the domain of dependence (margin nsteps + 1)."""
    m = nsteps + 1
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=2603, kmax=8, x0=x0 - m, y0=y0 - m,
                                     wx=w + 2 * m, wy=w + 2 * m)
    f = oracle.init_equilibrium(rho, ux, uy)
    prev = f
    for _ in range(nsteps):
        prev = f
        f = oracle.step(f, tau)
    sens, nonpos = oracle.sensor_fields(prev, tau, pull=True)
    sl = (slice(m, m + w), slice(m, m + w))
    r, vx, vy = oracle.moments(f)
    return {"rho": r[sl], "ux": vx[sl], "uy": vy[sl], "sens": sens[:, sl[0], sl[1]],
            "nonpos": nonpos[sl]}


def test_full_size_4096_fp32_bench_configuration():
    """The benchmark's workload and launch configuration (4096^2 FP32, tau = 0.6, Kn
    refine 1e-3, neq switch 1e-4, KL recorded, output every step, tile 16, automatic
    kernel choice), 100 steps, checked on four 16 x 16 windows -- at the density step,
    across both periodic seams, in the smooth interior -- against the oracle run on
    each window's domain of dependence."""
    kss = _kss()
    nx = ny = 4096
    tau, nsteps, w = 0.6, 100, 16
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=2603, kmax=8)
    lat = kss.Lattice(nx, ny, precision="fp32", tau=tau, refine_sensor="kn",
                      refine_threshold=1e-3, switch_sensor="neq", switch_threshold=1e-4,
                      record=("kl",), output_every=1, tile=16)
    lat.set_fields(rho, ux, uy)
    lat.step(nsteps)
    r, vx, vy = lat.read_moments()
    kl = lat.read_sensor("kl")
    kn = lat.read_sensor("kn")
    flags, tiles, counts = lat.read_flags()
    lat.close()
    for (x0, y0) in ((2040, 1000), (4088, 4088), (1000, 3000), (4090, 7)):
        ref = _cone_window(nx, ny, x0, y0, w, nsteps, tau)
        xs = (x0 + np.arange(w)) % nx
        ys = (y0 + np.arange(w)) % ny
        g = np.ix_(ys, xs)
        assert np.max(np.abs(r[g] - ref["rho"]) / ref["rho"]) <= 1e-5
        umax = 0.1 / math.sqrt(3.0)  # the lattice's velocity scale: max |u| = 0.1 c_s
        assert np.max(np.abs(vx[g] - ref["ux"])) <= 1e-5 * umax
        assert np.max(np.abs(vy[g] - ref["uy"])) <= 1e-5 * umax
        rr, uu, vv = ref["rho"], ref["ux"], ref["uy"]
        kn_ref = ref["sens"][oracle.SENSOR_ID["kn"]]
        parity.assert_sensor_close("kl", kl[g], ref["sens"][oracle.SENSOR_ID["kl"]], "fp32",
                                   nsteps, rr, uu, vv, kn_ref, tau)
        parity.assert_sensor_close("kn", kn[g], kn_ref, "fp32", nsteps, rr, uu, vv, kn_ref, tau)
        es = ref["sens"][oracle.SENSOR_ID["neq"]]
        rf, _, _ = oracle.flags(kn_ref, 1e-3, es, 1e-4, ref["nonpos"], 16)
        band = parity.band_mask(kn_ref, 1e-3, es, 1e-4)
        assert not ((flags[g] != rf) & ~band).any()
    # tile counts and totals are consistent with the flag field everywhere
    fr = (flags & 1).astype(np.int64).reshape(256, 16, 256, 16).sum(axis=(1, 3))
    fs = ((flags >> 1) & 1).astype(np.int64).reshape(256, 16, 256, 16).sum(axis=(1, 3))
    np.testing.assert_array_equal(tiles[0], fr)
    np.testing.assert_array_equal(tiles[1], fs)
    assert counts[0] == fr.sum() and counts[1] == fs.sum() and counts[2] == np.sum(flags >> 7)


@pytest.mark.parametrize("state", ["far", "nonpositive"])
@pytest.mark.parametrize("prec,kernel", [("fp32", "vector"), ("fp32", "tma"), ("fp64", "vector")])
def test_deferred_cells_everywhere(prec, kernel, state):
    """far: every cell far from equilibrium (populations perturbed by up to 30 %, most
    |x_q| >= 1/16), so its KL terms take the closed form in the fused pass.
    nonpositive: the same, and in 30 % of the cells one population made negative (after
    streaming, in as many cells), so those cells are deferred to the exact recomputation,
    more than the fix-up list holds (1/8 of the lattice) on the TMA path, which then
    scans.  Both must match the oracle."""
    kss = _kss()
    nx, ny, tau = 128, 128, 0.7
    rng = np.random.default_rng(123)
    rho, ux, uy = inputs.random_smooth(nx, ny, seed=4)
    f = oracle.init_equilibrium(rho, ux, uy) * (1.0 + 0.3 * rng.uniform(-1, 1, (9, ny, nx)))
    f[5, 10, 20] = -0.01  # and one non-positive cell
    if state == "nonpositive":
        hit = rng.random((ny, nx)) < 0.3
        q = rng.integers(0, 9, (ny, nx))
        jj, ii = np.nonzero(hit)
        f[q[hit], jj, ii] *= -0.1
    thr_r, thr_s = 0.5, 0.05
    lat = kss.Lattice(nx, ny, precision=prec, tau=tau, refine_threshold=thr_r,
                      switch_threshold=thr_s, record=("kl", "kn", "neq"), kernel=kernel)
    lat.set_populations(np.ascontiguousarray(f))
    lat.step(1)
    _check_step_outputs(lat, prec, f, tau, 1, thr_r, thr_s, 16)
    # and once more from the oracle's next (still far from equilibrium) state, stored in
    # the lattice's precision: the list path again
    f2 = oracle.step(f, tau)
    if prec == "fp32":
        f2 = f2.astype(np.float32).astype(np.float64)
    lat.set_populations(f2)
    lat.step(1)
    _check_step_outputs(lat, prec, f2, tau, 1, thr_r, thr_s, 16)
    lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", ["vector", "tma"])
def test_populations_do_not_depend_on_the_outputs(prec, kernel):
    """The collision rounds the same way whether a step evaluates no sensors, the
    {Kn, KL, neq} set or all of Table 1: the populations agree bit for bit."""
    kss = _kss()
    nx, ny, tau = 150, 70, 0.62
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=7, kmax=6)
    runs = [dict(output_every=1), dict(output_every=0), dict(output_every=3),
            dict(output_every=1, record=("alpha", "kl"))]
    states = []
    for kw in runs:
        lat = kss.Lattice(nx, ny, precision=prec, tau=tau, kernel=kernel, **kw)
        lat.set_fields(rho, ux, uy)
        lat.step(9)
        states.append(lat.get_populations())
        lat.close()
    for st in states[1:]:
        np.testing.assert_array_equal(st, states[0])


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp16dev"])
@pytest.mark.parametrize("every", [1, 0])
@pytest.mark.parametrize("nx,ny,nsteps", [(37, 21, 5), (1024, 640, 6), (2048, 2048, 7)])
def test_multi_step_launch_equals_single_steps(prec, every, nx, ny, nsteps):
    """kss_step(n) with every step an output step runs, on FP32 and FP64 storage, as one
    cooperative multi-step launch whose blocks wait only on their neighbours; it must give
    exactly the results of n single-step launches (populations, flags, tile counts,
    counts, sums and the recorded field).  (FP16 deviations and plain steps take one
    launch per step either way.)"""
    kss = _kss()
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=nx + nsteps, kmax=6)
    lats = []
    for _ in range(2):
        lat = kss.Lattice(nx, ny, precision=prec, tau=0.62, output_every=every,
                          record=("kl",), rho0=1.5)
        lat.set_fields(rho, ux, uy)
        lats.append(lat)
    lats[0].step(nsteps)
    for _ in range(nsteps):
        lats[1].step(1)
    a, b = lats
    assert a.step_count == b.step_count == nsteps
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    if every:
        fa, ta, ca = a.read_flags()
        fb, tb, cb = b.read_flags()
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(ta, tb)
        np.testing.assert_array_equal(ca, cb)
        np.testing.assert_array_equal(a.read_stats()[0], b.read_stats()[0])
        np.testing.assert_array_equal(a.read_sensor("kl"), b.read_sensor("kl"))
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("prec,every", [("fp32", 0), ("fp64", 0), ("fp16dev", 0), ("fp32", 3),
                                        ("fp64", 4)])
def test_runs_of_steps_replayed_as_graphs(prec, every):
    """kss_step(n) that is not one multi-step launch replays one recorded graph per
    (n, buffer, output phase): the same calls repeated (recorded, then replayed) equal
    single steps bit for bit, outputs included; a run longer than one graph (512 steps)
    goes in chunks of whole output periods."""
    kss = _kss()
    nx, ny = 96, 70
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=23, kmax=4)
    a = kss.Lattice(nx, ny, precision=prec, tau=0.7, output_every=every, record=("kl",))
    b = kss.Lattice(nx, ny, precision=prec, tau=0.7, output_every=every, record=("kl",))
    for lat in (a, b):
        lat.set_fields(rho, ux, uy)
    for n in (5, 5, 3, 5, 5, 2, 1100):
        a.step(n)
        for _ in range(n):
            b.step(1)
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())
        for x, y in zip(a.read_flags(), b.read_flags()):
            np.testing.assert_array_equal(x, y)
        sa, sb = a.read_stats(), b.read_stats()
        np.testing.assert_array_equal(sa[0], sb[0])
        assert sa[2] == sb[2]
        np.testing.assert_array_equal(a.read_sensor("kl"), b.read_sensor("kl"))
    assert a.step_count == b.step_count == 1125
    a.close()
    b.close()
