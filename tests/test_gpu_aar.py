"""GPU: adaptive algorithm refinement (kss_config.tau2 > 0) against the oracle -- the
two-relaxation collision in the switched region (oracle.collide_aar), the region
schedule of output steps (oracle.run_aar) and the quasi-equilibrium sensor of the model.
Tolerances as tests/parity.py; the qe sensor takes the neq scale (rho)."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

ALL = tuple(parity.SENSORS)


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


def _state(nx, ny, seed, tau, steps=6):
    r, u, v = inputs.smooth_jump(nx, ny, seed=seed, kmax=4)
    return oracle.step(oracle.init_equilibrium(r, u, v), tau, steps)


def _split(values):
    """A threshold between the two middle values of a sensor field (no cell on it)."""
    v = np.sort(values.ravel())
    k = v.size // 2
    return float(0.5 * (v[max(k - 1, 0)] + v[k])) if v.size > 1 else float(0.5 * v[0])


def _check_outputs(lat, prec, X, tau, thr_r, thr_s, tile, switch, names, nsteps=0):
    """Sensors (qe of the two-relaxation model), flags and counts of the step from X
    (the state after nsteps - 1 steps)."""
    ref, nonpos = oracle.sensor_fields(X, tau, pull=True, two_relax=True)
    ft = oracle.stream(X)
    r, u, v = oracle.moments(ft)
    kn = ref[oracle.SENSOR_ID["kn"]]
    for name in names:
        parity.assert_sensor_close(name, lat.read_sensor(name), ref[oracle.SENSOR_ID[name]],
                                   prec, nsteps, r, u, v, kn, tau, ft=ft, two_relax=True)
    er, es = ref[oracle.SENSOR_ID["kn"]], ref[oracle.SENSOR_ID[switch]]
    rf, rt, rc = oracle.flags(er, thr_r, es, thr_s, nonpos, tile)
    flags, tiles, counts = lat.read_flags()
    band = parity.band_mask(er, thr_r, es, thr_s)
    parity.assert_flags_match(flags, tiles, counts, rf, rt, rc, band, tile)
    return flags


@pytest.mark.parametrize("nx,ny,tile", [(37, 21, 16), (130, 67, 8), (5, 1, 8), (1, 5, 8),
                                        (200, 9, 32)])
@pytest.mark.parametrize("outputs", ["plain", "std", "std_qe", "full"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_one_step_in_a_prescribed_region(prec, outputs, nx, ny, tile):
    """kss_set_aar_region, then one step of each kernel variant (no outputs; the
    {Kn, KL, neq} set with neq as the switch sensor; the same set plus qe, computed in the
    fused pair loop, as the switch; all of Table 1 with qe as the switch) against
    oracle.collide_aar; the output step's switch flags become the region."""
    kss = _kss()
    tau, tau2 = 0.7, 1.35
    X = _state(nx, ny, seed=7 * nx + ny, tau=tau)
    reg = inputs.random_region(nx, ny, seed=nx + 3 * ny)
    ref0, _ = oracle.sensor_fields(X, tau, pull=True, two_relax=True)
    switch = "neq" if outputs == "std" else "qe"
    thr_r, thr_s = 1e-3, _split(ref0[oracle.SENSOR_ID[switch]])
    kw = {"plain": dict(output_every=0, record=()),
          "std": dict(output_every=1, record=("kn", "kl", "neq")),
          "std_qe": dict(output_every=1, record=("kn", "qe")),
          "full": dict(output_every=1, record=ALL)}[outputs]
    lat = kss.Lattice(nx, ny, precision=prec, tau=tau, tau2=tau2, tile=tile,
                      refine_threshold=thr_r, switch_sensor=switch, switch_threshold=thr_s,
                      **kw)
    lat.set_populations(X)
    np.testing.assert_array_equal(lat.get_aar_region(), np.zeros((ny, nx), np.uint8))
    lat.set_aar_region(reg)
    np.testing.assert_array_equal(lat.get_aar_region(), (reg != 0).astype(np.uint8))
    lat.step(1)
    got = lat.get_populations()
    want = oracle.collide_aar(oracle.stream(X), tau, tau2, reg)
    u = parity.UNIT_ROUNDOFF[prec]
    assert np.max(np.abs(got - want) / want) <= 64 * u * math.sqrt(2)
    # the test can tell the models apart: in switched cells the BGK step is far off
    bgk = oracle.step(X, tau)
    if np.any(reg):
        sw = np.broadcast_to(reg != 0, want.shape)
        assert np.max(np.abs(bgk - want)[sw] / want[sw]) > 10 * 64 * u
    if outputs == "plain":
        np.testing.assert_array_equal(lat.get_aar_region(), (reg != 0).astype(np.uint8))
    else:
        names = {"std": ("kn", "kl", "neq"), "std_qe": ("kn", "qe", "kl")}.get(outputs, ALL)
        flags = _check_outputs(lat, prec, X, tau, thr_r, thr_s, tile, switch, names)
        np.testing.assert_array_equal(lat.get_aar_region(), (flags >> 1) & 1)
    lat.close()


@pytest.mark.parametrize("switch", ["qe", "neq"])
@pytest.mark.parametrize("every", [1, 3])
def test_schedule_against_the_oracle_fp64(switch, every):
    """12 steps from an empty region: every output step's switch flags rule the following
    steps (oracle.run_aar).  FP64: every switch decision of the oracle lies far outside
    the library's rounding, so regions must agree exactly."""
    kss = _kss()
    nx, ny, tau, tau2, n, tile = 96, 80, 0.62, 1.1, 12, 16
    X = _state(nx, ny, seed=41, tau=tau)
    ref0, _ = oracle.sensor_fields(X, tau, pull=True, two_relax=True)
    thr = _split(ref0[oracle.SENSOR_ID[switch]])
    res = oracle.run_aar(X, tau, tau2, n, output_every=every, switch=(switch, thr),
                         refine=("kn", 1e-3), tile=tile)
    assert res["switch_margin"] > 1e-9 * thr
    assert 0 < res["region"].sum() < nx * ny
    lat = kss.Lattice(nx, ny, precision="fp64", tau=tau, tau2=tau2, tile=tile,
                      switch_sensor=switch, switch_threshold=thr, output_every=every,
                      record=("qe", "kl"))
    lat.set_populations(X)
    lat.step(n)
    got = lat.get_populations()
    u = parity.UNIT_ROUNDOFF["fp64"]
    assert np.max(np.abs(got - res["f"]) / res["f"]) <= 64 * u * math.sqrt(n + 1)
    np.testing.assert_array_equal(lat.get_aar_region(), res["region"])
    flags, tiles, counts = lat.read_flags()
    band = parity.band_mask(res["sensors"][oracle.SENSOR_ID["kn"]], 1e-3,
                            res["sensors"][oracle.SENSOR_ID[switch]], thr)
    parity.assert_flags_match(flags, tiles, counts, res["flags"], res["tiles"], res["counts"],
                              band, tile)
    ft = oracle.stream(oracle.run_aar(X, tau, tau2, n - 1, output_every=every,
                                      switch=(switch, thr), tile=tile)["f"])
    r, vx, vy = oracle.moments(ft)
    kn = res["sensors"][oracle.SENSOR_ID["kn"]]
    for name in ("qe", "kl"):
        parity.assert_sensor_close(name, lat.read_sensor(name),
                                   res["sensors"][oracle.SENSOR_ID[name]], "fp64", n, r, vx,
                                   vy, kn, tau, two_relax=True)
    sums, _, step = lat.read_stats()
    assert step == n
    assert np.all(np.abs(sums - res["sums"]) <= 64 * u * math.sqrt(n + 1) * res["sums"][0])
    lat.close()


def test_fp32_trajectory_in_a_prescribed_region():
    """20 FP32 steps with a fixed region (no output steps until the last) against the
    FP64 oracle; the last step's flags rule the region afterwards."""
    kss = _kss()
    nx, ny, tau, tau2, n, tile = 130, 67, 0.8, 0.6, 20, 16
    X = _state(nx, ny, seed=5, tau=tau)
    reg = inputs.random_region(nx, ny, seed=77, frac=0.5)
    lat = kss.Lattice(nx, ny, precision="fp32", tau=tau, tau2=tau2, tile=tile,
                      output_every=n, record=("kn", "neq"))
    lat.set_populations(X)
    lat.set_aar_region(reg)
    lat.step(n)
    f = X
    for _ in range(n - 1):
        f = oracle.step_aar(f, tau, tau2, reg)
    want = oracle.step_aar(f, tau, tau2, reg)
    got = lat.get_populations()
    u = parity.UNIT_ROUNDOFF["fp32"]
    assert np.max(np.abs(got - want) / want) <= 64 * u * math.sqrt(n + 1)
    flags = _check_outputs(lat, "fp32", f, tau, 1e-3, 1e-4, tile, "neq", ("kn", "neq"), n)
    np.testing.assert_array_equal(lat.get_aar_region(), (flags >> 1) & 1)
    lat.close()


def test_fp16_deviations_one_step_against_the_oracle_codec():
    """FP16 deviation storage: from a state both sides store exactly, one step in a
    prescribed region agrees with the oracle's step rounded by the oracle's codec within
    one binary16 quantum of the code plus a few FP32 roundings."""
    from tests.test_gpu_fp16dev import K, _quantum, _stored_state

    kss = _kss()
    nx, ny, tau, tau2 = 130, 67, 0.75, 1.2
    X = _stored_state(nx, ny, seed=19, tau=tau)
    reg = inputs.random_region(nx, ny, seed=19)
    lat = kss.Lattice(nx, ny, precision="fp16dev", tau=tau, tau2=tau2, dev_exp=K,
                      output_every=0)
    lat.set_populations(X)
    lat.set_aar_region(reg)
    lat.step(1)
    got = lat.get_populations()
    fo = oracle.step_aar(X, tau, tau2, reg)
    ho = oracle.dev16_encode(fo, rho0=1.0, dev_exp=K)
    want = oracle.dev16_decode(ho, rho0=1.0, dev_exp=K)
    bound = _quantum(ho) + 8 * 2.0**-24 * np.abs(want)
    assert np.all(np.abs(got - want) <= bound)
    assert np.mean(got == want) > 0.95
    lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
@pytest.mark.parametrize("every", [1, 0])
def test_empty_region_is_bgk_bit_for_bit(prec, every):
    """With the switch off the region stays empty, and the two-relaxation kernels give
    the BGK populations of a lattice without the model, bit for bit."""
    kss = _kss()
    nx, ny = 150, 70
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=3, kmax=6)
    states = []
    for tau2 in (0.0, 0.9):
        lat = kss.Lattice(nx, ny, precision=prec, tau=0.62, tau2=tau2, switch_threshold=-1.0,
                          output_every=every)
        lat.set_fields(rho, ux, uy)
        lat.step(9)
        states.append(lat.get_populations())
        if tau2:
            assert not lat.get_aar_region().any()
        lat.close()
    np.testing.assert_array_equal(states[0], states[1])


@pytest.mark.parametrize("switch", ["neq", "qe"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_deferred_cells_write_the_region(prec, switch):
    """Far from equilibrium (populations perturbed by up to 30 %) the {Kn, KL, neq} step
    defers most cells to its exact recomputation, which decides their switch flags after
    the rows were stored: the region must still be the step's switch flags."""
    kss = _kss()
    nx, ny, tau, tau2 = 128, 96, 0.7, 1.25
    rng = np.random.default_rng(321)
    rho, ux, uy = inputs.random_smooth(nx, ny, seed=8)
    f = oracle.init_equilibrium(rho, ux, uy) * (1.0 + 0.3 * rng.uniform(-1, 1, (9, ny, nx)))
    reg = inputs.random_region(nx, ny, seed=321)
    ref, _ = oracle.sensor_fields(f, tau, pull=True, two_relax=True)
    thr_r, thr_s = 0.5, _split(ref[oracle.SENSOR_ID[switch]])
    lat = kss.Lattice(nx, ny, precision=prec, tau=tau, tau2=tau2, refine_threshold=thr_r,
                      switch_sensor=switch, switch_threshold=thr_s,
                      record=("kl", "kn", "neq", "qe"))
    lat.set_populations(np.ascontiguousarray(f))
    lat.set_aar_region(reg)
    lat.step(1)
    want = oracle.collide_aar(oracle.stream(f), tau, tau2, reg)
    u = parity.UNIT_ROUNDOFF[prec]
    got = lat.get_populations()
    assert np.max(np.abs(got - want) / np.abs(want)) <= 64 * u * math.sqrt(2)
    flags = _check_outputs(lat, prec, f, tau, thr_r, thr_s, 16, switch,
                           ("kn", "kl", "neq", "qe"))
    region = lat.get_aar_region()
    np.testing.assert_array_equal(region, (flags >> 1) & 1)
    assert 0 < region.sum() < nx * ny
    lat.close()


def test_region_api():
    kss = _kss()
    nx, ny = 40, 24
    reg = inputs.random_region(nx, ny, seed=1)
    with kss.Lattice(nx, ny, precision="fp32", tau=0.8) as lat:
        for call in (lambda: lat.set_aar_region(reg), lambda: lat.get_aar_region()):
            with pytest.raises(kss.KssError) as e:
                call()
            assert e.value.code == -5
    with kss.Lattice(nx, ny, precision="fp32", tau=0.8, tau2=1.0) as lat:
        lat.set_aar_region(reg)
        np.testing.assert_array_equal(lat.get_aar_region(), (reg != 0).astype(np.uint8))
        r, u, v = inputs.random_smooth(nx, ny, seed=1)
        lat.set_fields(r, u, v)  # a new state starts with an empty region
        assert not lat.get_aar_region().any()
        import torch

        dev = torch.from_numpy(reg).cuda()
        lat.set_aar_region(dev)
        out = lat.get_aar_region(device=True)
        np.testing.assert_array_equal(out.cpu().numpy(), (reg != 0).astype(np.uint8))


@pytest.mark.parametrize("prec,every", [("fp32", 1), ("fp32", 3), ("fp64", 1),
                                        ("fp16dev", 2)])
def test_batch_members_with_and_without_the_model(prec, every):
    """A batch mixing AAR members (prescribed regions, neq or qe as the switch) and BGK
    members, all with one output cadence: every member equals the same lattice stepped
    alone, bit for bit (populations, flags, regions).  Mixed cadences are refused."""
    kss = _kss()
    specs = [dict(nx=37, ny=21, tau=0.7, tau2=1.3, switch_sensor="qe"),
             dict(nx=130, ny=67, tau=1.0),
             dict(nx=64, ny=64, tau=0.55, tau2=0.9),
             dict(nx=200, ny=9, tau=0.6, tau2=2.0, record=("kl", "qe")),
             dict(nx=5, ny=1, tau=1.3)]
    thr = {"qe": 2e-4, "neq": 1e-3}
    for sp in specs:
        sp.setdefault("switch_sensor", "neq")
        sp["switch_threshold"] = thr[sp["switch_sensor"]]
        sp["output_every"] = every
    with pytest.raises(kss.KssError) as e:
        kss.Batch([dict(specs[0]), dict(specs[1], output_every=every + 1)], precision=prec)
    assert e.value.code == -6
    b = kss.Batch(specs, precision=prec)
    singles = []
    for k, sp in enumerate(specs):
        fld = inputs.smooth_jump(sp["nx"], sp["ny"], seed=60 + k, kmax=4)
        lat = kss.Lattice(precision=prec, **sp)
        for x in (b[k], lat):
            x.set_fields(*fld)
            if sp.get("tau2"):
                x.set_aar_region(inputs.random_region(sp["nx"], sp["ny"], seed=k))
        singles.append(lat)
    for n in (7, 1, 5):
        b.step(n)
        for lat in singles:
            lat.step(n)
        for k, sp in enumerate(specs):
            a, c = b[k], singles[k]
            np.testing.assert_array_equal(a.get_populations(), c.get_populations())
            np.testing.assert_array_equal(a.read_flags()[0], c.read_flags()[0])
            if sp.get("tau2"):
                np.testing.assert_array_equal(a.get_aar_region(), c.get_aar_region())
    if every > 1:  # a member set again is out of phase with the others
        b[1].set_fields(*inputs.smooth_jump(130, 67, seed=61, kmax=4))
        with pytest.raises(kss.KssError) as e:
            b.step(1)
        assert e.value.code == -5
    for lat in singles:
        lat.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("switch", ["neq", "qe"])
@pytest.mark.parametrize("nx,ny,n", [(37, 21, 6), (1024, 640, 7)])
def test_multi_step_launch_equals_single_steps(prec, switch, nx, ny, n):
    """kss_step(n) of an AAR lattice with every step an output step runs as one
    cooperative multi-step launch: a block reads the region its own block wrote at the
    previous step (possibly in another CTA).  It must equal n single launches bit for bit:
    populations, regions, flags, counts, sums and the recorded fields."""
    kss = _kss()
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=nx + n, kmax=6)
    sens, _ = oracle.sensor_fields(oracle.init_equilibrium(rho, ux, uy), 0.62, pull=True,
                                   two_relax=True)
    thr = _split(sens[oracle.SENSOR_ID[switch]])  # about half the cells switch
    lats = []
    for _ in range(2):
        lat = kss.Lattice(nx, ny, precision=prec, tau=0.62, tau2=1.4, switch_sensor=switch,
                          switch_threshold=thr, record=("kl", "qe"))
        lat.set_fields(rho, ux, uy)
        lat.set_aar_region(inputs.random_region(nx, ny, seed=n))
        lats.append(lat)
    lats[0].step(n)
    for _ in range(n):
        lats[1].step(1)
    a, b = lats
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    np.testing.assert_array_equal(a.get_aar_region(), b.get_aar_region())
    assert 0 < a.get_aar_region().sum() < nx * ny
    for x, y in zip(a.read_flags(), b.read_flags()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.read_stats()[0], b.read_stats()[0])
    for name in ("kl", "qe"):
        np.testing.assert_array_equal(a.read_sensor(name), b.read_sensor(name))
    for lat in lats:
        lat.close()
