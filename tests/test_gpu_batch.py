"""GPU: batches of uneven lattices advanced by one launch per step (kss_batch_*).

Every member of a batch must give exactly what the same lattice gives stepped alone
(populations, sensors, flags, tile counts and counts bit for bit; conservation sums
bit for bit at the default CTA height, within the FP rounding bound otherwise), and
the small members are also checked against the FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu


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


# uneven members: ragged widths and heights, a 1-wide and a 1-high lattice, tiles 8/16
SPECS = [
    dict(nx=37, ny=21, tau=0.7, tile=16, output_every=1),
    dict(nx=130, ny=67, tau=1.0, tile=16, output_every=2),
    dict(nx=64, ny=64, tau=0.55, tile=8, output_every=1),
    dict(nx=200, ny=9, tau=0.6, tile=16, output_every=1, record=("kl", "neq")),
    dict(nx=1, ny=5, tau=0.8, tile=8, output_every=1),
    dict(nx=300, ny=260, tau=0.9, tile=16, output_every=4),
    dict(nx=5, ny=1, tau=1.3, tile=8, output_every=1),
]


def _fields(sp, k):
    return inputs.random_smooth(sp["nx"], sp["ny"], seed=100 + k, kmax=4, mach=0.1)


def _singles(specs, prec):
    kss = _kss()
    lats = []
    for k, sp in enumerate(specs):
        lat = kss.Lattice(precision=prec, **sp)
        lat.set_fields(*_fields(sp, k))
        lats.append(lat)
    return lats


def _batch(specs, prec):
    kss = _kss()
    b = kss.Batch(specs, precision=prec)
    for k, sp in enumerate(specs):
        b[k].set_fields(*_fields(sp, k))
    return b


def _assert_same(a, b, sums_exact=True, prec="fp32", nsteps=1):
    """Member a and single lattice b describe the same step identically."""
    assert a.step_count == b.step_count
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    fa, ta, ca = a.read_flags()
    fb, tb, cb = b.read_flags()
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(ta, tb)
    np.testing.assert_array_equal(ca, cb)
    sa, _, stepa = a.read_stats()
    sb, _, stepb = b.read_stats()
    assert stepa == stepb
    if sums_exact:
        np.testing.assert_array_equal(sa, sb)
    else:
        tol = 64 * parity.UNIT_ROUNDOFF[prec] * math.sqrt(nsteps + 1) * abs(sb[0])
        assert np.all(np.abs(sa - sb) <= tol), (sa, sb)
    for name in ("kl", "kn", "alpha"):
        np.testing.assert_array_equal(a.read_sensor(name), b.read_sensor(name))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_members_equal_single_lattices(prec):
    b = _batch(SPECS, prec)
    singles = _singles(SPECS, prec)
    b.step(7)      # one captured graph of 7 launches
    b.step(1)      # a direct launch
    for lat in singles:
        lat.step(8)
    for k in range(len(SPECS)):
        _assert_same(b[k], singles[k])
    b.step(4)
    for lat in singles:
        lat.step(4)
    for k in range(len(SPECS)):
        _assert_same(b[k], singles[k])
    for lat in singles:
        lat.close()
    b.close()


def test_members_with_all_sensors_run_their_own_sets():
    """A member recording all-sensor fields makes output steps launch the all-sensor
    kernel; every other member still runs its {Kn, KL, neq} path: all equal to their
    single-lattice runs bit for bit."""
    specs = SPECS[:4] + [dict(nx=90, ny=40, tau=0.75, tile=16, output_every=1,
                              record=("alpha", "tau_ns", "kl"))]
    b = _batch(specs, "fp32")
    singles = _singles(specs, "fp32")
    b.step(5)
    for lat in singles:
        lat.step(5)
    for k in range(len(specs)):
        _assert_same(b[k], singles[k])
        np.testing.assert_array_equal(b[k].read_sensor("neq"), singles[k].read_sensor("neq"))
    np.testing.assert_array_equal(b[4].read_sensor("tau_ns"), singles[4].read_sensor("tau_ns"))
    for lat in singles:
        lat.close()
    b.close()


def test_batch_members_against_the_oracle():
    specs = SPECS[:4]
    nsteps = 12
    b = _batch(specs, "fp32")
    b.step(nsteps)
    for k, sp in enumerate(specs):
        rho, ux, uy = _fields(sp, k)
        f = oracle.init_equilibrium(rho, ux, uy)
        for _ in range(nsteps - 1):
            f = oracle.step(f, sp["tau"])
        prev = f
        ref, nonpos = oracle.sensor_fields(prev, sp["tau"], pull=True)
        ft = oracle.stream(prev)
        r, u, v = oracle.moments(ft)
        kn = ref[oracle.SENSOR_ID["kn"]]
        for name in ("kn", "kl", "neq", "tau_ns", "alpha"):
            sid = oracle.SENSOR_ID[name]
            parity.assert_sensor_close(name, b[k].read_sensor(name), ref[sid], "fp32", nsteps,
                                       r, u, v, kn, sp["tau"], ft=ft)
        er, es = ref[oracle.SENSOR_ID["kn"]], ref[oracle.SENSOR_ID["neq"]]
        rf, rt, rcnt = oracle.flags(er, 1e-3, es, 1e-4, nonpos, sp["tile"])
        flags, tiles, counts = b[k].read_flags()
        band = parity.band_mask(er, 1e-3, es, 1e-4)
        parity.assert_flags_match(flags, tiles, counts, rf, rt, rcnt, band, sp["tile"])
        fin = oracle.step(prev, sp["tau"])
        rr, ru, rv = oracle.moments(fin)
        gr, gu, gv = b[k].read_moments()
        assert np.max(np.abs(gr - rr) / rr) <= 1e-5
    b.close()


@pytest.mark.parametrize("rows", [16, 32, 64])
@pytest.mark.parametrize("ctas_per_sm,graph", [(0, 1), (1, 0), (3, 1)])
def test_batch_tunings_give_the_same_states(rows, ctas_per_sm, graph):
    specs = [dict(sp, tile=min(sp["tile"], 16)) for sp in SPECS]
    b = _batch(specs, "fp32")
    b.set_tuning(rows=rows, ctas_per_sm=ctas_per_sm, graph=graph)
    assert b.tuning["rows"] == rows and b.tuning["ctas_per_sm"] == ctas_per_sm
    singles = _singles(specs, "fp32")
    b.step(6)
    for lat in singles:
        lat.step(6)
    for k in range(len(specs)):
        # the default CTA height of the single-lattice step is 32 rows
        _assert_same(b[k], singles[k], sums_exact=(rows == 32), nsteps=6)
    for lat in singles:
        lat.close()
    b.close()


def test_invalid_tunings_are_rejected():
    kss = _kss()
    b = _batch([dict(nx=40, ny=40, tau=0.8, tile=32)], "fp32")
    for kw in (dict(rows=16), dict(rows=48), dict(ctas_per_sm=-1), dict(graph=2)):
        with pytest.raises(kss.KssError) as e:
            b.set_tuning(**kw)
        assert e.value.code == -1
    b.close()
    with pytest.raises(kss.KssError):
        kss.Batch([dict(nx=8, ny=8), dict(nx=8, ny=8, precision="fp64")])


def test_member_stepped_alone_between_batched_steps():
    specs = SPECS[:4]
    b = _batch(specs, "fp32")
    singles = _singles(specs, "fp32")
    b.step(3)
    b[1].step(1)           # flips member 1's buffers behind the batch's back
    b.step(2)
    b[2].step(3)
    b.step(1)
    for k, lat in enumerate(singles):
        lat.step(6 + (1 if k == 1 else 0) + (3 if k == 2 else 0))
    for k in range(len(specs)):
        _assert_same(b[k], singles[k])
    for lat in singles:
        lat.close()
    b.close()


def test_autotune_keeps_states_and_uses_its_cache(tmp_path):
    kss = _kss()
    cache = str(tmp_path / "tune.txt")
    specs = SPECS[:5]
    b = _batch(specs, "fp32")
    singles = _singles(specs, "fp32")
    b[0].read_sensor("kn")          # step-0 outputs exist before the timed launches
    t = b.autotune(cache, steps=3)
    assert t["rows"] in (16, 32, 64) and t["ctas_per_sm"] in (0, 2, 3, 4)
    assert t["ms_per_step"] > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].count("\t") == 4
    # the stored states are unchanged and the step-0 outputs are evaluated again
    for k in range(len(specs)):
        _assert_same(b[k], singles[k])
    b.step(5)
    for lat in singles:
        lat.step(5)
    for k in range(len(specs)):
        _assert_same(b[k], singles[k], sums_exact=(t["rows"] == 32), nsteps=5)
    # after a step the timed launches would overwrite the previous state: refused
    with pytest.raises(kss.KssError) as e:
        b.autotune(cache, steps=3)
    assert e.value.code == -5
    b.close()
    # a second batch of the same shape takes the cached choice without timing
    b2 = _batch(specs, "fp32")
    t2 = b2.autotune(cache, steps=3)
    assert (t2["rows"], t2["ctas_per_sm"], t2["multi_step"]) == (t["rows"], t["ctas_per_sm"],
                                                                 t["multi_step"])
    assert t2["ms_per_step"] == pytest.approx(t["ms_per_step"], rel=1e-6)
    assert len(open(cache).read().splitlines()) == 1
    b2.close()
    for lat in singles:
        lat.close()


def test_seeded_64_lattice_workload():
    """The 64 uneven lattices (sizes 64^2..1024^2, tau ~ U[0.51, 1.5], Mach ~ U[0.01,
    0.15], seed 13618): 10 batched steps equal 10 steps of each lattice alone, and the
    64^2 members match the oracle."""
    kss = _kss()
    specs = inputs.batch_specs()
    cfgs = [dict(nx=s, ny=s, tau=tau) for s, tau, _, _ in specs]
    b = kss.Batch(cfgs, precision="fp32")
    for k, (s, tau, mach, fs) in enumerate(specs):
        b[k].set_fields(*inputs.batch_fields(s, mach, fs))
    b.step(10)
    for k, (s, tau, mach, fs) in enumerate(specs):
        lat = kss.Lattice(s, s, precision="fp32", tau=tau)
        lat.set_fields(*inputs.batch_fields(s, mach, fs))
        lat.step(10)
        np.testing.assert_array_equal(b[k].get_populations(), lat.get_populations())
        fa, ta, ca = b[k].read_flags()
        fb, tb, cb = lat.read_flags()
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(ta, tb)
        np.testing.assert_array_equal(b[k].read_stats()[0], lat.read_stats()[0])
        lat.close()
        if s == 64:
            f = oracle.init_equilibrium(*inputs.batch_fields(s, mach, fs))
            for _ in range(10):
                f = oracle.step(f, tau)
            rr, ru, rv = oracle.moments(f)
            gr, gu, gv = b[k].read_moments()
            assert np.max(np.abs(gr - rr) / rr) <= 1e-5
            umax = np.max(np.hypot(ru, rv))
            assert np.max(np.abs(gr * gu - rr * ru)) <= 1e-5 * np.max(rr) * umax
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp16dev"])
@pytest.mark.parametrize("rows", [16, 32, 64])
def test_multi_step_batch_equals_per_step_launches(prec, rows):
    """Every member an output step of the {Kn, KL, neq} set: kss_batch_step(n) runs all n
    steps as one cooperative launch (multi_step = 1) and must give, member by member, the
    results of one launch per step (multi_step = 0) bit for bit, and those of the member
    stepped alone at its default CTA height (a lone FP16-deviation lattice takes eight
    cells per lane, CTA blocks 256 columns wide, so its conservation sums are added in
    another order: equal within the rounding bound)."""
    specs = [dict(sp, output_every=1, tile=min(sp["tile"], 16)) for sp in SPECS]
    a = _batch(specs, prec)
    b = _batch(specs, prec)
    a.set_tuning(rows=rows, multi_step=1)
    b.set_tuning(rows=rows, multi_step=0)
    singles = _singles(specs, prec)
    for n in (9, 1, 4):  # multi-step, single launch, multi-step again
        a.step(n)
        b.step(n)
        for lat in singles:
            lat.step(n)
        for k in range(len(specs)):
            _assert_same(a[k], b[k])
            _assert_same(a[k], singles[k], sums_exact=(rows == 32 and prec != "fp16dev"),
                         prec="fp64" if prec == "fp64" else "fp32", nsteps=14)
    for lat in singles:
        lat.close()
    a.close()
    b.close()


def test_multi_step_batch_of_the_seeded_workload_shapes():
    """The 64-lattice workload's member shapes (64^2 .. 1024^2) in one multi-step launch
    against one launch per step, 12 steps."""
    kss = _kss()
    shapes = inputs.batch_specs(24)
    specs = [dict(nx=size, ny=size, tau=tau) for size, tau, _, _ in shapes]
    fields = [inputs.batch_fields(size, mach, seed) for size, _, mach, seed in shapes]
    runs = []
    for multi in (1, 0):
        bt = kss.Batch(specs, precision="fp32", record=("kl",))
        bt.set_tuning(multi_step=multi)
        for k, f in enumerate(fields):
            bt[k].set_fields(*f)
        bt.step(12)
        runs.append(bt)
    for k in range(len(specs)):
        _assert_same(runs[0][k], runs[1][k])
    for bt in runs:
        bt.close()


def test_autotune_times_multi_step_launches_and_restores_the_states(tmp_path):
    """Every member an output step every step: the tuner also times multi-step launches
    (which advance the states) at each CTA height and restores the stored states."""
    specs = [dict(sp, output_every=1, tile=min(sp["tile"], 16)) for sp in SPECS]
    b = _batch(specs, "fp32")
    singles = _singles(specs, "fp32")
    t = b.autotune(str(tmp_path / "tune.txt"), steps=4)
    assert t["multi_step"] in (0, 1) and t["ms_per_step"] > 0
    for k in range(len(specs)):
        np.testing.assert_array_equal(b[k].get_populations(), singles[k].get_populations())
    b.step(6)
    for lat in singles:
        lat.step(6)
    for k in range(len(specs)):
        _assert_same(b[k], singles[k], sums_exact=(t["rows"] == 32), nsteps=6)
    for lat in singles:
        lat.close()
    b.close()
