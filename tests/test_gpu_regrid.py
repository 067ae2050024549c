"""GPU: regridding on the flags (kss_regrid, kss_regrid_flags) against the oracle's
buffered tile mask and Berger-Rigoutsos clustering (oracle/regrid.py): integer work,
compared bit for bit (the boxes as ordered lists)."""
import time

import numpy as np
import pytest

import oracle
from oracle import regrid as orc_regrid
from paper_2603_13618_gb300 import inputs

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


def _blobs(ny, nx, seed, nblobs=6, noise=0.0005):
    """Synthetic refine flags: a few filled ellipses and scattered single cells, plus
    switch and non-positive bits that must not count."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx]
    f = np.zeros((ny, nx), dtype=np.uint8)
    for _ in range(nblobs):
        cy, cx = rng.uniform(0, ny), rng.uniform(0, nx)
        ry, rx = rng.uniform(1.0, max(1.5, ny / 6)), rng.uniform(1.0, max(1.5, nx / 6))
        f[((y - cy) / ry) ** 2 + ((x - cx) / rx) ** 2 <= 1] |= 1
    f[rng.random((ny, nx)) < noise] |= 1
    f[rng.random((ny, nx)) < 0.01] |= 2
    f[rng.random((ny, nx)) < 0.001] |= 128
    return f


@pytest.mark.parametrize("ny,nx,tile,buf,eff", [
    (96, 130, 8, 2, 0.98), (200, 64, 16, 2, 0.7), (37, 21, 8, 0, 0.5), (1, 300, 8, 2, 0.9),
    (256, 256, 16, 3, 1.0), (512, 384, 8, 2, 0.98), (64, 64, 32, 1, 0.0)])
def test_regrid_flags_equals_the_oracle(ny, nx, tile, buf, eff):
    kss = _kss()
    for seed in range(3):
        flags = _blobs(ny, nx, seed=seed + nx)
        want_mask = orc_regrid.tile_mask(flags, tile, buf)
        want = orc_regrid.cluster(want_mask, eff)
        got, mask = kss.regrid_flags(flags, tile=tile, buffer=buf, efficiency=eff)
        np.testing.assert_array_equal(mask, want_mask)
        assert got == want


def test_empty_and_full_flag_fields():
    kss = _kss()
    got, mask = kss.regrid_flags(np.zeros((50, 70), dtype=np.uint8), tile=8)
    assert got == [] and not mask.any()
    got, mask = kss.regrid_flags(np.ones((50, 70), dtype=np.uint8), tile=8)
    assert got == [(0, 0, 9, 7)] and mask.all()


def test_box_capacity_and_arguments():
    kss = _kss()
    flags = _blobs(128, 128, seed=4, nblobs=12, noise=0.002)
    full, _ = kss.regrid_flags(flags, tile=8, efficiency=1.0)
    assert len(full) > 3
    part, _ = kss.regrid_flags(flags, tile=8, efficiency=1.0, max_boxes=3)
    assert part == full[:3]
    with pytest.raises(kss.KssError):
        kss.regrid_flags(flags, tile=12)
    with pytest.raises(kss.KssError):
        kss.regrid_flags(flags, tile=8, efficiency=1.5)


def test_lattice_regrid_on_an_oracle_state():
    """The lattice's own step: its flags agree with the oracle's away from the threshold
    band (the thresholds are chosen far from the sensor values here), and its regrid
    equals the oracle's regrid of the oracle's flags."""
    kss = _kss()
    nx, ny, tau, tile = 160, 96, 0.7, 8
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=9, kmax=4)
    f = oracle.step(oracle.init_equilibrium(rho, ux, uy), tau, 10)
    ref, nonpos = oracle.sensor_fields(f, tau, pull=True)
    kn = ref[oracle.SENSOR_ID["kn"]]
    thr = float(np.quantile(kn, 0.9))
    # a threshold in a gap of the Kn values, so both sides tag the same cells
    srt = np.sort(kn.ravel())
    gaps = np.diff(srt)
    k = int(np.argmax(gaps * (srt[1:] > thr)))
    thr = 0.5 * (srt[k] + srt[k + 1])
    assert gaps[k] > 1e-6 * thr
    oflags, _, _ = oracle.flags(kn, thr, ref[oracle.SENSOR_ID["neq"]], -1.0, nonpos, tile)
    lat = kss.Lattice(nx, ny, precision="fp64", tau=tau, tile=tile, refine_threshold=thr,
                      switch_threshold=-1.0)
    lat.set_populations(f)
    lat.step(1)
    np.testing.assert_array_equal(lat.read_flags()[0] & 1, oflags & 1)
    got, mask = lat.regrid(buffer=2, efficiency=0.9)
    want_mask = orc_regrid.tile_mask(oflags, tile, 2)
    np.testing.assert_array_equal(mask, want_mask)
    assert got == orc_regrid.cluster(want_mask, 0.9)
    lat.close()


def test_regrid_of_the_4096_workload():
    """The headline workload after 100 steps: 4096^2, tile 16 (256^2 tiles), buffer 2,
    efficiency 0.98: the boxes cover the marked tiles of the returned mask, are disjoint
    and meet the efficiency; the time of one regrid is printed."""
    kss = _kss()
    n = 4096
    rho, ux, uy = inputs.smooth_jump(n, n, seed=2603, kmax=8)
    lat = kss.Lattice(n, n, precision="fp32", tau=0.6)
    lat.set_fields(rho, ux, uy)
    lat.step(100)
    lat.regrid()
    t0 = time.perf_counter()
    boxes, mask = lat.regrid(buffer=2, efficiency=0.98)
    dt = time.perf_counter() - t0
    cover = np.zeros(mask.shape, dtype=np.int64)
    for (x0, y0, x1, y1) in boxes:
        cover[y0:y1, x0:x1] += 1
        assert mask[y0:y1, x0:x1].sum() >= 0.98 * (x1 - x0) * (y1 - y0) or (x1 - x0, y1 - y0) == (1, 1)
    assert cover.max() <= 1 and np.all(cover[mask == 1] == 1)
    print(f"regrid 4096^2: {len(boxes)} boxes over {int(mask.sum())} marked tiles, {dt * 1e3:.2f} ms")
    lat.close()
