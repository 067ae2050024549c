"""Slab lattices (kss_slab_create) on the GPU: a lattice cut into y-slabs, each stepped
with halo rows exchanged between steps (paper_2603_13618_gb300/slabs.step_local: the
ranks' exchange done by copies in one process), equals the same lattice stepped whole,
bit for bit: populations, the recorded sensor fields, flags, tile counts and counts; the
sums of the slabs add to the lattice's to rounding (another order of addition)."""
import numpy as np
import pytest

from paper_2603_13618_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kss():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_13618_gb300 import kss

    kss.load()
    return kss


def _run(kss, prec, nslabs, nx, ny, nsteps, tile=16, tau=0.62):
    from paper_2603_13618_gb300 import slabs

    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=nx + ny, kmax=6)
    kw = dict(precision=prec, tau=tau, record=("kl", "kn"), output_every=1, tile=tile)
    whole = kss.Lattice(nx, ny, **kw)
    whole.set_fields(rho, ux, uy)
    for _ in range(nsteps):
        whole.step(1)
    parts = slabs.split_rows(ny, nslabs, tile)
    ss = []
    for y0, rows in parts:
        s = kss.Lattice(nx, rows, slab=True, **kw)
        s.set_fields(*(np.ascontiguousarray(a[y0:y0 + rows]) for a in (rho, ux, uy)))
        ss.append(s)
    slabs.step_local(ss, nsteps)
    return whole, ss


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp16dev"])
@pytest.mark.parametrize("nslabs", [1, 3])
def test_slabs_equal_the_whole_lattice(kss, prec, nslabs):
    nx, ny, nsteps = 300, 211, 7
    whole, ss = _run(kss, prec, nslabs, nx, ny, nsteps)
    cat = lambda xs, ax: np.concatenate(xs, axis=ax)  # noqa: E731
    np.testing.assert_array_equal(cat([s.get_populations() for s in ss], 1),
                                  whole.get_populations())
    for name in ("kl", "kn"):
        np.testing.assert_array_equal(cat([s.read_sensor(name) for s in ss], 0),
                                      whole.read_sensor(name))
    outs = [s.read_flags() for s in ss]
    fw, tw, cw = whole.read_flags()
    np.testing.assert_array_equal(cat([o[0] for o in outs], 0), fw)
    np.testing.assert_array_equal(cat([o[1] for o in outs], 1), tw)
    np.testing.assert_array_equal(sum(o[2] for o in outs), cw)
    # the sums add per-thread partials in the arithmetic type (FP32: a few rows of cells
    # added in single precision before the double-float reduction), so two block
    # decompositions agree to a few u per partial: at most 16 u sum(rho) in all
    sw = whole.read_stats()[0]
    u = 2.0**-53 if prec == "fp64" else 2.0**-24
    np.testing.assert_allclose(sum(s.read_stats()[0] for s in ss), sw, rtol=0,
                               atol=16 * u * sw[0])
    assert all(s.read_stats()[2] == nsteps for s in ss)
    for s in ss + [whole]:
        s.close()


def test_slab_steps_one_step_per_call_and_edges_need_a_slab(kss):
    lat = kss.Lattice(64, 32, precision="fp32", slab=True)
    lat.set_fields(*inputs.smooth_jump(64, 32, seed=1, kmax=3))
    b, a = lat.slab_edges(device=True)
    assert b.shape == (3, 64) and a.shape == (3, 64)
    with pytest.raises(kss.KssError):
        lat.step(2)
    plain = kss.Lattice(64, 32, precision="fp32")
    with pytest.raises(kss.KssError):
        plain.slab_edges(device=True)
    # host buffers round-trip exactly: the edge rows are the stored populations' rows
    hb, ha = lat.slab_edges(device=False)
    f = lat.get_populations()
    np.testing.assert_array_equal(hb, f[[4, 7, 8], 0, :].astype(np.float32))
    np.testing.assert_array_equal(ha, f[[2, 5, 6], -1, :].astype(np.float32))
    lat.close()
    plain.close()
