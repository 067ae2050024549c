"""GPU: failure detection without a GPU fault.  The library's device-side waits are
bounded: a wait whose flag nothing sets gives up after its deadline, records the expiry
in the lattice's error word and returns.  kss_testing_expire_wait runs that same bounded
wait on a word nothing writes; the host must then see KSS_ERR_TIMEOUT (sticky on that
lattice) while the GPU context stays usable for everything else."""
import ctypes

import numpy as np
import pytest

import oracle
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


def test_an_expired_wait_is_reported_and_the_context_stays_usable():
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    nx, ny, tau = 64, 48, 0.7
    r, u, v = inputs.random_smooth(nx, ny, seed=5)
    lat = kss.Lattice(nx, ny, precision="fp32", tau=tau)
    lat.set_fields(r, u, v)
    lat.step(2)
    lat.sync()
    # argument checks first
    assert lib.kss_testing_expire_wait(lat._h, ctypes.c_int64(0)) == -1
    assert lib.kss_testing_expire_wait(lat._h, ctypes.c_int64(2_000_000_000)) == -1
    # about a millisecond of waiting on a flag that nothing sets
    assert lib.kss_testing_expire_wait(lat._h, ctypes.c_int64(2_000_000)) == 0
    with pytest.raises(kss.KssError) as e:
        lat.sync()
    assert e.value.code == -4  # KSS_ERR_TIMEOUT
    for call in (lambda: lat.step(1), lambda: lat.read_stats(), lambda: lat.sync()):
        with pytest.raises(kss.KssError) as e:
            call()
        assert e.value.code == -4  # sticky on this lattice
    lat.close()
    # the device is unharmed: a new lattice steps and matches the oracle
    other = kss.Lattice(nx, ny, precision="fp64", tau=tau)
    other.set_fields(r, u, v)
    other.step(3)
    want = oracle.step(oracle.init_equilibrium(r, u, v), tau, 3)
    np.testing.assert_allclose(other.get_populations(), want, rtol=1e-13)
    other.close()


def test_an_expired_mbarrier_wait_is_reported():
    """The TMA kernel's bounded mbarrier wait, on a barrier whose phase never completes."""
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    lat = kss.Lattice(64, 48, precision="fp32", tau=0.7)
    lat.set_fields(*inputs.random_smooth(64, 48, seed=6))
    lat.sync()
    assert lib.kss_testing_expire_mbarrier(lat._h, ctypes.c_int64(0)) == -1
    assert lib.kss_testing_expire_mbarrier(lat._h, ctypes.c_int64(2_000_000)) == 0
    with pytest.raises(kss.KssError) as e:
        lat.sync()
    assert e.value.code == -4  # KSS_ERR_TIMEOUT, sticky
    with pytest.raises(kss.KssError) as e:
        lat.step(1)
    assert e.value.code == -4
    lat.close()
    ok = kss.Lattice(64, 48, precision="fp32", tau=0.7, kernel="tma")
    ok.set_fields(*inputs.random_smooth(64, 48, seed=6))
    ok.step(2)
    ok.sync()
    ok.close()


def test_injected_allocation_failures_release_what_they_took():
    """Every device allocation of kss_create is made to fail in turn: the call reports
    KSS_ERR_OOM and leaves no allocation behind; then a batch creation the same way."""
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    base = lib.kss_testing_live_allocations()
    failed = 0
    for k in range(64):
        assert lib.kss_testing_fail_after(0, k) == 0
        try:
            lat = kss.Lattice(96, 40, precision="fp32", tau=0.7, tau2=0.9)
        except kss.KssError as e:
            assert e.code == -2  # KSS_ERR_OOM
            assert lib.kss_testing_live_allocations() == base
            failed += 1
            continue
        lib.kss_testing_fail_after(0, -1)
        # the creation that got through works and releases everything on close
        lat.set_fields(*inputs.random_smooth(96, 40, seed=2))
        lat.step(3)
        lat.close()
        assert lib.kss_testing_live_allocations() == base
        break
    assert failed >= 10  # every allocation of a lattice was made to fail once
    for k in range(8):
        lib.kss_testing_fail_after(0, 20 * k)
        try:
            b = kss.Batch([dict(nx=64, ny=64, tau=0.7), dict(nx=128, ny=96, tau=0.9)],
                          precision="fp32")
        except kss.KssError as e:
            assert e.code == -2
            assert lib.kss_testing_live_allocations() == base
            continue
        lib.kss_testing_fail_after(0, -1)
        b.close()
        assert lib.kss_testing_live_allocations() == base
    lib.kss_testing_fail_after(0, -1)


def test_an_injected_launch_failure_is_sticky_and_local():
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    nx, ny, tau = 64, 48, 0.7
    r, u, v = inputs.random_smooth(nx, ny, seed=8)
    a = kss.Lattice(nx, ny, precision="fp64", tau=tau)
    b = kss.Lattice(nx, ny, precision="fp64", tau=tau)
    for lat in (a, b):
        lat.set_fields(r, u, v)
    assert lib.kss_testing_fail_after(1, 1) == 0  # the second kss_step from now
    a.step(1)
    with pytest.raises(kss.KssError) as e:
        a.step(1)
    assert e.value.code == -3  # KSS_ERR_CUDA
    for call in (lambda: a.step(1), lambda: a.read_stats(), lambda: a.sync()):
        with pytest.raises(kss.KssError) as e:
            call()
        assert e.value.code == -3  # sticky on that lattice
    b.step(3)  # the other lattice is unaffected
    np.testing.assert_allclose(b.get_populations(),
                               oracle.step(oracle.init_equilibrium(r, u, v), tau, 3), rtol=1e-13)
    base = lib.kss_testing_live_allocations()
    a.close()
    assert lib.kss_testing_live_allocations() < base  # the failed lattice frees its memory
    b.close()
