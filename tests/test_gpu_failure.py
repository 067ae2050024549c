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
