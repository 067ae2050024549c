"""GPU: the hand-written discrete adjoint (kss_adjoint_*, and its torch.autograd front
end) against the FP64 oracle's adjoint and against central finite differences of the
FP64 oracle's forward objective.

Objective: J = sum_x W(x) eps_KL(x) of step N; gradients in the initial density rho0
(initial populations f^eq(rho0, u0), u0 fixed) and in tau.
"""
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


def _kss():
    from paper_2603_13618_gb300 import kss

    return kss


def _rel_inf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("nx,ny,N,E,tau,weighted", [
    (37, 21, 1, 1, 0.7, False), (37, 21, 7, 3, 0.7, True), (130, 67, 13, 20, 1.0, False),
    (64, 64, 10, 4, 0.55, True), (1, 5, 4, 2, 0.8, False), (5, 1, 6, 6, 1.3, False),
    (200, 9, 9, 1, 0.6, True)])
def test_fp64_adjoint_equals_the_oracle_adjoint(nx, ny, N, E, tau, weighted):
    kss = _kss()
    r, u, v = inputs.random_smooth(nx, ny, seed=nx + 7 * ny, kmax=3, drho_amp=0.02, mach=0.12)
    w = np.random.default_rng(nx).uniform(0.3, 2.0, (ny, nx)) if weighted else None
    Jr, gr, gtr = oracle.adjoint_kl(r, u, v, tau, N, weight=w)
    with kss.Adjoint(nx, ny, N, precision="fp64", checkpoint_every=E) as adj:
        J = adj.forward(r, u, v, tau, weight=w)
        g, gt = adj.backward()
    assert J == pytest.approx(Jr, rel=1e-12)
    assert _rel_inf(g, gr) <= 1e-10
    if N == 1:
        assert gt == 0.0
    else:
        assert gt == pytest.approx(gtr, rel=1e-10)


def test_fp32_adjoint_at_512_by_200_steps():
    """512 x 512, 200 steps, checkpoints every 20 (the adjoint workload): the FP32
    gradient against the FP64 oracle adjoint, and its directional derivative and tau
    derivative against central differences (h = 1e-3, with the h/2 Richardson
    combination) of the FP64 oracle's forward objective, all to 1e-4 relative."""
    kss = _kss()
    n, N, tau = 512, 200, 0.6
    r, u, v = inputs.random_smooth(n, n, seed=1361, kmax=8, drho_amp=1e-2, mach=0.1)
    with kss.Adjoint(n, n, N, precision="fp32", checkpoint_every=20) as adj:
        J = adj.forward(r, u, v, tau)
        g, gt = adj.backward()
    Jr, gr, gtr = oracle.adjoint_kl(r, u, v, tau, N, store_every=20)
    assert J == pytest.approx(Jr, rel=1e-4)
    assert _rel_inf(g, gr) <= 1e-3
    assert gt == pytest.approx(gtr, rel=1e-4)
    d = np.random.default_rng(1361).standard_normal((n, n))
    f = lambda t: oracle.objective_kl(r + t * d, u, v, tau, N)
    h = 1e-3
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    fd = (4 * d2 - d1) / 3
    assert float(np.sum(g * d)) == pytest.approx(fd, rel=1e-4)
    ft = lambda t: oracle.objective_kl(r, u, v, t, N)
    fdt = (4 * (ft(tau + h / 2) - ft(tau - h / 2)) / h - (ft(tau + h) - ft(tau - h)) / (2 * h)) / 3
    assert gt == pytest.approx(fdt, rel=1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_objective_equals_the_summed_kl_field_of_a_lattice_run(prec):
    kss = _kss()
    nx, ny, N, tau = 96, 80, 25, 0.7
    r, u, v = inputs.random_smooth(nx, ny, seed=5, kmax=4)
    with kss.Adjoint(nx, ny, N, precision=prec, checkpoint_every=6) as adj:
        J = adj.forward(r, u, v, tau)
    lat = kss.Lattice(nx, ny, precision=prec, tau=tau, record=("kl",))
    lat.set_fields(r, u, v)
    lat.step(N)
    kl = lat.read_sensor("kl")
    lat.close()
    assert J == pytest.approx(float(np.sum(kl)), rel=1e-11 if prec == "fp64" else 1e-5)


def test_autograd_function():
    import torch

    from paper_2603_13618_gb300 import autograd

    kss = _kss()
    nx, ny, N = 48, 40, 12
    r, u, v = inputs.random_smooth(nx, ny, seed=11, kmax=3)
    rho = torch.tensor(r, device="cuda", requires_grad=True)
    tau = torch.tensor(0.8, dtype=torch.float64, device="cuda", requires_grad=True)
    ux, uy = torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda")
    J = autograd.kl_objective(rho, tau, ux, uy, N, precision="fp64", checkpoint_every=5)
    (3.0 * J).backward()
    Jr, gr, gtr = oracle.adjoint_kl(r, u, v, 0.8, N)
    assert float(J.detach()) == pytest.approx(Jr, rel=1e-12)
    assert _rel_inf(rho.grad.cpu().numpy(), 3.0 * gr) <= 1e-10
    assert float(tau.grad) == pytest.approx(3.0 * gtr, rel=1e-10)
    # the plain call gives the same numbers
    with kss.Adjoint(nx, ny, N, precision="fp64", checkpoint_every=5) as adj:
        assert adj.forward(r, u, v, 0.8) == float(J.detach())
        g, gt = adj.backward()
    np.testing.assert_array_equal(3.0 * g, rho.grad.cpu().numpy())


def test_backward_needs_a_forward_pass():
    kss = _kss()
    r, u, v = inputs.random_smooth(16, 16, seed=2, kmax=2)
    with kss.Adjoint(16, 16, 3, precision="fp32", checkpoint_every=2) as adj:
        with pytest.raises(kss.KssError) as e:
            adj.backward()
        assert e.value.code == -5
        adj.forward(r, u, v, 0.9)
        adj.backward()
        with pytest.raises(kss.KssError) as e:
            adj.backward()
        assert e.value.code == -5
        with pytest.raises(kss.KssError):
            adj.forward(r, u, v, 0.5)


def test_repeated_calls_replay_the_recorded_sweeps():
    """The forward and backward sweeps are recorded as graphs for the (tau, weight) of the
    call and replayed: repeated calls, and calls after tau or the weight changed, give
    exactly what a fresh object gives."""
    kss = _kss()
    nx, ny, N = 40, 36, 9
    r, u, v = inputs.random_smooth(nx, ny, seed=4, kmax=3)
    w = np.random.default_rng(4).uniform(0.5, 1.5, (ny, nx))

    def fresh(tau, weight):
        with kss.Adjoint(nx, ny, N, precision="fp32", checkpoint_every=4) as a:
            J = a.forward(r, u, v, tau, weight=weight)
            return (J,) + a.backward()

    with kss.Adjoint(nx, ny, N, precision="fp32", checkpoint_every=4) as adj:
        for tau, weight in ((0.8, None), (0.8, None), (0.9, None), (0.9, w), (0.8, None)):
            J = adj.forward(r, u, v, tau, weight=weight)
            g, gt = adj.backward()
            J0, g0, gt0 = fresh(tau, weight)
            assert J == J0 and gt == gt0
            np.testing.assert_array_equal(g, g0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n,N,E", [(96, 23, 5), (512, 200, 20), (70, 9, 9), (64, 6, 1)])
def test_multistep_reverse_sweep_equals_one_launch_per_step(prec, n, N, E):
    """The reverse sweep of each segment in one cooperative launch (blocks waiting on their
    neighbours' previous reverse step), which also recomputes the previous segment's states,
    gives the gradients of one launch per reverse step after plain recomputing steps, bit
    for bit: the same per-block arithmetic, the same partials and order of addition.  The
    cases cover a partial last segment (fewer reverse iterations than recomputed steps),
    full segments, one segment (nothing to recompute) and a checkpoint every step."""
    from paper_2603_13618_gb300 import kss

    r, u, v = inputs.random_smooth(n, n - 3, seed=n + N, kmax=6, drho_amp=1e-2, mach=0.1)
    out = []
    for multi in (True, False):
        adj = kss.Adjoint(n, n - 3, N, precision=prec, checkpoint_every=E)
        adj.set_multistep(multi)
        J = adj.forward(r, u, v, 0.6)
        g, gt = adj.backward()
        out.append((J, g, gt))
        adj.close()
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
