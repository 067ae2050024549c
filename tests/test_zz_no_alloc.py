"""The allocation-free fused step (kss_step_f32_noalloc) against the library's own
lattice path (kss_step through a kss_lattice), on two calls in a row, and directly
against the FP64 oracle (every cell, two ragged sizes).

The entry point exists for callers that cannot allocate device memory (they own all
buffers, or must not allocate while running); it keeps the kernel's scratch in a
fixed device array instead.  Both paths run the same FP32 fused kernel, so every
output must agree within the FP32 parity tolerances (in practice bit for bit).
This file is collected last so that a failure here does not stop the other tests.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2603_13618_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

KN, NEQ, KL = 5, 6, 9


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_step_matches_lattice_step(torch_cuda):
    torch = torch_cuda
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    nx, ny, tau, tile = 300, 201, 0.65, 16
    thr_r, thr_s = 1e-3, 1e-4
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=77, kmax=6)
    lat = kss.Lattice(nx, ny, precision="fp32", tau=tau, refine_sensor="kn",
                      refine_threshold=thr_r, switch_sensor="neq", switch_threshold=thr_s,
                      record=("kl",), tile=tile)
    lat.set_fields(rho, ux, uy)
    lat.step(3)

    pitch = -(-nx // 32) * 32
    dev = "cuda"
    fa = torch.zeros((9, ny, pitch), dtype=torch.float32, device=dev)
    fb = torch.zeros_like(fa)
    fa[:, :, :nx] = torch.from_numpy(lat.get_populations()).to(dev, torch.float32)
    sensor = torch.zeros((ny, pitch), dtype=torch.float32, device=dev)
    flags = torch.zeros((ny, pitch), dtype=torch.uint8, device=dev)
    tiles = torch.zeros((2, -(-ny // tile), -(-nx // tile)), dtype=torch.int32, device=dev)
    sums = torch.zeros(3, dtype=torch.float64, device=dev)
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    src, dst = fa, fb
    for call in range(2):
        rc = lib.kss_step_f32_noalloc(_ptr(src), _ptr(dst), nx, ny, pitch, tau, KN, thr_r, NEQ,
                                      thr_s, tile, KL, _ptr(sensor), _ptr(flags), _ptr(tiles),
                                      _ptr(sums), _ptr(counts), ctypes.c_void_p(stream))
        assert rc == 0, (call, rc)
        lat.step(1)
        torch.cuda.synchronize()
        want_f = lat.get_populations()
        got_f = dst[:, :, :nx].double().cpu().numpy()
        np.testing.assert_allclose(got_f, want_f, rtol=64 * 2.0**-24 * math.sqrt(5), atol=0)
        np.testing.assert_allclose(sensor[:, :nx].double().cpu().numpy(), lat.read_sensor("kl"),
                                   rtol=1e-3, atol=1e-9)
        fl, tl, cnt = lat.read_flags()
        np.testing.assert_array_equal(flags[:, :nx].cpu().numpy(), fl)
        np.testing.assert_array_equal(tiles.cpu().numpy(), tl)
        np.testing.assert_array_equal(counts.cpu().numpy(), cnt)
        s_want, _, _ = lat.read_stats()
        np.testing.assert_allclose(sums.cpu().numpy(), s_want, rtol=1e-12, atol=1e-9)
        src, dst = dst, src
    lat.close()


@pytest.mark.parametrize("nx,ny,tau", [(300, 201, 0.6), (1031, 517, 1.0)])
def test_noalloc_step_matches_the_oracle(torch_cuda, nx, ny, tau):
    """One call from the FP32-rounded equilibrium of the smooth-jump fields: populations,
    the recorded KL field, flags (outside the threshold band), tile counts, counts and
    sums against the oracle's step of the same FP32 state, at every cell."""
    torch = torch_cuda
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    tile, thr_r, thr_s = 16, 1e-3, 1e-4
    rho, ux, uy = inputs.smooth_jump(nx, ny, seed=nx + ny, kmax=6)
    f0 = oracle.init_equilibrium(rho, ux, uy).astype(np.float32).astype(np.float64)
    pitch = -(-nx // 32) * 32
    dev = "cuda"
    fa = torch.zeros((9, ny, pitch), dtype=torch.float32, device=dev)
    fa[:, :, :nx] = torch.from_numpy(f0).to(dev, torch.float32)
    fb = torch.zeros_like(fa)
    sensor = torch.zeros((ny, pitch), dtype=torch.float32, device=dev)
    flags = torch.zeros((ny, pitch), dtype=torch.uint8, device=dev)
    tiles = torch.zeros((2, -(-ny // tile), -(-nx // tile)), dtype=torch.int32, device=dev)
    sums = torch.zeros(3, dtype=torch.float64, device=dev)
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    rc = lib.kss_step_f32_noalloc(_ptr(fa), _ptr(fb), nx, ny, pitch, tau, KN, thr_r, NEQ,
                                  thr_s, tile, KL, _ptr(sensor), _ptr(flags), _ptr(tiles),
                                  _ptr(sums), _ptr(counts),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    got_f = fb[:, :, :nx].double().cpu().numpy()

    sens, nonpos = oracle.sensor_fields(f0, tau, pull=True)
    ft = oracle.stream(f0)
    r, u, v = oracle.moments(ft)
    fin = oracle.collide(ft, tau)
    u32 = parity.UNIT_ROUNDOFF["fp32"]
    assert np.max(np.abs(got_f - fin) / fin) <= 64 * u32 * math.sqrt(2)
    kn = sens[oracle.SENSOR_ID["kn"]]
    parity.assert_sensor_close("kl", sensor[:, :nx].double().cpu().numpy(),
                               sens[oracle.SENSOR_ID["kl"]], "fp32", 1, r, u, v, kn, tau,
                               neq=parity.neq_field(ft), where=f"noalloc {nx}x{ny}")
    es = sens[oracle.SENSOR_ID["neq"]]
    rf, rt, rcnt = oracle.flags(kn, thr_r, es, thr_s, nonpos, tile)
    band = parity.band_mask(kn, thr_r, es, thr_s)
    parity.assert_flags_match(flags[:, :nx].cpu().numpy(), tiles.cpu().numpy(),
                              counts.cpu().numpy(), rf, rt, rcnt, band, tile)
    assert 0 < int(counts[0]) < nx * ny
    want = oracle.sums(ft)
    assert np.all(np.abs(sums.cpu().numpy() - want) <= 16 * u32 * want[0])


def test_noalloc_rejects_problems_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    # 16384 x 16384: 128 x 512 = 65536 CTAs > KSS_NOALLOC_MAX_BLOCKS (16384); rejected
    # before any launch, so tiny stand-in buffers are never touched
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    b8 = torch.zeros(64, dtype=torch.uint8, device="cuda")
    i32 = torch.zeros(64, dtype=torch.int32, device="cuda")
    d = torch.zeros(3, dtype=torch.float64, device="cuda")
    c = torch.zeros(3, dtype=torch.int64, device="cuda")
    # (the output address is a stand-in past the input's 9 x 16384^2 floats: the call
    # rejects the size before it touches either buffer)
    far = buf.data_ptr() + 9 * 16384 * 16384 * 4
    rc = lib.kss_step_f32_noalloc(_ptr(buf), far, 16384, 16384, 16384, 0.8, KN, 1e-3,
                                  NEQ, 1e-4, 8, KL, _ptr(buf), _ptr(b8), _ptr(i32), _ptr(d),
                                  _ptr(c), None)
    assert rc == -7
    # an in-place step (f_out = f_in), or overlapping population ranges, is an argument
    # error: the pull step would read populations that other CTAs already overwrote
    big = torch.zeros(2 * 9 * 64 * 8, dtype=torch.float32, device="cuda")
    for dst in (big.data_ptr(), big.data_ptr() + 4 * 9 * 64 * 8 - 16):
        rc = lib.kss_step_f32_noalloc(_ptr(big), dst, 64, 8, 64, 0.8, KN, 1e-3, NEQ, 1e-4, 8,
                                      KL, None, _ptr(b8), _ptr(i32), _ptr(d), _ptr(c), None)
        assert rc == -1
    # a non-{Kn, KL, neq} sensor is an argument error
    rc = lib.kss_step_f32_noalloc(_ptr(big), big.data_ptr() + 4 * 9 * 64 * 8, 64, 8, 64, 0.8, 0,
                                  1e-3, NEQ, 1e-4, 8,
                                  KL, _ptr(buf), _ptr(b8), _ptr(i32), _ptr(d), _ptr(c), None)
    assert rc == -1
