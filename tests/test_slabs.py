"""The y-slab decomposition (paper_2603_13618_gb300/slabs.py) on CPU: each gloo rank steps
one slab with the FP64 oracle (tests/slab_oracle.py) and exchanges its halo rows with its
neighbours; the slabs' rows stitched together must equal the whole-lattice oracle bit for
bit (populations, sensor fields, flags, tile counts), the reduced counts exactly and the
reduced sums to rounding (they add the slabs in another order)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NX, NY, TILE, TAU, NSTEPS = 40, 48, 8, 0.65, 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _initial(ny=NY):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2603_13618_gb300 import inputs

    rho, ux, uy = inputs.smooth_jump(NX, ny, seed=5, kmax=4)
    return oracle.init_equilibrium(rho, ux, uy)


def _whole(f0):
    """The whole lattice's oracle run and the outputs of its last step."""
    import oracle

    f = f0
    for _ in range(NSTEPS - 1):
        f = oracle.step(f, TAU)
    sens, nonpos = oracle.sensor_fields(f, TAU, pull=True)
    kn, neq = sens[oracle.SENSOR_ID["kn"]], sens[oracle.SENSOR_ID["neq"]]
    flags, tiles, counts = oracle.flags(kn, 1e-3, neq, 1e-4, nonpos, TILE)
    sums = oracle.sums(oracle.stream(f))
    return oracle.step(f, TAU), sens, flags, tiles, counts, sums


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2603_13618_gb300 import slabs
    from tests.slab_oracle import OracleSlab

    dist.init_process_group("gloo")
    y0, rows = slabs.split_rows(NY, world, TILE)[rank]
    slab = OracleSlab(_initial()[:, y0:y0 + rows], TAU, tile=TILE)
    drv = slabs.SlabDriver(slab, dist, rank, world, device=False)
    drv.step(NSTEPS)
    sums, counts, step = drv.stats()
    out.put((rank, y0, slab.f, slab.sens, slab.flags, slab.tiles, counts, sums, step))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slabs_on_gloo_ranks_equal_the_whole_lattice(world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    fin, sens, flags, tiles, counts, sums = _whole(_initial())
    np.testing.assert_array_equal(np.concatenate([r[2] for r in res], axis=1), fin)
    np.testing.assert_array_equal(np.concatenate([r[3] for r in res], axis=1), sens)
    np.testing.assert_array_equal(np.concatenate([r[4] for r in res], axis=0), flags)
    np.testing.assert_array_equal(np.concatenate([r[5] for r in res], axis=1), tiles)
    for r in res:
        assert r[8] == NSTEPS
        np.testing.assert_array_equal(r[6], counts)      # reduced over the ranks
        np.testing.assert_allclose(r[7], sums, rtol=1e-13, atol=1e-13 * sums[0])
    assert counts[0] > 0 and counts[1] > 0               # both tags occur


def test_one_slab_is_the_periodic_lattice():
    """One rank (no process group): the slab's own rows wrap around."""
    sys.path.insert(0, ROOT)
    from paper_2603_13618_gb300 import slabs
    from tests.slab_oracle import OracleSlab

    slab = OracleSlab(_initial(), TAU, tile=TILE)
    drv = slabs.SlabDriver(slab, None, 0, 1, device=False)
    drv.step(NSTEPS)
    fin, sens, flags, tiles, counts, sums = _whole(_initial())
    np.testing.assert_array_equal(slab.f, fin)
    np.testing.assert_array_equal(slab.flags, flags)
    np.testing.assert_array_equal(drv.stats()[1], counts)


def test_local_ring_of_slabs_equals_the_whole_lattice():
    """Several slabs held by one process (slabs.step_local), a ragged last slab (45 rows:
    the last tile row is partial)."""
    sys.path.insert(0, ROOT)
    from paper_2603_13618_gb300 import slabs
    from tests.slab_oracle import OracleSlab

    f0 = _initial(45)
    parts = slabs.split_rows(45, 4, TILE)
    assert parts == [(0, 8), (8, 16), (24, 8), (32, 13)]
    ss = [OracleSlab(f0[:, y0:y0 + r], TAU, tile=TILE) for y0, r in parts]
    slabs.step_local(ss, NSTEPS)
    fin, sens, flags, tiles, counts, sums = _whole(f0)
    np.testing.assert_array_equal(np.concatenate([s.f for s in ss], axis=1), fin)
    np.testing.assert_array_equal(np.concatenate([s.flags for s in ss], axis=0), flags)
    np.testing.assert_array_equal(np.concatenate([s.tiles for s in ss], axis=1), tiles)
    assert sum(int(s.counts[0]) for s in ss) == counts[0]


def test_split_rows():
    sys.path.insert(0, ROOT)
    from paper_2603_13618_gb300 import slabs

    assert slabs.split_rows(64, 4, 16) == [(0, 16), (16, 16), (32, 16), (48, 16)]
    assert slabs.split_rows(70, 3, 16) == [(0, 16), (16, 32), (48, 22)]
    assert slabs.split_rows(33, 3, 16) == [(0, 16), (16, 16), (32, 1)]
    assert slabs.split_rows(4096, 8, 16)[-1] == (3584, 512)
    for ny, k, t in ((70, 3, 16), (4096, 7, 16), (100, 13, 8), (33, 1, 16)):
        parts = slabs.split_rows(ny, k, t)
        assert len(parts) == k and parts[0][0] == 0
        assert all(a[0] + a[1] == b[0] for a, b in zip(parts, parts[1:]))
        assert parts[-1][0] + parts[-1][1] == ny
        assert all(r % t == 0 for _, r in parts[:-1]) and all(r > 0 for _, r in parts)
    with pytest.raises(ValueError):
        slabs.split_rows(32, 3, 16)
    assert slabs.neighbours(0, 4) == (3, 1) and slabs.neighbours(3, 4) == (2, 0)
