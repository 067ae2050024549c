"""One y-slab of a decomposed lattice stepped by the FP64 oracle (test infrastructure):
the slab's rows of the state and its two halo rows.  A step is the oracle's periodic step
of the slab with one halo row on each side: pull streaming reads only adjacent rows, so
the slab's own rows come out exactly as in the whole lattice, and the halo rows' own
results are dropped.  The interface is the one the slab driver steps
(paper_2603_13618_gb300/slabs.py)."""
import numpy as np

import oracle

UP_Q, DOWN_Q = [2, 5, 6], [4, 7, 8]


class OracleSlab:
    on_device = False

    def __init__(self, f_rows, tau, thr_r=1e-3, thr_s=1e-4, tile=16):
        self.f = np.ascontiguousarray(f_rows, dtype=np.float64)
        self.tau, self.thr_r, self.thr_s, self.tile = tau, thr_r, thr_s, tile
        nx = self.f.shape[2]
        self.lo = np.zeros((9, nx))  # row -1: only q = 2, 5, 6 are read
        self.hi = np.zeros((9, nx))  # row ny: only q = 4, 7, 8 are read
        self.nstep = 0
        self.sens = self.flags = self.tiles = self.counts = self.sums = None

    def slab_edges(self, device=False, out=None):
        to_below = np.ascontiguousarray(self.f[DOWN_Q, 0, :])
        to_above = np.ascontiguousarray(self.f[UP_Q, -1, :])
        if out is None:
            return to_below, to_above
        for o, a in zip(out, (to_below, to_above)):
            if hasattr(o, "copy_"):  # a torch tensor (the exchange buffers of the driver)
                import torch

                o.copy_(torch.from_numpy(a))
            else:
                np.copyto(o, a)
        return out

    def set_halos(self, from_below, from_above):
        self.lo[UP_Q] = np.asarray(from_below, dtype=np.float64)
        self.hi[DOWN_Q] = np.asarray(from_above, dtype=np.float64)

    def step(self, n=1):
        assert n == 1
        ext = np.ascontiguousarray(np.concatenate([self.lo[:, None], self.f, self.hi[:, None]],
                                                  axis=1))
        with np.errstate(all="ignore"):
            sens, nonpos = oracle.sensor_fields(ext, self.tau, pull=True)
        ft = np.ascontiguousarray(oracle.stream(ext)[:, 1:-1])
        self.sens = sens[:, 1:-1]
        kn, neq = self.sens[oracle.SENSOR_ID["kn"]], self.sens[oracle.SENSOR_ID["neq"]]
        self.flags, self.tiles, self.counts = oracle.flags(
            np.ascontiguousarray(kn), self.thr_r, np.ascontiguousarray(neq), self.thr_s,
            np.ascontiguousarray(nonpos[1:-1]), self.tile)
        self.sums = oracle.sums(ft)
        self.f = oracle.collide(ft, self.tau)
        self.nstep += 1

    def read_stats(self):
        return self.sums, self.counts, self.nstep
