"""Domain decomposition of one periodic lattice into y-slabs, one per rank.

The paper's solver shares its lattice out between the processes of a distributed-memory
machine (section "Adaptive refinement and parallel processing").  Here the lattice of
NX x NY cells is cut into slabs of whole rows; rank r steps slab r (a lattice made by
kss_slab_create, see include/kss.h).  Per step, pull streaming needs across each face
only the three populations whose velocity crosses it: a slab's last row sends
q = 2, 5, 6 (c_y = +1) to the slab above, its first row q = 4, 7, 8 (c_y = -1) to the
slab below.  Those rows are exchanged with the two neighbouring ranks (periodic in y:
rank 0's lower neighbour is the last rank) before the step.  On an output step the
lattice's conservation sums and tag counts are the sums over the slabs (an all-reduce);
its flags, tile counts and sensor fields are the slabs' rows in order.

Everything here is host orchestration on torch.distributed (gloo on CPU tensors, NCCL on
device tensors): which rows a rank owns, the halo exchange and the reductions.  The
stepping is the slab object's (duck-typed: `slab_edges(device=..., out=...)`,
`set_halos(from_below, from_above)`, `step(1)`, `read_stats()`), so the same driver runs
a GPU slab (kss.Lattice(slab=True)) or any other implementation of one slab's step.
"""
from __future__ import annotations


def split_rows(ny: int, nslabs: int, tile: int = 16):
    """[(y0, rows)] of nslabs slabs covering rows 0 .. ny - 1: each inner boundary is the
    multiple of tile nearest to an even share of the rows (so that every slab but the last
    holds whole tiles, and the slabs' tile counts are the lattice's), at least one tile
    apart; the last slab takes the rest."""
    ntiles = -(-ny // tile)
    if nslabs < 1 or nslabs > ntiles:
        raise ValueError(f"{nslabs} slabs for {ntiles} tile rows")
    bounds = [0]
    for r in range(1, nslabs):
        b = tile * int(r * ny / (nslabs * tile) + 0.5)
        b = max(b, bounds[-1] + tile)                      # at least one tile per slab
        b = min(b, tile * (ntiles - (nslabs - r)))         # room for the slabs after it
        bounds.append(b)
    bounds.append(ny)
    return [(a, b - a) for a, b in zip(bounds, bounds[1:])]


def neighbours(rank: int, world: int):
    """(below, above): the ranks whose slabs border this one (periodic in y)."""
    return (rank - 1) % world, (rank + 1) % world


# message tags: rows moving up (a slab's last row into the slab above) and down
TAG_UP, TAG_DOWN = 1, 2


def exchange(dist, rank: int, world: int, to_below, to_above, from_below, from_above):
    """One step's halo exchange.  This slab's to_above becomes the upper neighbour's
    from_below, its to_below the lower neighbour's from_above.  One rank (or no process
    group) is the periodic lattice in one slab: its own rows wrap around."""
    if dist is None or world == 1:
        from_below.copy_(to_above)
        from_above.copy_(to_below)
        return
    below, above = neighbours(rank, world)
    ops = [dist.P2POp(dist.isend, to_above, above, tag=TAG_UP),
           dist.P2POp(dist.irecv, from_below, below, tag=TAG_UP),
           dist.P2POp(dist.isend, to_below, below, tag=TAG_DOWN),
           dist.P2POp(dist.irecv, from_above, above, tag=TAG_DOWN)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


class SlabDriver:
    """Steps this rank's slab of a decomposed lattice.

    device: exchange buffers on the GPU (NCCL) or on the host (gloo)."""

    def __init__(self, slab, dist=None, rank: int = 0, world: int = 1, device: bool = True):
        self.slab, self.dist, self.rank, self.world = slab, dist, rank, world
        self.device = device
        self.to_below, self.to_above = (_as_torch(a) for a in slab.slab_edges(device=device))
        self.from_below = self.to_above.new_empty(self.to_above.shape)
        self.from_above = self.to_below.new_empty(self.to_below.shape)

    def halos(self) -> None:
        """Fill the slab's halo rows from its neighbours' current edge rows."""
        self.slab.slab_edges(device=self.device, out=(self.to_below, self.to_above))
        exchange(self.dist, self.rank, self.world, self.to_below, self.to_above,
                 self.from_below, self.from_above)
        self.slab.set_halos(self.from_below, self.from_above)

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            self.halos()
            self.slab.step(1)

    def stats(self):
        """(sums[3], counts[3], step) of the whole lattice: the slabs' sums and counts
        added over the ranks."""
        import torch

        sums, counts, step = self.slab.read_stats()
        if self.dist is None or self.world == 1:
            return sums, counts, step
        dev = "cuda" if self.device else "cpu"
        s = torch.tensor(list(sums), dtype=torch.float64, device=dev)
        c = torch.tensor(list(counts), dtype=torch.int64, device=dev)
        self.dist.all_reduce(s)
        self.dist.all_reduce(c)
        return s.cpu().numpy(), c.cpu().numpy(), step


def step_local(slabs, n: int = 1) -> None:
    """n steps of all slabs of one lattice held by this process (in order from y = 0, on
    one device or on the host): the same exchange as between ranks, by copies."""
    k = len(slabs)
    for _ in range(n):
        edges = [s.slab_edges(device=_on_device(s)) for s in slabs]
        for r, s in enumerate(slabs):
            s.set_halos(edges[(r - 1) % k][1], edges[(r + 1) % k][0])
        for s in slabs:
            s.step(1)


def _on_device(slab) -> bool:
    return bool(getattr(slab, "on_device", True))


def _as_torch(a):
    """A torch view of a host numpy array (sharing its memory), or the tensor itself."""
    import torch

    return a if isinstance(a, torch.Tensor) else torch.from_numpy(a)
