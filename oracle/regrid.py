"""Plain CPU oracle of regrid steps (1)-(2) acting on the refine flags (section "Adaptive
refinement and parallel processing": tagged cells, a buffer around them, and a
clustering algorithm that groups them into rectangular patches; the applications use two
buffer cells and a grid efficiency threshold, section "Application to adaptive mesh
refinement").

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only tests/ may import this module.  It shares
no code with the CUDA library.

Definitions (the paper cites Berger & Rigoutsos for the clustering but prints no
algorithm; this is the method of that reference as read here, at the granularity of the
tagging tiles):

* Tile mask.  A tile (tile x tile cells) is marked when some cell within `buffer` cells
  (Chebyshev distance, periodic) of the tile has the refine flag (bit 0).
* Clustering of the marked tiles into boxes [x0, x1) x [y0, y1) (tile units), breadth
  first from the whole tile grid.  For a box:
  1. signatures sx[i] = marked tiles in column i, sy[j] = in row j;
  2. no marked tile: drop the box; else shrink it to the bounding box of its marks;
  3. accept it if marks / area >= efficiency, or if it is one tile wide and high;
  4. else split at a hole: a zero signature strictly inside the box, the one nearest the
     box centre (ties: x before y, then the lower index); the hole's row / column is left
     out of both halves;
  5. else at the strongest inflection: d[i] = s[i-1] - 2 s[i] + s[i+1] for interior i;
     between i and i+1 where d[i] d[i+1] < 0, strength |d[i+1] - d[i]|, the strongest
     one (ties: nearest the centre, then x before y, then the lower index);
  6. else bisect the longer side (x if equal) at its middle (x0 + w // 2).
  Children go to the next level in order (lower half first); a level's accepted boxes
  are reported in the order of the level's list.
"""
from __future__ import annotations

import numpy as np


def tile_mask(flags: np.ndarray, tile: int, buffer: int) -> np.ndarray:
    """uint8 [nty, ntx]: 1 where a refine-flagged cell lies within `buffer` cells of the
    tile (periodic), by brute force over each tile's neighbourhood."""
    ny, nx = flags.shape
    ntx, nty = -(-nx // tile), -(-ny // tile)
    ref = (flags & 1) != 0
    out = np.zeros((nty, ntx), dtype=np.uint8)
    for ty in range(nty):
        for tx in range(ntx):
            ys = np.arange(ty * tile - buffer, min((ty + 1) * tile, ny) + buffer) % ny
            xs = np.arange(tx * tile - buffer, min((tx + 1) * tile, nx) + buffer) % nx
            out[ty, tx] = 1 if ref[np.ix_(ys, xs)].any() else 0
    return out


def _tile_key(i, lo, hi):
    """Distance of tile i from the centre of [lo, hi), in half tiles."""
    return abs(2 * i - (lo + hi - 1))


def _cut_key(i, lo, hi):
    """Distance of the cut between tiles i - 1 and i from the centre of [lo, hi), in half
    tiles."""
    return abs(2 * i - (lo + hi))


def cluster(mask: np.ndarray, efficiency: float):
    """Boxes (x0, y0, x1, y1) covering the marked tiles of mask [nty, ntx]."""
    nty, ntx = mask.shape
    m = mask.astype(np.int64)
    level = [(0, 0, ntx, nty)]
    out = []
    while level:
        nxt = []
        for (x0, y0, x1, y1) in level:
            sub = m[y0:y1, x0:x1]
            sx = sub.sum(axis=0)
            sy = sub.sum(axis=1)
            total = int(sx.sum())
            if total == 0:
                continue
            nzx = np.nonzero(sx)[0]
            nzy = np.nonzero(sy)[0]
            x0, x1 = x0 + int(nzx[0]), x0 + int(nzx[-1]) + 1
            y0, y1 = y0 + int(nzy[0]), y0 + int(nzy[-1]) + 1
            sx = m[y0:y1, x0:x1].sum(axis=0)
            sy = m[y0:y1, x0:x1].sum(axis=1)
            w, h = x1 - x0, y1 - y0
            if total >= efficiency * (w * h) or (w == 1 and h == 1):
                out.append((x0, y0, x1, y1))
                continue
            # holes strictly inside
            best = None
            for axis, s, lo, hi in ((0, sx, x0, x1), (1, sy, y0, y1)):
                for k in range(1, len(s) - 1):
                    if s[k] == 0:
                        i = lo + k
                        key = (_tile_key(i, lo, hi), axis, i)
                        if best is None or key < best[0]:
                            best = (key, axis, i)
            if best is not None:
                _, axis, i = best
                if axis == 0:
                    nxt += [(x0, y0, i, y1), (i + 1, y0, x1, y1)]
                else:
                    nxt += [(x0, y0, x1, i), (x0, i + 1, x1, y1)]
                continue
            # strongest inflection
            best = None
            for axis, s, lo, hi in ((0, sx, x0, x1), (1, sy, y0, y1)):
                n = len(s)
                d = [0] * n
                for k in range(1, n - 1):
                    d[k] = int(s[k - 1]) - 2 * int(s[k]) + int(s[k + 1])
                for k in range(1, n - 2):
                    if d[k] * d[k + 1] < 0:
                        i = lo + k + 1  # split between k and k + 1
                        key = (-abs(d[k + 1] - d[k]), _cut_key(i, lo, hi), axis, i)
                        if best is None or key < best[0]:
                            best = (key, axis, i)
            if best is not None:
                _, axis, i = best
                if axis == 0:
                    nxt += [(x0, y0, i, y1), (i, y0, x1, y1)]
                else:
                    nxt += [(x0, y0, x1, i), (x0, i, x1, y1)]
                continue
            if w >= h:
                i = x0 + w // 2
                nxt += [(x0, y0, i, y1), (i, y0, x1, y1)]
            else:
                i = y0 + h // 2
                nxt += [(x0, y0, x1, i), (x0, i, x1, y1)]
        level = nxt
    return out
