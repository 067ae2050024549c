"""Pins of the regrid oracle (oracle/regrid.py): the buffered tile mask against a
dilation built from numpy rolls, and the clustering against hand-worked layouts and the
invariants every clustering must keep (coverage, disjointness, efficiency)."""
import numpy as np
import pytest

from oracle import regrid


def test_tile_mask_against_rolled_dilation():
    rng = np.random.default_rng(2)
    for (ny, nx, tile, buf) in [(40, 56, 8, 2), (37, 21, 16, 2), (64, 64, 8, 0), (30, 50, 8, 5)]:
        flags = (rng.random((ny, nx)) < 0.01).astype(np.uint8) * rng.choice([1, 3, 129], (ny, nx)).astype(np.uint8)
        flags[rng.random((ny, nx)) < 0.05] |= 2  # switch bits alone never mark
        ref = (flags & 1).astype(bool)
        dil = ref.copy()
        for dy in range(-buf, buf + 1):
            for dx in range(-buf, buf + 1):
                dil |= np.roll(np.roll(ref, dy, axis=0), dx, axis=1)
        ntx, nty = -(-nx // tile), -(-ny // tile)
        pad = np.zeros((nty * tile, ntx * tile), dtype=bool)
        pad[:ny, :nx] = dil
        want = pad.reshape(nty, tile, ntx, tile).any(axis=(1, 3)).astype(np.uint8)
        np.testing.assert_array_equal(regrid.tile_mask(flags, tile, buf), want)


def _check_invariants(mask, boxes, eff):
    cover = np.zeros(mask.shape, dtype=np.int64)
    for (x0, y0, x1, y1) in boxes:
        assert 0 <= x0 < x1 <= mask.shape[1] and 0 <= y0 < y1 <= mask.shape[0]
        cover[y0:y1, x0:x1] += 1
        sub = mask[y0:y1, x0:x1]
        w, h = x1 - x0, y1 - y0
        assert sub.sum() >= eff * w * h or (w == 1 and h == 1)
        # boxes are tight: every edge row / column holds a mark
        assert sub[0].any() and sub[-1].any() and sub[:, 0].any() and sub[:, -1].any()
    assert cover.max(initial=0) <= 1                      # disjoint
    assert np.all(cover[mask.astype(bool)] == 1)          # every marked tile covered


def test_empty_full_and_separated_blobs():
    m = np.zeros((10, 12), dtype=np.uint8)
    assert regrid.cluster(m, 0.7) == []
    m[2:6, 3:9] = 1
    assert regrid.cluster(m, 0.7) == [(3, 2, 9, 6)]
    # a second blob beyond an empty column: one hole split, two exact boxes
    m[1:3, 10:12] = 1
    assert sorted(regrid.cluster(m, 0.9)) == [(3, 2, 9, 6), (10, 1, 12, 3)]


def test_hole_nearest_the_centre_wins():
    m = np.zeros((4, 11), dtype=np.uint8)
    m[:, [0, 1, 3, 4, 5, 7, 8, 9, 10]] = 1   # holes at columns 2 and 6; centre column 5
    boxes = regrid.cluster(m, 1.0)
    # first cut at the hole at 6 (distance |12 - 10| = 2 < |4 - 10| = 6), then at 2
    assert boxes == [(7, 0, 11, 4), (0, 0, 2, 4), (3, 0, 6, 4)]


def test_l_shape_splits_at_the_inflection():
    m = np.zeros((8, 8), dtype=np.uint8)
    m[0:8, 0:2] = 1    # vertical bar
    m[0:2, 2:8] = 1    # horizontal bar
    boxes = regrid.cluster(m, 0.95)
    # column signature 8 8 2 2 2 2 2 2: Laplacian 0 -6 6 0 ... changes sign between
    # columns 1 and 2 (strength 12), the strongest cut: the bar and the arm
    assert boxes == [(0, 0, 2, 8), (2, 0, 8, 2)]


def test_bisection_when_no_hole_or_inflection():
    m = np.zeros((2, 8), dtype=np.uint8)
    m[0, :] = 1
    m[1, 0] = m[1, 7] = 1     # a frame that needs cutting, no interior hole
    boxes = regrid.cluster(m, 1.0)
    _check_invariants(m, boxes, 1.0)
    assert all(m[y0:y1, x0:x1].all() for (x0, y0, x1, y1) in boxes)


@pytest.mark.parametrize("eff", [0.5, 0.7, 0.98, 1.0])
def test_random_masks_keep_the_invariants(eff):
    rng = np.random.default_rng(int(eff * 100))
    for _ in range(20):
        ny, nx = rng.integers(1, 40, 2)
        m = np.zeros((ny, nx), dtype=np.uint8)
        for _ in range(rng.integers(0, 6)):          # a few rectangles and noise
            y0, x0 = rng.integers(0, ny), rng.integers(0, nx)
            m[y0:y0 + rng.integers(1, 12), x0:x0 + rng.integers(1, 12)] = 1
        m[rng.random((ny, nx)) < 0.03] = 1
        boxes = regrid.cluster(m, eff)
        _check_invariants(m, boxes, eff)
        if eff == 1.0:
            assert sum((x1 - x0) * (y1 - y0) for (x0, y0, x1, y1) in boxes) == int(m.sum())
