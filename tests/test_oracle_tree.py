"""Pins of the numpy octree oracle to the paper's combinatorics (Sec. 2.3
interaction-list rule; Sec. 3.2.3, Eqs. 14-19 surface-to-volume model)."""
import numpy as np
import pytest

from conftest import golden
from oracle import tree


@pytest.mark.parametrize("k", [2, 3, 4, 8, 16])
def test_neighbour_census(k):
    """Of the k^3 boxes, 8 corners have 7 neighbours, 12(k-2) edge boxes
    have 11, 6(k-2)^2 face boxes have 17 and (k-2)^3 interior boxes 26."""
    nb = tree.neighbour_counts(k)
    counts = {v: int(np.sum(nb == v)) for v in np.unique(nb)}
    want = {7: 8, 11: 12 * (k - 2), 17: 6 * (k - 2) ** 2, 26: (k - 2) ** 3}
    want = {a: b for a, b in want.items() if b}
    assert counts == want


def test_eq19_direct_work_sums():
    rows = golden("eq19_direct_work.txt")
    sums = {int(r[0]): float(r[1]) for r in rows if r[0] != "ratio"}
    for k, s in sums.items():
        assert tree.direct_work_sum(k) == s
    for r in rows:
        if r[0] == "ratio":
            kf, kc, R = int(r[1]), int(r[2]), float(r[3])
            assert round(tree.direct_work_sum(kf) / tree.direct_work_sum(kc), 2) == R


def test_interaction_list_sizes():
    """An interior box has 216 - 27 = 189 interaction-list boxes; over the
    eight positions of a box inside its parent the offsets cover all
    7^3 - 3^3 = 316 vectors with max-norm 2 or 3."""
    lo, hi = np.array([0, 0, 0]), np.array([63, 63, 63])
    offsets = set()
    for oct_ in range(8):
        t = np.array([20 + (oct_ & 1), 20 + ((oct_ >> 1) & 1), 20 + ((oct_ >> 2) & 1)])
        il = tree.interaction_list(t, lo, hi)
        assert len(il) == 189
        d = il - t
        assert np.all(np.max(np.abs(d), axis=1) >= 2)
        assert np.all(np.max(np.abs(d), axis=1) <= 3)
        offsets |= {tuple(v) for v in d}
        near = tree.near_list(t, lo, hi)
        assert len(near) == 27
        # near + interaction list = children of the parent's neighbours
        allc = {tuple(v) for v in np.concatenate([il, near])}
        assert len(allc) == 216
    assert len(offsets) == 316


def test_morton_interleave():
    c = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 3, 3], [2, 5, 1], [1023, 0, 1023]])
    k = tree.interleave(c, 10)
    assert list(k[:4]) == [1, 2, 4, 63]
    assert np.array_equal(tree.deinterleave(k, 10), c)
    # key of (2,5,1): x bits 0,1,0 ; y 1,0,1 ; z 1,0,0 -> groups (zyx) 110, 001, 010
    assert int(k[4]) == 0b010_001_110


def test_leaf_map_is_floor_and_clamped():
    lo = (0.0, 0.0, 0.0)
    pts = np.array([[0.0, 0.0, 0.0], [0.999999, 1.0, 3.999], [4.0, 4.0, 4.0], [-1e-9, 2.5, 1e9]])
    c = tree.leaf_coords(pts, lo, 1.0, 2)
    assert c.tolist() == [[0, 0, 0], [0, 1, 3], [3, 3, 3], [0, 2, 3]]
