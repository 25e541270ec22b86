"""Plain numpy octree for checking the GPU tree bit for bit.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows the hierarchical space decomposition and the list definitions of
Sec. 2.3 ("Hierarchical space decomposition", "Overview of the algorithm"):

* uniform-depth octree with k = 2^L leaf boxes per axis (Sec. 3.2.3);
* a box's near domain is itself plus its nearest neighbours, i.e. the boxes
  of the same level whose integer coordinates differ by at most one on every
  axis (Chebyshev distance <= 1);
* a box's interaction list: take the children of every box within
  Chebyshev distance 1 of its parent and drop those within Chebyshev
  distance 1 of the box itself; lists start at level 2.

Conventions the CUDA path must reproduce exactly (they are choices, not
paper facts): the point-to-leaf map is ``floor((x - lo) * inv_s)`` evaluated
as one rounded subtraction followed by one rounded multiplication in FP64,
clamped to [0, 2^L - 1]; Morton keys interleave x into bit 0, y into bit 1
and z into bit 2 of each 3-bit group; observers are ordered by (key,
original index).
"""
from __future__ import annotations

import numpy as np


def leaf_coords(pts: np.ndarray, lo, inv_s: float, L: int) -> np.ndarray:
    """Integer leaf coordinates (M, 3) of points (M, 3)."""
    pts = np.asarray(pts, dtype=np.float64)
    q = np.floor((pts - np.asarray(lo, dtype=np.float64)) * np.float64(inv_s))
    q = np.clip(q, 0, (1 << L) - 1)
    return q.astype(np.int64)


def interleave(c: np.ndarray, L: int) -> np.ndarray:
    """Morton keys of integer coordinates c (M, 3), L bits per axis."""
    c = np.asarray(c, dtype=np.uint64)
    key = np.zeros(c.shape[0], dtype=np.uint64)
    for bit in range(L):
        for a in range(3):
            key |= ((c[:, a] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(3 * bit + a)
    return key


def deinterleave(keys: np.ndarray, L: int) -> np.ndarray:
    keys = np.asarray(keys, dtype=np.uint64)
    c = np.zeros((keys.shape[0], 3), dtype=np.int64)
    for bit in range(L):
        for a in range(3):
            c[:, a] |= (((keys >> np.uint64(3 * bit + a)) & np.uint64(1)).astype(np.int64) << bit)
    return c


def sort_points(pts, lo, inv_s, L):
    """Keys and the stable (key, original index) order of the points."""
    keys = interleave(leaf_coords(pts, lo, inv_s, L), L)
    perm = np.argsort(keys, kind="stable")
    return keys, perm


def level_boxes(sorted_leaf_keys: np.ndarray, L: int):
    """Occupied boxes per level, from the sorted leaf keys of the points.
    Returns {level: sorted unique keys} for levels 0..L."""
    out = {}
    k = np.unique(sorted_leaf_keys)
    for lev in range(L, -1, -1):
        out[lev] = k
        k = np.unique(k >> np.uint64(3))
    return out


def source_rect(voxel_offset, n_vox, b: int, L: int, level: int):
    """Boxes at `level` that overlap the voxel block [a, a + n) (voxel units
    in the tree frame, leaf = b^3 voxels): inclusive integer bounds."""
    a = np.asarray(voxel_offset, dtype=np.int64)
    n = np.asarray(n_vox, dtype=np.int64)
    shift = L - level
    lo = (a // b) >> shift
    hi = ((a + n - 1) // b) >> shift
    return lo, hi


def in_rect(c, lo, hi):
    c = np.asarray(c)
    return np.all((c >= lo) & (c <= hi), axis=-1)


def near_list(t_coord, src_lo, src_hi):
    """Source boxes (integer coordinates, sorted by Morton key) within
    Chebyshev distance 1 of the target box, clipped to the source block."""
    t = np.asarray(t_coord, dtype=np.int64)
    d = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    c = t[None, :] + d
    c = c[in_rect(c, src_lo, src_hi)]
    return c


def interaction_list(t_coord, src_lo, src_hi):
    """Interaction list of a box: same-level boxes that are children of the
    parent's neighbours but are not neighbours themselves."""
    t = np.asarray(t_coord, dtype=np.int64)
    p = t >> 1
    cand = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                q = p + np.array([dx, dy, dz])
                for cz in (0, 1):
                    for cy in (0, 1):
                        for cx in (0, 1):
                            cand.append(2 * q + np.array([cx, cy, cz]))
    c = np.array(cand)
    far = np.max(np.abs(c - t[None, :]), axis=1) > 1
    c = c[far]
    c = c[in_rect(c, src_lo, src_hi)]
    return c


def sorted_by_morton(coords, L):
    if len(coords) == 0:
        return np.zeros(0, dtype=np.uint64)
    return np.sort(interleave(np.asarray(coords), L))


# ------------------------------------------------- Eqs. 14-19 work model
def neighbour_counts(k: int) -> np.ndarray:
    """Number of nearest neighbours of every box of a full k^3 grid
    (Sec. 3.2.3: 7 for corner, 11 for edge, 17 for face, 26 for interior
    boxes), counted by brute force."""
    c = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), -1).reshape(-1, 3)
    lo = np.maximum(c - 1, 0)
    hi = np.minimum(c + 1, k - 1)
    span = hi - lo + 1
    return np.prod(span, axis=1) - 1


def direct_work_sum(k: int) -> float:
    """sum over boxes of (N_B + 1/2): the per-box direct work of Eq. 14 in
    units of B^2 (B particles per box, large-B limit)."""
    return float(np.sum(neighbour_counts(k) + 0.5))
