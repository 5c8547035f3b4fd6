"""Read an H^2 representation given as the flat arrays of the C ABI
(tree arrays, CSR block lists, element offsets; blocks column-major) into the
oracle's H2 form.

TEST INFRASTRUCTURE ONLY (see the package header). Pure data marshalling:
every block is copied as is (promoted to complex128), no arithmetic.
"""
from __future__ import annotations

import numpy as np

from .h2build import H2
from .tree import Partition, Tree


def from_flat(a, perm) -> H2:
    """a: an object with the attributes of the C ABI arrays (n, level_ptr,
    child, begin, size, rank, U, U_off, W, W_off, T, T_off, adm_ptr, adm_col,
    S, S_off, near_ptr, near_col, Z, Z_off); perm: tree position -> voxel."""
    nc = len(a.size)
    child = np.asarray(a.child, dtype=np.int64).reshape(nc, 2)

    def blk(flat, off, r, c):
        return np.asarray(flat[off:off + r * c]).reshape(c, r).T.astype(np.complex128)

    parent = np.full(nc, -1, dtype=np.int64)
    for t in range(nc):
        if child[t, 0] >= 0:
            parent[child[t]] = t
    leaves = [t for t in range(nc) if child[t, 0] < 0]
    rank = np.asarray(a.rank, dtype=np.int64)
    size = np.asarray(a.size, dtype=np.int64)
    U = {t: blk(a.U, a.U_off[t], size[t], rank[t]) for t in leaves}
    W = None if a.W is None else {t: blk(a.W, a.W_off[t], size[t], rank[t]) for t in leaves}
    T = {t: blk(a.T, a.T_off[t], rank[t], rank[parent[t]]) for t in range(1, nc)}
    S, Z = {}, {}
    adm, near = [], []
    for t in range(nc):
        for j in range(a.adm_ptr[t], a.adm_ptr[t + 1]):
            s = int(a.adm_col[j])
            S[(t, s)] = blk(a.S, a.S_off[j], rank[t], rank[s])
            adm.append((t, s))
        for j in range(a.near_ptr[t], a.near_ptr[t + 1]):
            s = int(a.near_col[j])
            Z[(t, s)] = blk(a.Z, a.Z_off[j], size[t], size[s])
            near.append((t, s))
    level = np.zeros(nc, dtype=np.int64)
    lp = np.asarray(a.level_ptr, dtype=np.int64)
    for l in range(len(lp) - 1):
        level[lp[l]:lp[l + 1]] = l
    tree = Tree(int(a.n) // 3, np.asarray(perm, dtype=np.int64), level, parent, child,
                np.asarray(a.begin, dtype=np.int64) // 3, size // 3,
                np.zeros((nc, 3)), np.zeros((nc, 3)), lp)
    return H2(tree, Partition(adm, near), rank, U, W, T, S, Z)
