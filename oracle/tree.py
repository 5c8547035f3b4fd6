"""Cluster tree and H^2 block partition (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. III.A: the unknowns are split recursively into two sub-domains of similar
size until a cluster holds no more than n_min (the "leafsize") unknowns; then,
starting from (root, root), a row cluster t and a column cluster s form an
admissible block if the strong admissibility condition (Eq. 4)

    max(diam(t), diam(s)) <= eta * dist(t, s)

holds, and otherwise their children are checked, down to the leaves, where the
remaining pairs become inadmissible (near-field) blocks.

Readings taken where the paper leaves details open:
  * the three field components of a voxel always stay in the same cluster, so
    the recursion splits voxels and a cluster of v voxels holds 3 v unknowns;
  * the split axis is the longest edge of the bounding box of the cluster's
    voxel centres (ties: x before y before z), at the median voxel along that
    axis (ties in coordinate broken by natural voxel index); an odd count puts
    the extra voxel in the first child;
  * a cluster is a leaf when 3 v <= n_min;
  * diam and dist are taken on the axis-aligned bounding boxes of the voxel
    centres; a pair at distance 0 is never admissible;
  * if exactly one of an inadmissible pair is a leaf, the other is split.

Pins (tests/test_oracle_tree.py): the leaves partition the unknowns, every
cluster is a contiguous range split into its two children, sizes of siblings
differ by at most one voxel, and the admissible and near blocks tile the N x N
index square exactly once, with near blocks only between leaves.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Tree:
    nv: int
    perm: np.ndarray        # tree position -> natural voxel index
    level: np.ndarray       # per cluster (BFS order)
    parent: np.ndarray      # -1 for the root
    child: np.ndarray       # (nc, 2), -1 for leaves
    vbegin: np.ndarray      # first voxel (tree position)
    vsize: np.ndarray       # number of voxels
    lo: np.ndarray          # (nc, 3) bounding box of voxel centres
    hi: np.ndarray
    level_ptr: np.ndarray   # clusters of level l: [level_ptr[l], level_ptr[l+1])

    @property
    def nc(self) -> int:
        return int(self.level.shape[0])

    @property
    def n(self) -> int:
        return 3 * self.nv

    @property
    def begin(self) -> np.ndarray:
        return 3 * self.vbegin

    @property
    def size(self) -> np.ndarray:
        return 3 * self.vsize

    def is_leaf(self, t: int) -> bool:
        return self.child[t, 0] < 0

    def leaves(self) -> np.ndarray:
        return np.nonzero(self.child[:, 0] < 0)[0]

    def rows(self, t: int) -> np.ndarray:
        """Tree-order unknown indices of cluster t."""
        b = 3 * int(self.vbegin[t])
        return np.arange(b, b + 3 * int(self.vsize[t]))

    def unknown_perm(self) -> np.ndarray:
        """Tree-order unknown index -> natural unknown index."""
        return (3 * self.perm[:, None] + np.arange(3)[None, :]).reshape(-1)

    def ancestors_or_self(self, t: int):
        out = []
        while t >= 0:
            out.append(t)
            t = int(self.parent[t])
        return out


def _split_axis(lo, hi) -> int:
    ext = hi - lo
    m = ext.max()
    for ax in range(3):
        if ext[ax] >= m * (1.0 - 1e-12):
            return ax
    return 0


def build_tree(centres: np.ndarray, n_min: int) -> Tree:
    """Balanced binary cluster tree of the voxels (Sec. III.A)."""
    centres = np.asarray(centres, dtype=np.float64)
    nv = centres.shape[0]
    if nv == 0:
        raise ValueError("empty voxel set")
    # Recursive split producing nodes with explicit voxel lists.
    nodes = []  # (voxels, parent, depth)

    def split(vox, parent, depth):
        idx = len(nodes)
        nodes.append([vox, parent, depth, -1, -1])
        if 3 * len(vox) <= n_min or len(vox) < 2:
            return idx
        pts = centres[vox]
        ax = _split_axis(pts.min(axis=0), pts.max(axis=0))
        order = np.lexsort((vox, pts[:, ax]))  # by coordinate, then voxel index
        srt = vox[order]
        h = (len(vox) + 1) // 2
        c1 = split(srt[:h], idx, depth + 1)
        c2 = split(srt[h:], idx, depth + 1)
        nodes[idx][3] = c1
        nodes[idx][4] = c2
        return idx

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        split(np.arange(nv), -1, 0)
    finally:
        sys.setrecursionlimit(old)

    # Tree order of voxels: depth-first order of the leaves.
    vbegin_dfs = [0] * len(nodes)
    perm = []

    def place(i, start):
        vbegin_dfs[i] = start
        c1, c2 = nodes[i][3], nodes[i][4]
        if c1 < 0:
            perm.extend(nodes[i][0].tolist())
            return start + len(nodes[i][0])
        mid = place(c1, start)
        return place(c2, mid)

    sys.setrecursionlimit(max(old, 10000))
    try:
        place(0, 0)
    finally:
        sys.setrecursionlimit(old)

    # Renumber in breadth-first (level) order.
    order = sorted(range(len(nodes)), key=lambda i: (nodes[i][2], vbegin_dfs[i]))
    new_id = {old_i: new_i for new_i, old_i in enumerate(order)}
    nc = len(nodes)
    level = np.empty(nc, dtype=np.int64)
    parent = np.full(nc, -1, dtype=np.int64)
    child = np.full((nc, 2), -1, dtype=np.int64)
    vbegin = np.empty(nc, dtype=np.int64)
    vsize = np.empty(nc, dtype=np.int64)
    lo = np.empty((nc, 3))
    hi = np.empty((nc, 3))
    for old_i, nd in enumerate(nodes):
        t = new_id[old_i]
        level[t] = nd[2]
        parent[t] = new_id[nd[1]] if nd[1] >= 0 else -1
        if nd[3] >= 0:
            child[t] = (new_id[nd[3]], new_id[nd[4]])
        vbegin[t] = vbegin_dfs[old_i]
        vsize[t] = len(nd[0])
        pts = centres[nd[0]]
        lo[t] = pts.min(axis=0)
        hi[t] = pts.max(axis=0)
    nlev = int(level.max()) + 1
    level_ptr = np.searchsorted(level, np.arange(nlev + 1))
    return Tree(nv, np.asarray(perm, dtype=np.int64), level, parent, child,
                vbegin, vsize, lo, hi, level_ptr)


def diam(tree: Tree, t: int) -> float:
    d = tree.hi[t] - tree.lo[t]
    return float(np.sqrt(np.dot(d, d)))


def dist(tree: Tree, t: int, s: int) -> float:
    gap = np.maximum(0.0, np.maximum(tree.lo[t] - tree.hi[s], tree.lo[s] - tree.hi[t]))
    return float(np.sqrt(np.dot(gap, gap)))


def admissible(tree: Tree, t: int, s: int, eta: float) -> bool:
    """Strong admissibility, Eq. 4 (with dist > 0 required)."""
    d = dist(tree, t, s)
    return d > 0.0 and max(diam(tree, t), diam(tree, s)) <= eta * d


@dataclasses.dataclass
class Partition:
    adm: list   # (t, s) admissible blocks
    near: list  # (t, s) inadmissible leaf blocks


def partition(tree: Tree, eta: float) -> Partition:
    """Block partition by recursion from (root, root), Sec. III.A."""
    adm, near = [], []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        if admissible(tree, t, s, eta):
            adm.append((t, s))
            continue
        lt, ls = tree.is_leaf(t), tree.is_leaf(s)
        if lt and ls:
            near.append((t, s))
        elif lt:
            stack.extend((t, int(c)) for c in tree.child[s][::-1])
        elif ls:
            stack.extend((int(c), s) for c in tree.child[t][::-1])
        else:
            for c1 in tree.child[t][::-1]:
                for c2 in tree.child[s][::-1]:
                    stack.append((int(c1), int(c2)))
    adm.sort()
    near.sort()
    return Partition(adm, near)
