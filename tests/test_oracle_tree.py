"""Pins of the oracle's cluster tree and block partition (Sec. III.A, Eq. 4)."""
import numpy as np
import pytest

import synth
from oracle import tree as otree

CASES = [
    ("cube8", synth.uniform_grid((8, 8, 8), (1 / 16,) * 3, 4.0), 64),
    ("ragged", synth.uniform_grid((7, 5, 6), (1 / 16,) * 3, 4.0), 40),
    ("slab", synth.uniform_grid((12, 10, 2), (1 / 32, 1 / 32, 0.03), 3.0), 30),
    ("array", synth.cube_array_1d(12, 2, 1 / 16, 0.25, 2.54), 24),
]


@pytest.mark.parametrize("name,v,n_min", CASES, ids=[c[0] for c in CASES])
def test_tree_invariants(name, v, n_min):
    tr = otree.build_tree(v.centres, n_min)
    assert sorted(tr.perm.tolist()) == list(range(v.nv))
    assert tr.vbegin[0] == 0 and tr.vsize[0] == v.nv
    for t in range(tr.nc):
        if tr.is_leaf(t):
            assert 3 * tr.vsize[t] <= n_min
        else:
            c1, c2 = tr.child[t]
            assert 3 * tr.vsize[t] > n_min
            assert tr.parent[c1] == t and tr.parent[c2] == t
            assert tr.level[c1] == tr.level[t] + 1
            assert tr.vbegin[c1] == tr.vbegin[t]
            assert tr.vbegin[c2] == tr.vbegin[c1] + tr.vsize[c1]
            assert tr.vsize[c1] + tr.vsize[c2] == tr.vsize[t]
            assert 0 <= tr.vsize[c1] - tr.vsize[c2] <= 1  # balanced splitting
        # the bounding box covers exactly the cluster's voxels
        pts = v.centres[tr.perm[tr.vbegin[t]:tr.vbegin[t] + tr.vsize[t]]]
        assert np.array_equal(pts.min(0), tr.lo[t]) and np.array_equal(pts.max(0), tr.hi[t])
    leaves = tr.leaves()
    cover = np.zeros(v.nv, dtype=int)
    for t in leaves:
        cover[tr.vbegin[t]:tr.vbegin[t] + tr.vsize[t]] += 1
    assert np.all(cover == 1)
    # BFS order by level
    assert np.all(np.diff(tr.level) >= 0)


def test_split_rule_gives_2x4x4_leaves_on_32_cube():
    v = synth.uniform_grid((32, 32, 32), (1 / 16,) * 3, 4.0)
    tr = otree.build_tree(v.centres, 96)
    leaves = tr.leaves()
    assert len(leaves) == 1024
    ext = np.round((tr.hi[leaves] - tr.lo[leaves]) * 16).astype(int)
    assert np.all(ext == np.array([1, 3, 3]))


@pytest.mark.parametrize("name,v,n_min", CASES, ids=[c[0] for c in CASES])
def test_partition_tiles_matrix_once(name, v, n_min):
    tr = otree.build_tree(v.centres, n_min)
    pa = otree.partition(tr, 1.0)
    n = tr.n
    cov = np.zeros((n, n), dtype=np.int32)
    for t, s in pa.adm + pa.near:
        cov[np.ix_(tr.rows(t), tr.rows(s))] += 1
    assert np.all(cov == 1)
    for t, s in pa.near:
        assert tr.is_leaf(t) and tr.is_leaf(s)
        assert not otree.admissible(tr, t, s, 1.0)
    for t, s in pa.adm:
        # brute force Eq. 4 on the voxel centres' boxes
        P = v.centres[tr.perm[tr.vbegin[t]:tr.vbegin[t] + tr.vsize[t]]]
        Q = v.centres[tr.perm[tr.vbegin[s]:tr.vbegin[s] + tr.vsize[s]]]
        dP = np.linalg.norm(P.max(0) - P.min(0))
        dQ = np.linalg.norm(Q.max(0) - Q.min(0))
        gap = np.maximum(0, np.maximum(P.min(0) - Q.max(0), Q.min(0) - P.max(0)))
        assert max(dP, dQ) <= np.linalg.norm(gap) and np.linalg.norm(gap) > 0
        # maximality: the parent pair (when both have parents) is not admissible
        pt, ps = tr.parent[t], tr.parent[s]
        if pt >= 0 and ps >= 0 and tr.level[t] == tr.level[s]:
            assert not otree.admissible(tr, pt, ps, 1.0)
    # symmetric partition
    assert sorted((s, t) for t, s in pa.adm) == pa.adm
    assert sorted((s, t) for t, s in pa.near) == pa.near
