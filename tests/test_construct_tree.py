"""The product-side constructor against the oracle, on the host.

- Cluster tree and block partition (Sec. III.A, Eq. 4): the constructor's
  level-synchronous bisection and its partition recursion are written
  independently of the oracle's; both must give the same tree order, the same
  clusters and children, and the same admissible and near-field pairs.
- Minimal rank (Abstract; Sec. III.B, Eq. 7; Sec. III.C, Eqs. 11 and 15): the
  rank the constructor gives every cluster -- from Stage I cross approximations
  and the Stage II Gram and projected-Gram eigenvalues -- equals the rank of the
  truncated SVD of the dense G_(t) at the same eps (every row of t against every
  column admissible with t or an ancestor of t, Eq. 10). Leaves must agree
  exactly; non-leaf clusters, whose Stage II matrix is G_(t) projected on the
  children's truncated bases, within max(2, 5 %).
"""
import math

import numpy as np
import pytest

import synth
from oracle import h2build, tree as otree, vie

TREE_CASES = [
    ("ragged", synth.uniform_grid((7, 5, 6), (1 / 16,) * 3, 4.0), 40),
    ("odd", synth.random_eps_grid((7, 5, 5), (1 / 16,) * 3, 2.0, 6.0, seed=9), 40),
    ("slab", synth.uniform_grid((24, 20, 2), (1 / 32, 1 / 32, 0.03), 3.0), 60),
    ("array", synth.cube_array_1d(40, 2, 1 / 16, 0.25, 2.54), 24),
    ("cube12_leaf96", synth.uniform_grid((12, 12, 12), (1 / 16,) * 3, 4.0), 96),
    ("void", synth.void_grid((10, 9, 8), (1 / 16,) * 3, 4.0, 0.1, seed=7), 96),
]


@pytest.mark.parametrize("name,v,n_min", TREE_CASES, ids=[c[0] for c in TREE_CASES])
def test_tree_and_partition_match_oracle(name, v, n_min):
    from paper_1703_01175_gb300 import construct
    ot = otree.build_tree(v.centres, n_min)
    op = otree.partition(ot, 1.0)
    ct = construct.cluster_tree(v.centres, n_min)
    adm, near = construct.block_partition(ct, 1.0)
    assert np.array_equal(ct.perm, ot.perm)
    assert np.array_equal(ct.level_ptr, ot.level_ptr)
    assert np.array_equal(ct.child, ot.child)
    assert np.array_equal(ct.vbegin, ot.vbegin) and np.array_equal(ct.vsize, ot.vsize)
    assert [tuple(map(int, p)) for p in adm] == [tuple(map(int, p)) for p in op.adm]
    assert [tuple(map(int, p)) for p in near] == [tuple(map(int, p)) for p in op.near]


@pytest.fixture(scope="module")
def rank_case():
    from paper_1703_01175_gb300 import build, construct
    build.build_all()
    # 864 voxels, leaves of 14 voxels: three levels carry bases, ranks well below n_t
    v = synth.random_eps_grid((12, 12, 6), (1 / 16,) * 3, 2.0, 6.0, seed=21)
    arrs, tr, info = construct.build_vie_h2(v.centres, v.dv, v.eps_r, n_min=48, eta=1.0, eps=1e-4,
                                            out_dtype=np.complex128, threads=2)
    return v, arrs, tr


def test_constructor_ranks_are_svd_ranks(rank_case):
    v, arrs, tr = rank_case
    eps = 1e-4
    ot = otree.build_tree(v.centres, 48)
    op = otree.partition(ot, 1.0)
    assert np.array_equal(ot.perm, tr.perm)
    Kt = h2build.to_tree_order(vie.assemble_K(v.centres, v.dv, 2 * math.pi), ot)
    F = h2build.far_columns(ot, op)
    checked = {True: 0, False: 0}
    truncated = 0
    for t in range(ot.nc):
        G = Kt[np.ix_(ot.rows(t), F[t])]
        k_svd = 0 if G.shape[1] == 0 else h2build.truncation_rank(np.linalg.svd(G, compute_uv=False), eps)
        k = int(arrs.rank[t])
        if ot.is_leaf(t):
            assert k == k_svd, (t, k, k_svd)
        else:
            assert abs(k - k_svd) <= max(2, math.ceil(0.05 * k_svd)), (t, k, k_svd)
        if k_svd:
            checked[ot.is_leaf(t)] += 1
            truncated += k_svd < len(ot.rows(t))
    # the case exercises both kinds of cluster, and truncation happens
    assert checked[True] >= 32 and checked[False] >= 16 and truncated >= 32
