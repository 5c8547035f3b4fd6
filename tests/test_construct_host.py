"""Product-side constructor (Stage I grouped ACA + reduced SVD, Stage II
Gram projections and couplings) on a small random-permittivity grid, on the
host:

- the stored couplings are exactly symmetric per admissible pair,
  S^{s,t} = (S^{t,s})^T, as Eq. 8 with one basis per cluster gives for the
  complex-symmetric kernel (the couplings-once product relies on it);
- the constructed H^2 product (the oracle's FP64 product of the arrays)
  matches the oracle's dense E-VIE matrix within 10 eps.
"""
import numpy as np
import pytest

import synth
from oracle import h2io, h2mv, vie


@pytest.fixture(scope="module")
def built():
    from paper_1703_01175_gb300 import build, construct
    build.build_all()
    v = synth.random_eps_grid((8, 8, 6), (1 / 16,) * 3, 2.0, 6.0, seed=21)   # 384 voxels, N = 1152
    arrs, tr, info = construct.build_vie_h2(v.centres, v.dv, v.eps_r, n_min=48, eta=1.0, eps=1e-4,
                                            out_dtype=np.complex128, threads=2)
    return v, arrs, tr


def test_couplings_symmetric_per_pair(built):
    v, a, tr = built
    blocks = {}
    for t in range(len(a.rank)):
        for j in range(a.adm_ptr[t], a.adm_ptr[t + 1]):
            s = int(a.adm_col[j])
            r, c = int(a.rank[t]), int(a.rank[s])
            blocks[(t, s)] = np.asarray(a.S[a.S_off[j]:a.S_off[j] + r * c]).reshape(c, r).T
    assert blocks, "no admissible blocks"
    nonzero = 0
    for (t, s), b in blocks.items():
        assert (s, t) in blocks
        assert np.array_equal(b, blocks[(s, t)].T)
        nonzero += b.size > 0
    assert nonzero > 0


def test_product_matches_dense_vie(built):
    v, a, tr = built
    hZ = h2io.from_flat(a, tr.perm)
    idx = (3 * np.asarray(tr.perm)[:, None] + np.arange(3)[None, :]).reshape(-1)
    Zd = vie.assemble_Z(v.centres, v.dv, v.eps_r, 2 * np.pi)[np.ix_(idx, idx)]
    for seed in (1, 2):
        x = synth.random_complex(a.n, seed)
        yd = Zd @ x
        assert np.linalg.norm(h2mv.h2_matvec(hZ, x) - yd) <= 10 * 1e-4 * np.linalg.norm(yd)
