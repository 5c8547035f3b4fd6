"""Pins of the oracle's truncated-SVD H^2 build and H^2 product.

- bases are unitary and transfers have orthonormal columns (Eqs. 12, 16);
- every expanded basis captures its G_(t) to the prescribed accuracy;
- with no truncation the H^2 product equals the dense product (exact case);
- at eps = 1e-4 the product error is of order eps (Sec. IV.B);
- leaf ranks equal the SVD rank of G_(t) formed independently here, and the
  non-leaf ranks of the projected construction stay within two of the SVD rank
  of the unprojected G_(t) -- the paper's minimal-rank claim (Abstract,
  Sec. III.B-C);
- the relations that storing blocks once per pair relies on: couplings
  S^{s,t} = (S^{t,s})^T (Eq. 8, one basis per cluster, K complex symmetric)
  and near blocks Z^{s,t} = diag(1/chi_s) (Z^{t,s})^T diag(chi_t), t != s.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import h2build, h2mv, tree as otree, vie

K = 2.0 * math.pi


def _setup(v, n_min, eps):
    Kd = vie.assemble_K(v.centres, v.dv, K)
    tr = otree.build_tree(v.centres, n_min)
    pa = otree.partition(tr, 1.0)
    Kt = h2build.to_tree_order(Kd, tr)
    hK = h2build.build_h2_K(Kt, tr, pa, eps)
    chi = vie.chi_unknowns(v.eps_r)[tr.unknown_perm()]
    hZ = h2build.system_h2(hK, chi)
    Zt = np.eye(tr.n) - Kt * chi[None, :]
    return Kt, tr, pa, hK, hZ, Zt


@pytest.fixture(scope="module")
def cube8():
    return _setup(synth.workload("cube8").voxels, 64, 1e-4)


@pytest.fixture(scope="module")
def ragged():
    v = synth.random_eps_grid((7, 5, 6), (1 / 16,) * 3, 2.0, 6.0, seed=3)
    return _setup(v, 40, 1e-4)


def _G_of(tr, pa, Kt, t):
    """G_(t) of Eq. 10 formed directly: rows of t, columns of every s that is
    admissible with t or an ancestor of t."""
    anc = set()
    a = t
    while a >= 0:
        anc.add(a)
        a = tr.parent[a]
    cols = [tr.rows(s) for (u, s) in pa.adm if u in anc]
    if not cols:
        return np.zeros((len(tr.rows(t)), 0), dtype=complex)
    return Kt[np.ix_(tr.rows(t), np.concatenate(cols))]


@pytest.mark.parametrize("case", ["cube8", "ragged"])
def test_bases_unitary_and_capture_G(case, request):
    Kt, tr, pa, hK, hZ, Zt = request.getfixturevalue(case)
    for t, U in hK.U.items():
        if U.size:
            assert np.abs(U.conj().T @ U - np.eye(U.shape[1])).max() < 1e-12
    for t in range(tr.nc):
        if not tr.is_leaf(t):
            c1, c2 = tr.child[t]
            P = np.vstack([hK.T[c1], hK.T[c2]])
            if P.size:
                assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() < 1e-12
    Ux = {}
    for _, b in h2mv.expand_level_bases(hK, "U"):
        Ux.update(b)
    for t in range(tr.nc):
        G = _G_of(tr, pa, Kt, t)
        if G.size == 0:
            assert hK.rank[t] == 0
            continue
        V = Ux[t]
        res = G - V @ (V.conj().T @ G)
        # each level of nesting adds at most eps*||G|| of projection error
        depth = int(tr.level.max() - tr.level[t]) + 1
        assert np.linalg.norm(res, 2) <= 2 * depth * 1e-4 * np.linalg.norm(G, 2)


def test_exact_when_untruncated():
    v = synth.random_eps_grid((5, 4, 4), (1 / 16,) * 3, 2.0, 6.0, seed=5)
    Kt, tr, pa, hK, hZ, Zt = _setup(v, 24, 1e-15)
    assert len(pa.adm) > 0
    A = h2mv.h2_dense(hZ)
    assert np.abs(A - Zt).max() <= 1e-12 * np.abs(Zt).max()
    x = synth.random_complex(tr.n, 3)
    assert np.linalg.norm(h2mv.h2_matvec(hZ, x) - Zt @ x) <= 1e-12 * np.linalg.norm(Zt @ x)


@pytest.mark.parametrize("case", ["cube8", "ragged"])
def test_error_of_order_eps(case, request):
    Kt, tr, pa, hK, hZ, Zt = request.getfixturevalue(case)
    for seed in (1, 2):
        x = synth.random_complex(tr.n, seed)
        y = h2mv.h2_matvec(hZ, x)
        y0 = Zt @ x
        assert np.linalg.norm(y - y0) <= 10 * 1e-4 * np.linalg.norm(y0)
    # matrix form agrees with the product form
    A = h2mv.h2_dense(hZ)
    x = synth.random_complex(tr.n, 4)
    assert np.linalg.norm(A @ x - h2mv.h2_matvec(hZ, x)) <= 1e-12 * np.linalg.norm(A @ x)
    # admissible blocks of K are reproduced to ~eps relative to their G_(t)
    Ux = {}
    for _, b in h2mv.expand_level_bases(hK, "U"):
        Ux.update(b)
    for (t, s), S in hK.S.items():
        blk = Kt[np.ix_(tr.rows(t), tr.rows(s))]
        approx = Ux[t] @ S @ Ux[s].T
        Gn = np.linalg.norm(_G_of(tr, pa, Kt, t), 2) + np.linalg.norm(_G_of(tr, pa, Kt, s), 2)
        assert np.linalg.norm(blk - approx, 2) <= 20 * 1e-4 * Gn


@pytest.mark.parametrize("case", ["cube8", "ragged"])
def test_minimal_rank_claim(case, request):
    Kt, tr, pa, hK, hZ, Zt = request.getfixturevalue(case)
    for t in range(tr.nc):
        G = _G_of(tr, pa, Kt, t)
        if G.size == 0:
            assert hK.rank[t] == 0
            continue
        sig = scipy.linalg.svd(G, compute_uv=False, lapack_driver="gesvd")
        r_svd = int(np.sum(sig > 1e-4 * sig[0]))
        if tr.is_leaf(t):
            assert hK.rank[t] == r_svd
        else:
            assert abs(int(hK.rank[t]) - r_svd) <= 2


@pytest.mark.parametrize("case", ["cube8", "ragged"])
def test_pairwise_symmetry_of_stored_blocks(case, request):
    """Couplings of the system H^2 are transposes of each other per pair, and
    the near blocks of a pair are related through chi; checked on the FP64
    oracle data, so that a missing transpose or a chi on the wrong side of a
    block fails here."""
    Kt, tr, pa, hK, hZ, Zt = request.getfixturevalue(case)
    chi = np.diag(np.eye(tr.n) - Zt) / np.diag(Kt)   # recover chi from the dense forms
    n_pairs = 0
    for (t, s), S in hZ.S.items():
        if t < s and S.size:
            assert np.abs(hZ.S[(s, t)] - S.T).max() <= 1e-12 * max(1.0, np.abs(S).max())
            n_pairs += 1
    assert n_pairs > 0
    n_near = 0
    for (t, s), Z in hZ.Z.items():
        if t < s:
            rt, rs = tr.rows(t), tr.rows(s)
            partner = (Z.T * chi[rt][None, :]) / chi[rs][:, None]
            assert np.abs(hZ.Z[(s, t)] - partner).max() <= 1e-12 * np.abs(Z).max()
            n_near += 1
    assert n_near > 0


@pytest.mark.parametrize("case", ["cube8", "ragged"])
def test_row_product_equals_full_product(case, request):
    """oracle.h2rows evaluates rows of the H^2 product from the flat C-ABI
    arrays (Eqs. 8-9 written out per row); on these operators every row must
    equal the full product h2mv.h2_matvec, for one and for several columns,
    and with the flat arrays stored in complex64 (the rounded data)."""
    from oracle import h2rows
    from paper_1703_01175_gb300 import h2 as h2py
    Kt, tr, pa, hK, hZ, Zt = request.getfixturevalue(case)
    for dtype in (np.complex128, np.complex64):
        flat = h2py.arrays_from_blocks(tr.n, tr.level_ptr, tr.child, tr.begin, tr.size, hZ.rank,
                                       hZ.U, hZ.W, hZ.T, hZ.S, hZ.Z, dtype=dtype)
        X = synth.random_complex(tr.n, 3, cols=3)
        rows = np.arange(tr.n)
        Y = h2rows.matvec_rows(flat, X, rows)
        ref = np.stack([h2mv.h2_matvec(hZ, X[:, j]) for j in range(3)], axis=1)
        tol = 1e-12 if dtype == np.complex128 else 1e-6
        assert np.linalg.norm(Y - ref) <= tol * np.linalg.norm(ref)
        y1 = h2rows.matvec_rows(flat, X[:, 1], rows[::7])
        assert np.allclose(y1, Y[::7, 1], rtol=0, atol=1e-13 * np.abs(Y).max())
