"""Minimal-rank nested H^2 build by truncated SVD (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Follows Sec. III.C with the Stage-I factorisation replaced by the exact dense
blocks (an A B^T form with zero error), so every rank is the SVD rank of the
matrix the paper's Stage II decomposes:

  * leaf t (Eqs. 10-12): G_(t) is the block of rows of t against every column
    cluster s that forms an admissible block with t or with any ancestor of t;
    its SVD, truncated at sigma_i > eps * sigma_1, gives the unitary basis V^t
    (the left singular vectors, equivalently the eigenvectors of G_(t) G_(t)^H);
  * non-leaf t, bottom-up (Eqs. 13-16): the same G_(t) projected on
    blkdiag(V^{t1}, V^{t2})^H is decomposed the same way and its left singular
    vectors P, split by block rows, are the transfer matrices T^{t1}, T^{t2};
    V^t = [V^{t1} T^{t1}; V^{t2} T^{t2}] (Eq. 9);
  * couplings (Eq. 18): S^{t,s} = V^{tH} K^{(t,s)} conj(V^s).

The bases are built for the complex-symmetric K (K = K^T), so one basis per
cluster represents K^{(t,s)} ~ V^t S^{t,s} V^{sT} (Eq. 8). The system matrix
Z = I - K diag(chi) then has row basis U^t = V^t, column basis
W^t = diag(chi|t) V^t (nested with the same transfers, since Eq. 9 acts on
rows), couplings -S^{t,s} and near blocks delta_ts I - K^{(t,s)} diag(chi|s).

A cluster whose G_(t) has no columns gets rank 0.

Pins (tests/test_oracle_h2.py): orthonormal bases and transfers, expanded
bases equal to the nested products, exact agreement with the dense product
when nothing is truncated, error of order eps otherwise, leaf ranks equal to
the SVD rank of the independently formed G_(t), and non-leaf ranks within two
of the SVD rank of the unprojected G_(t) (the paper's minimal-rank claim).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .tree import Tree, Partition


@dataclasses.dataclass
class H2:
    """An H^2 matrix in nested form. Rows/columns are in tree order.

    rank[t]    k_t
    U[t]       leaf row basis (n_t x k_t)
    W[t]       leaf column basis (n_t x k_t), or None when W = U
    T[t]       transfer of non-root t to its parent (k_t x k_parent)
    S[(t,s)]   coupling of admissible block (k_t x k_s): block ~ U^t S W^{sT}
    Z[(t,s)]   dense near-field block (n_t x n_s)
    """
    tree: Tree
    part: Partition
    rank: np.ndarray
    U: dict
    W: dict | None
    T: dict
    S: dict
    Z: dict


def truncation_rank(sigma: np.ndarray, eps: float) -> int:
    """Number of singular values above eps * sigma_1 (the reading of
    'prescribed accuracy' used for Eqs. 6, 7, 11 and 15)."""
    if sigma.size == 0 or sigma[0] == 0.0:
        return 0
    return int(np.count_nonzero(sigma > eps * sigma[0]))


def far_columns(tree: Tree, part: Partition) -> list:
    """F(t): tree-order column indices of every s admissible with t or with an
    ancestor of t (the columns of G_(t) in Eq. 10)."""
    partners = [[] for _ in range(tree.nc)]
    for t, s in part.adm:
        partners[t].append(s)
    out = []
    for t in range(tree.nc):
        cols = []
        for a in tree.ancestors_or_self(t):
            for s in partners[a]:
                cols.append(tree.rows(s))
        out.append(np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64))
    return out


def build_bases(Kt: np.ndarray, tree: Tree, part: Partition, eps: float):
    """Leaf bases, transfers and expanded bases of the symmetric K (tree order).

    Returns (rank, V_leaf, T, V_expanded)."""
    F = far_columns(tree, part)
    nc = tree.nc
    rank = np.zeros(nc, dtype=np.int64)
    Vx = {}      # expanded basis per cluster
    V_leaf, T = {}, {}
    for t in range(nc - 1, -1, -1):  # deepest clusters first (BFS order)
        rows = tree.rows(t)
        G = Kt[np.ix_(rows, F[t])]
        if tree.is_leaf(t):
            if G.shape[1] == 0:
                V = np.zeros((len(rows), 0), dtype=np.complex128)
            else:
                Uu, sig, _ = np.linalg.svd(G, full_matrices=False)
                V = Uu[:, :truncation_rank(sig, eps)]
            V_leaf[t] = V
            Vx[t] = V
        else:
            c1, c2 = (int(c) for c in tree.child[t])
            B1, B2 = Vx[c1], Vx[c2]
            k1, k2 = B1.shape[1], B2.shape[1]
            n1 = B1.shape[0]
            if G.shape[1] == 0 or k1 + k2 == 0:
                P = np.zeros((k1 + k2, 0), dtype=np.complex128)
            else:
                proj = np.vstack([B1.conj().T @ G[:n1], B2.conj().T @ G[n1:]])
                Pu, sig, _ = np.linalg.svd(proj, full_matrices=False)
                P = Pu[:, :truncation_rank(sig, eps)]
            T[c1] = P[:k1]
            T[c2] = P[k1:]
            Vx[t] = np.vstack([B1 @ T[c1], B2 @ T[c2]])
        rank[t] = Vx[t].shape[1]
    return rank, V_leaf, T, Vx


def build_h2_K(Kt: np.ndarray, tree: Tree, part: Partition, eps: float) -> H2:
    """Truncated-SVD H^2 of the symmetric K given densely in tree order."""
    rank, V_leaf, T, Vx = build_bases(Kt, tree, part, eps)
    S = {}
    for t, s in part.adm:
        blk = Kt[np.ix_(tree.rows(t), tree.rows(s))]
        S[(t, s)] = Vx[t].conj().T @ blk @ Vx[s].conj()
    Z = {}
    for t, s in part.near:
        Z[(t, s)] = Kt[np.ix_(tree.rows(t), tree.rows(s))].copy()
    return H2(tree, part, rank, V_leaf, None, T, S, Z)


def system_h2(hK: H2, chi_tree: np.ndarray) -> H2:
    """H^2 of Z = I - K diag(chi) from the H^2 of K (chi in tree order)."""
    tree = hK.tree
    W = {t: chi_tree[tree.rows(t)][:, None] * U for t, U in hK.U.items()}
    S = {ts: -blk for ts, blk in hK.S.items()}
    Z = {}
    for (t, s), blk in hK.Z.items():
        z = -blk * chi_tree[tree.rows(s)][None, :]
        if t == s:
            z = z + np.eye(z.shape[0])
        Z[(t, s)] = z
    return H2(tree, hK.part, hK.rank.copy(), dict(hK.U), W, dict(hK.T), S, Z)


def to_tree_order(A: np.ndarray, tree: Tree) -> np.ndarray:
    p = tree.unknown_perm()
    return A[np.ix_(p, p)]
