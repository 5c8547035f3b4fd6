"""Selected rows of the H^2 product y = A x, read from the flat arrays of the
C ABI (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

For geometries whose H^2 data is too large for the dictionary form of
h2build.H2 in host memory, this evaluates rows i of y = A x straight from the
definition (Sec. III.C, Eqs. 8-9; the near blocks of Sec. IV.A):

    y_i = sum_{s in N(t)} Z^{t,s}[i, :] x|_s
        + sum_{a ancestor-or-self of t} u_i^(a) sum_{s in R(a)} S^{a,s} xh^s

with t the leaf holding row i, N(t) its near-field partners, R(a) the
admissible partners of a, u_i^(a) row i of the expanded row basis of a
(u_i^(t) is row i of U^t, and u_i^(parent) = u_i^(child) T^child, Eq. 9), and
xh^s = W^{sT} x|_s the column coefficients (xh^leaf = W^{leaf T} x|_leaf,
xh^t = T^{t1 T} xh^{t1} + T^{t2 T} xh^{t2}). Every block is read from the flat
arrays as stored (complex64 or complex128) and promoted to complex128; x may
hold several columns. No blocking or reordering beyond these sums.

Pinned by tests/test_oracle_h2.py: on small operators every row equals the
oracle's full product h2mv.h2_matvec.
"""
from __future__ import annotations

import numpy as np


def _blk(flat, off, r, c):
    return np.asarray(flat[int(off):int(off) + r * c]).reshape(c, r).T.astype(np.complex128)


def matvec_rows(a, x: np.ndarray, rows) -> np.ndarray:
    """a: object with the C ABI arrays (n, level_ptr, child, begin, size, rank,
    U, U_off, W, W_off, T, T_off, adm_ptr, adm_col, S, S_off, near_ptr,
    near_col, Z, Z_off), tree order; x: (n,) or (n, R); rows: tree-order row
    indices. Returns y[rows] (len(rows),) or (len(rows), R), complex128."""
    x = np.asarray(x, dtype=np.complex128)
    vec = x.ndim == 1
    if vec:
        x = x[:, None]
    nc = len(a.size)
    child = np.asarray(a.child, dtype=np.int64).reshape(nc, 2)
    parent = np.full(nc, -1, dtype=np.int64)
    for t in range(nc):
        if child[t, 0] >= 0:
            parent[child[t]] = t
    rank = np.asarray(a.rank, dtype=np.int64)
    size = np.asarray(a.size, dtype=np.int64)
    begin = np.asarray(a.begin, dtype=np.int64)
    Wf, Wo = (a.W, a.W_off) if a.W is not None else (a.U, a.U_off)
    # column coefficients xh^t, leaves first, then up the tree (children follow parents in BFS order)
    xh = {}
    for t in range(nc - 1, -1, -1):
        k = int(rank[t])
        if child[t, 0] < 0:
            if k:
                W = _blk(Wf, Wo[t], int(size[t]), k)
                xh[t] = W.T @ x[begin[t]:begin[t] + size[t]]
            else:
                xh[t] = np.zeros((0, x.shape[1]), dtype=np.complex128)
        else:
            acc = np.zeros((k, x.shape[1]), dtype=np.complex128)
            if k:
                for c in child[t]:
                    kc = int(rank[c])
                    if kc:
                        T = _blk(a.T, a.T_off[c], kc, k)
                        acc += T.T @ xh[int(c)]
            xh[t] = acc
    leaves = np.array([t for t in range(nc) if child[t, 0] < 0], dtype=np.int64)
    lb = begin[leaves]
    order = np.argsort(lb)
    leaves, lb = leaves[order], lb[order]
    out = np.zeros((len(rows), x.shape[1]), dtype=np.complex128)
    for r_i, i in enumerate(np.asarray(rows, dtype=np.int64)):
        t = int(leaves[np.searchsorted(lb, i, side="right") - 1])
        li = int(i - begin[t])
        # near field
        for j in range(int(a.near_ptr[t]), int(a.near_ptr[t + 1])):
            s = int(a.near_col[j])
            Zb = _blk(a.Z, a.Z_off[j], int(size[t]), int(size[s]))
            out[r_i] += Zb[li] @ x[begin[s]:begin[s] + size[s]]
        # far field: row i of the expanded basis, level by level up the tree
        u = _blk(a.U, a.U_off[t], int(size[t]), int(rank[t]))[li] if rank[t] else np.zeros(0, np.complex128)
        c = t
        while c >= 0:
            kc = int(rank[c])
            if kc:
                for j in range(int(a.adm_ptr[c]), int(a.adm_ptr[c + 1])):
                    s = int(a.adm_col[j])
                    ks = int(rank[s])
                    if ks:
                        out[r_i] += u @ (_blk(a.S, a.S_off[j], kc, ks) @ xh[s])
            p = int(parent[c])
            if p >= 0:
                kp = int(rank[p])
                u = u @ _blk(a.T, a.T_off[c], kc, kp) if (kc and kp) else np.zeros(kp, np.complex128)
            c = p
    return out[:, 0] if vec else out
