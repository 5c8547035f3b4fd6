"""Dense and H^2 matrix-vector products (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

The H^2 product follows Sec. IV.B literally, with the cluster bases expanded
from the leaf bases and transfers by Eq. 9:

  1) forward transformation   xh^s = W^{sT} x|_s            for all clusters s
  2) coupling multiplication  yh^t = sum_{s in R^t} S^{t,s} xh^s
  3) backward transformation  y_i += sum_{t containing i} (U^t yh^t)_i
  4) inadmissible blocks      y|_t += Z^{t,s} x|_s          (full products)

(W = U for the symmetric form of Eq. 8.) All vectors are in tree order and may
be (n,) or (n, r) for several right-hand sides.

Parity: pinned against the dense product (tests/test_oracle_h2.py).
"""
from __future__ import annotations

import numpy as np

from .h2build import H2


def expand_level_bases(h2: H2, which: str = "U"):
    """Yield (level, {t: expanded basis}) from the deepest level to the root,
    keeping only two levels in memory. which = "U" (rows) or "W" (columns)."""
    tree = h2.tree
    leafb = h2.U if which == "U" or h2.W is None else h2.W
    nlev = len(tree.level_ptr) - 1
    below = {}
    for lev in range(nlev - 1, -1, -1):
        cur = {}
        for t in range(int(tree.level_ptr[lev]), int(tree.level_ptr[lev + 1])):
            if tree.is_leaf(t):
                cur[t] = leafb[t]
            else:
                c1, c2 = (int(c) for c in tree.child[t])
                cur[t] = np.vstack([below[c1] @ h2.T[c1], below[c2] @ h2.T[c2]])
        yield lev, cur
        # leaves of shallower levels may still be needed as children: keep them
        below = cur


def h2_matvec(h2: H2, x: np.ndarray) -> np.ndarray:
    """y = A_H2 x, steps 1-4 above (FP64)."""
    tree = h2.tree
    x = np.asarray(x, dtype=np.complex128)
    xh = {}
    for _, bases in expand_level_bases(h2, "W"):
        for t, B in bases.items():
            xh[t] = B.T @ x[tree.rows(t)]
    yh = {}
    for (t, s), S in h2.S.items():
        v = S @ xh[s]
        yh[t] = yh[t] + v if t in yh else v
    y = np.zeros_like(x)
    for _, bases in expand_level_bases(h2, "U"):
        for t, B in bases.items():
            if t in yh:
                y[tree.rows(t)] += B @ yh[t]
    for (t, s), Zb in h2.Z.items():
        y[tree.rows(t)] += Zb @ x[tree.rows(s)]
    return y


def h2_dense(h2: H2) -> np.ndarray:
    """The full matrix the H^2 data represents (small cases only)."""
    tree = h2.tree
    A = np.zeros((tree.n, tree.n), dtype=np.complex128)
    Ux, Wx = {}, {}
    for _, b in expand_level_bases(h2, "U"):
        Ux.update(b)
    for _, b in expand_level_bases(h2, "W"):
        Wx.update(b)
    for (t, s), S in h2.S.items():
        A[np.ix_(tree.rows(t), tree.rows(s))] += Ux[t] @ S @ Wx[s].T
    for (t, s), Zb in h2.Z.items():
        A[np.ix_(tree.rows(t), tree.rows(s))] += Zb
    return A
