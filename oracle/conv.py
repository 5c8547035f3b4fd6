"""3-D convolution of the learned preconditioner, forward and backward (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Layout: a batch is [B][V][C] on a Dx x Dy x Dz grid, voxel v = ix + Dx (iy + Dy iz);
weights [Cout][27][Cin] with tap t = dx + 3 (dy + 3 dz) reading the neighbour at
offset (dx - 1, dy - 1, dz - 1); zero padding outside the grid; bias [Cout].

  forward        z[b, v, co] = bias[co] + sum_{t, ci} w[co, t, ci] x[b, v + off(t), ci]
  data grad      dx[b, u, ci] = sum_{t, co} w[co, t, ci] dz[b, u - off(t), co]
  weight grad    dw[co, t, ci] = sum_{b, v} dz[b, v, co] x[b, v + off(t), ci]
  bias grad      db[co] = sum_{b, v} dz[b, v, co]

Each is the definition written with shifted views of a zero-padded grid, in
float64. Pins (tests/test_oracle_conv.py): a pure-loop brute force on a tiny
grid, and central finite differences of a scalar loss for every gradient.
"""
from __future__ import annotations

import numpy as np


def _grid(x, B, dims, C):
    Dx, Dy, Dz = dims
    return np.asarray(x, dtype=np.float64).reshape(B, Dz, Dy, Dx, C)


def _taps():
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                yield dx + 3 * (dy + 3 * dz), dx - 1, dy - 1, dz - 1


def _shift(xp, ox, oy, oz, dims):
    """View of the padded grid xp (pad 1) at offset (ox, oy, oz)."""
    Dx, Dy, Dz = dims
    return xp[:, 1 + oz:1 + oz + Dz, 1 + oy:1 + oy + Dy, 1 + ox:1 + ox + Dx, :]


def conv3d_forward(x, w, bias, B, dims, relu=False):
    Cout, _, Cin = w.shape
    g = _grid(x, B, dims, Cin)
    xp = np.pad(g, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros(g.shape[:4] + (Cout,))
    for t, ox, oy, oz in _taps():
        out += _shift(xp, ox, oy, oz, dims) @ np.asarray(w[:, t, :], dtype=np.float64).T
    if bias is not None:
        out += np.asarray(bias, dtype=np.float64)
    if relu:
        out = np.maximum(out, 0.0)
    return out.reshape(B, -1, Cout)


def conv3d_backward_data(dz, w, B, dims):
    Cout, _, Cin = w.shape
    g = _grid(dz, B, dims, Cout)
    gp = np.pad(g, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros(g.shape[:4] + (Cin,))
    for t, ox, oy, oz in _taps():
        out += _shift(gp, -ox, -oy, -oz, dims) @ np.asarray(w[:, t, :], dtype=np.float64)
    return out.reshape(B, -1, Cin)


def conv3d_backward_weight(dz, x, B, dims, Cin, Cout):
    gz = _grid(dz, B, dims, Cout).reshape(-1, Cout)
    gx = _grid(x, B, dims, Cin)
    xp = np.pad(gx, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    dw = np.zeros((Cout, 27, Cin))
    for t, ox, oy, oz in _taps():
        dw[:, t, :] = gz.T @ _shift(xp, ox, oy, oz, dims).reshape(-1, Cin)
    db = gz.sum(axis=0)
    return dw, db


def conv3d_bruteforce(x, w, bias, B, dims):
    """Seven nested loops, for tiny inputs only."""
    Dx, Dy, Dz = dims
    Cout, _, Cin = w.shape
    x = np.asarray(x, dtype=np.float64).reshape(B, Dx * Dy * Dz, Cin)
    out = np.zeros((B, Dx * Dy * Dz, Cout))
    for b in range(B):
        for iz in range(Dz):
            for iy in range(Dy):
                for ix in range(Dx):
                    v = ix + Dx * (iy + Dy * iz)
                    for co in range(Cout):
                        s = 0.0 if bias is None else float(bias[co])
                        for t in range(27):
                            nx, ny, nz = ix + t % 3 - 1, iy + (t // 3) % 3 - 1, iz + t // 9 - 1
                            if 0 <= nx < Dx and 0 <= ny < Dy and 0 <= nz < Dz:
                                u = nx + Dx * (ny + Dy * nz)
                                for ci in range(Cin):
                                    s += w[co, t, ci] * x[b, u, ci]
                        out[b, v, co] = s
    return out
