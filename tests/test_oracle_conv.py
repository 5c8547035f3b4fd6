"""Pins of the oracle's 3-D convolution: brute-force loops on a tiny grid and
central finite differences of a scalar loss for the data, weight and bias
gradients."""
import numpy as np

import synth
from oracle import conv


def _rand(shape, seed, stream):
    return (2.0 * synth.uniform(seed, int(np.prod(shape)), stream=stream) - 1.0).reshape(shape)


def test_forward_matches_bruteforce():
    dims, B, Cin, Cout = (3, 4, 2), 2, 3, 4
    x = _rand((B, 24, Cin), 1, 0)
    w = _rand((Cout, 27, Cin), 1, 1)
    b = _rand((Cout,), 1, 2)
    a = conv.conv3d_forward(x, w, b, B, dims)
    r = conv.conv3d_bruteforce(x, w, b, B, dims)
    assert np.abs(a - r).max() <= 1e-13


def test_gradients_by_finite_differences():
    dims, B, Cin, Cout = (3, 2, 3), 2, 2, 3
    V = 18
    x = _rand((B, V, Cin), 2, 0)
    w = _rand((Cout, 27, Cin), 2, 1)
    b = _rand((Cout,), 2, 2)
    G = _rand((B, V, Cout), 2, 3)          # loss L = sum(G * z)

    def L(x_, w_, b_):
        return float(np.sum(G * conv.conv3d_forward(x_, w_, b_, B, dims)))

    dx = conv.conv3d_backward_data(G, w, B, dims)
    dw, db = conv.conv3d_backward_weight(G, x, B, dims, Cin, Cout)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 7, 1), (0, 17, 1)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (L(x + e, w, b) - L(x - e, w, b)) / (2 * h)
        assert abs(fd - dx[idx]) <= 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0, 0), (2, 13, 1), (1, 26, 0)]:
        e = np.zeros_like(w)
        e[idx] = h
        fd = (L(x, w + e, b) - L(x, w - e, b)) / (2 * h)
        assert abs(fd - dw[idx]) <= 1e-6 * max(1.0, abs(fd))
    for co in range(Cout):
        e = np.zeros_like(b)
        e[co] = h
        fd = (L(x, w, b + e) - L(x, w, b - e)) / (2 * h)
        assert abs(fd - db[co]) <= 1e-6 * max(1.0, abs(fd))


def test_identity_kernel_and_shift():
    dims, B = (4, 3, 2), 1
    x = _rand((B, 24, 1), 3, 0)
    w = np.zeros((1, 27, 1))
    w[0, 13, 0] = 1.0                       # centre tap: identity
    assert np.allclose(conv.conv3d_forward(x, w, None, B, dims), x)
    w = np.zeros((1, 27, 1))
    w[0, 14, 0] = 1.0                       # +x neighbour
    out = conv.conv3d_forward(x, w, None, B, dims).reshape(2, 3, 4)
    g = x.reshape(2, 3, 4)
    assert np.allclose(out[:, :, :3], g[:, :, 1:]) and np.allclose(out[:, :, 3], 0.0)
