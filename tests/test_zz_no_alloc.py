"""The scratch-free product entry point (h2_matvec_noalloc), for callers that
must not call the CUDA allocator while running (a step inside a framework whose
caching allocator owns the device memory, or a real-time loop that cannot take
cudaMalloc's synchronisation).

- Its result equals the ordinary h2_matvec on the same operator and input, and
  the FP64 oracle's product on the same data within the FP32 tolerance, on two
  consecutive calls: the shared static array keeps the previous call's
  contents, so the second call checks that the entry point clears it.
- An operator whose coefficient vectors (2 x the sum of the ranks) exceed the
  array's H2_NOALLOC_MAX_COEF entries is refused with H2_ERR_ARG before any
  device work: y keeps its contents.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import cases
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

H2_ERR_ARG = 1
H2_NOALLOC_MAX_COEF = 1048576


def _entry():
    from paper_1703_01175_gb300 import build, h2
    build.build_all()
    L = h2.lib()
    L.h2_matvec_noalloc.restype = ctypes.c_int
    L.h2_matvec_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return h2, L


def test_noalloc_matches_matvec_and_oracle():
    h2, L = _entry()
    case = cases.get("cube12")
    A = h2.H2Matrix(case.arrays())
    try:
        stream = torch.cuda.current_stream().cuda_stream
        for seed in (1, 2):
            xh = synth.random_complex(A.n, seed)
            x = torch.from_numpy(xh.astype(np.complex64)).cuda()
            y_ref = A.matvec(x)
            y = torch.full_like(x, complex(7.0, -3.0))
            st = L.h2_matvec_noalloc(A.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     ctypes.c_void_p(stream))
            assert st == 0, L.h2_last_error().decode()
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
            assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
            y_or = case.oracle_matvec(xh)
            assert np.linalg.norm(a - y_or) <= 1e-5 * np.linalg.norm(y_or)
    finally:
        A.close()


def _wide_operator(h2):
    """A valid H^2 operator with more coefficients than the static array holds:
    a complete binary tree over N = 2^18 unknowns (leaves of 2 unknowns), the
    two children of every cluster admissible with each other, each leaf near
    only itself; ranks 2 at the leaves, 3 above them and 0 at the root, so the
    sum of the ranks is 655,354 and the product needs 1,310,708 coefficients."""
    nlev = 18
    n = 1 << nlev
    nc = (1 << nlev) - 1
    t = np.arange(nc, dtype=np.int64)
    lev = np.zeros(nc, dtype=np.int64)
    for l in range(nlev):
        lev[(1 << l) - 1:(1 << (l + 1)) - 1] = l
    idx = t - ((1 << lev) - 1)
    size = (n >> lev).astype(np.int32)
    begin = (idx * size).astype(np.int32)
    leaf = lev == nlev - 1
    child = np.where(leaf[:, None], -1, np.stack([2 * t + 1, 2 * t + 2], axis=1)).astype(np.int32).reshape(-1)
    rank = np.where(leaf, 2, 3).astype(np.int32)
    rank[0] = 0
    level_ptr = np.array([(1 << l) - 1 for l in range(nlev + 1)], dtype=np.int32)
    rng = np.random.default_rng(5)

    def cplx(m):
        return (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64)

    U_off = np.zeros(nc, dtype=np.int64)
    U_off[leaf] = 4 * np.arange(int(leaf.sum()))
    U = cplx(4 * int(leaf.sum()))
    parent = np.where(t > 0, (t - 1) // 2, -1)
    has_t = (t > 0) & (rank[np.maximum(parent, 0)] > 0)
    tsz = np.where(has_t, rank * rank[np.maximum(parent, 0)], 0).astype(np.int64)
    T_off = np.concatenate([[0], np.cumsum(tsz)[:-1]])
    T = cplx(int(tsz.sum()))
    sib = np.where(t % 2 == 1, t + 1, t - 1)
    adm_ptr = np.concatenate([[0, 0], np.arange(1, nc)]).astype(np.int32)
    adm_col = sib[1:].astype(np.int32)
    ssz = (rank[1:].astype(np.int64) * rank[sib[1:]])
    S_off = np.concatenate([[0], np.cumsum(ssz)[:-1]])
    S = cplx(int(ssz.sum()))
    nleaf = int(leaf.sum())
    near_ptr = np.concatenate([np.zeros(nc - nleaf + 1), np.arange(1, nleaf + 1)]).astype(np.int32)
    near_col = t[leaf].astype(np.int32)
    Z_off = 4 * np.arange(nleaf, dtype=np.int64)
    Z = cplx(4 * nleaf)
    arrs = h2.H2Arrays(n, level_ptr, child, begin, size, rank, U, U_off, None, None, T, T_off,
                       adm_ptr, adm_col, S, S_off, near_ptr, near_col, Z, Z_off)
    assert 2 * int(rank.astype(np.int64).sum()) > H2_NOALLOC_MAX_COEF
    return arrs


def test_noalloc_refuses_operators_above_the_limit():
    h2, L = _entry()
    A = h2.H2Matrix(_wide_operator(h2))
    try:
        x = torch.ones(A.n, dtype=torch.complex64, device="cuda")
        y = torch.full_like(x, complex(7.0, -3.0))
        st = L.h2_matvec_noalloc(A.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == H2_ERR_ARG
        assert "limit" in L.h2_last_error().decode()
        torch.cuda.synchronize()
        assert bool(torch.all(y == complex(7.0, -3.0)))
        # the ordinary entry point still computes the product of this operator
        y2 = A.matvec(x)
        torch.cuda.synchronize()
        assert bool(torch.all(torch.isfinite(torch.view_as_real(y2))))
    finally:
        A.close()
