"""Full-size checks on the 32^3-voxel cube (N = 98,304, leaf 96, eps 1e-4):
the H^2 data of the GPU constructor loaded through h2_load_device, the launch
configuration bench.py times.

- FP32 product vs the oracle's FP64 H^2 product on the same data: 1e-5;
- sampled rows against the oracle's dense VIE rows, evaluated one by one:
  representation error within 10 eps;
- GMRES to 1e-4 (single right-hand side, and the batched solve with the c64
  and the double-float basis):
  the oracle's FP64 residual of each GPU solution <= 1.05e-4. This
  random-permittivity cube is hard for restarted GMRES: with m = 50 the
  residual stagnates near 7e-4 (the GPU and the oracle agree on that on the
  smaller 16^3 version), so the solves use m = 400;
- split-bf16 products of 8 right-hand sides: sampled columns within eps;
- double-float and FP64 accumulation agree to 1e-12;
- couplings and near blocks stored once per pair: within 1e-6 of full storage.
"""
import math

import numpy as np
import pytest

import synth
from oracle import h2io, h2mv, vie

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def full():
    from paper_1703_01175_gb300 import build, construct_gpu, h2
    build.build_all()
    w = synth.workload("cube32")
    v = w.voxels
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps)
    arrs, perm = dh.to_host(), dh.perm
    A = h2.H2Matrix.from_device(dh)
    dh.free()
    hZ = h2io.from_flat(arrs, perm)
    yield w, arrs, perm, A, hZ
    A.close()


def test_full_size_product_matches_oracle(full):
    w, arrs, perm, A, hZ = full
    x = synth.random_complex(arrs.n, 21)
    y = A.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    y_or = h2mv.h2_matvec(hZ, x)
    assert np.linalg.norm(y - y_or) <= 1e-5 * np.linalg.norm(y_or)
    assert np.abs(y - y_or).max() <= 1e-5 * np.abs(y_or).max()
    # sampled rows of the dense operator Z = I - K diag(chi), natural order
    v = w.voxels
    rng = np.random.default_rng(5)
    rows_tree = np.sort(rng.choice(arrs.n, 24, replace=False))
    unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)   # tree -> natural unknown
    x_nat = np.empty_like(x)
    x_nat[unk] = x
    Zr = vie.z_rows(v.centres, v.dv, v.eps_r, 2 * math.pi, unk[rows_tree])
    exact = Zr @ x_nat
    err = np.abs(y[rows_tree] - exact)
    assert err.max() <= 10 * w.eps * np.abs(exact).max()
    assert np.linalg.norm(y[rows_tree] - exact) <= 10 * w.eps * np.linalg.norm(exact)


def test_full_size_gmres_residual(full):
    w, arrs, perm, A, hZ = full
    b = synth.default_rhs(w)[(3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)]
    x, info = A.gmres(torch.from_numpy(b).cuda(), tol=w.tol, restart=400, maxit=3000, refine=True)
    assert info[0]["status"] == 0, info
    x = x.cpu().numpy()
    res = np.linalg.norm(b - h2mv.h2_matvec(hZ, x)) / np.linalg.norm(b)
    assert res <= 1.05 * w.tol


def test_full_size_split_product_sampled_columns(full):
    """Split-bf16 tensor-core product of 8 right-hand sides at full size:
    every column against the oracle's FP64 product, within eps."""
    w, arrs, perm, A, hZ = full
    R = 8
    X = synth.random_complex(arrs.n, 23, cols=R).astype(np.complex64)
    Xt = torch.from_numpy(np.asfortranarray(X)).cuda().t().contiguous().t()
    Y = A.matvec(Xt, prec="splitbf16").cpu().numpy()
    for j in range(R):
        y_or = h2mv.h2_matvec(hZ, X[:, j].astype(np.complex128))
        assert np.linalg.norm(Y[:, j] - y_or) <= w.eps * np.linalg.norm(y_or)


def test_full_size_accumulated_products_agree(full):
    """Double-float and FP64 accumulation of the stored data agree to 1e-12."""
    w, arrs, perm, A, hZ = full
    x = torch.from_numpy(synth.random_complex(arrs.n, 24)).cuda()
    ya = A.matvec(x, prec="fp64acc")
    yd = A.matvec(x, prec="dfacc")
    assert float(torch.linalg.norm(ya - yd) / torch.linalg.norm(ya)) <= 1e-12


@pytest.mark.parametrize("arnoldi", ["fp32", "df"])
def test_full_size_batched_gmres(full, arnoldi):
    """The batched solve bench.py times (split-bf16 products, c64-basis
    Arnoldi with eta = 0.1, double-float restart residuals, m = 400; and the
    double-float-basis variant) on 4 plane waves: the oracle's FP64 residual
    of every solution <= 1.05 tol."""
    w, arrs, perm, A, hZ = full
    R = 4
    B = synth.random_plane_waves(w.voxels, R, seed=5)[(3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)]
    Bt = torch.from_numpy(np.asfortranarray(B)).cuda().t().contiguous().t()
    X, info = A.gmres_batched(Bt, tol=w.tol, restart=400, maxit=3000, refine=True, prec="splitbf16", arnoldi=arnoldi,
                              reorth_eta=0.1)
    X = X.cpu().numpy()
    for j in range(R):
        assert info[j]["status"] == 0, info[j]
        res = np.linalg.norm(B[:, j] - h2mv.h2_matvec(hZ, X[:, j])) / np.linalg.norm(B[:, j])
        assert res <= 1.05 * w.tol


def test_full_size_symmetric_couplings(full):
    """Couplings stored once per admissible pair at full size (ranks up to 79,
    so tasks with a second row pair per lane run too): exactly half the
    coupling entries stored, exact symmetry of the constructed couplings, and
    the product within 1e-6 of the full-storage product and within 1e-5 of the
    oracle's FP64 product on the same data."""
    from paper_1703_01175_gb300 import h2
    w, arrs, perm, A, hZ = full
    B = h2.H2Matrix(arrs, sym_couple=True)
    try:
        st = B.sym_stats()
        assert 2 * st["stored_elems"] == A.stats()["coupling_elems"]
        assert st["max_asym"] == 0.0
        x = synth.random_complex(arrs.n, 25)
        xt = torch.from_numpy(x.astype(np.complex64)).cuda()
        ys = B.matvec(xt).cpu().numpy()
        yf = A.matvec(xt).cpu().numpy()
        assert np.linalg.norm(ys - yf) <= 1e-6 * np.linalg.norm(yf)
        yo = h2mv.h2_matvec(hZ, x.astype(np.complex64).astype(np.complex128))
        assert np.linalg.norm(ys - yo) <= 1e-5 * np.linalg.norm(yo)
        # and the near field once per leaf pair (chi of the workload, nowhere zero)
        B.sym_near(np.repeat(np.asarray(w.voxels.eps_r, dtype=np.complex128)[perm] - 1.0, 3))
        assert B.sym_near_stats()["max_asym"] <= 1e-5
        yn = B.matvec(xt).cpu().numpy()
        assert np.linalg.norm(yn - yf) <= 1e-6 * np.linalg.norm(yf)
        assert np.linalg.norm(yn - yo) <= 1e-5 * np.linalg.norm(yo)
    finally:
        B.close()
