"""Full-size geometries of the paper's scaling experiments (Sec. V), built on
the GPU by construct_gpu and loaded through h2_load_device -- the launch
configuration bench.py's --geometry legs time:

  slab256   : 256 x 256 x 2 slab, 8 x 8 x 0.06 wavelengths, eps_r 3,
              N = 393,216; 128 right-hand sides (a 2-D geometry, Sec. V.C);
  cube64v   : 64^3 cube, side 4, eps_r 4 with 10 % void voxels,
              N = 786,432; 256 right-hand sides (3-D);
  array4096 : 4096 cubes of 4^3 voxels on a line, pitch 0.5, eps_r 2.54,
              N = 786,432; 256 right-hand sides (a 1-D geometry, Sec. V.B, V.D);
  cube48    : 48^3 cube, side 3, smooth eps_r in [2, 8] from Gaussian bumps,
              N = 331,776; 32 right-hand sides (the learned preconditioner's
              geometry).

For each, on sampled rows (the oracle's FP64 product of the full data would not
fit in host memory at this size, so oracle.h2rows evaluates rows of Eqs. 8-9
from the same flat arrays):
- FP32 product vs the oracle's FP64 product on the same data: 1e-5;
- FP32 product vs the oracle's dense VIE rows (vie.z_rows): 10 eps (25 eps
  on the 64^3 cube, whose rows cross the most admissible blocks);
- split-bf16 tensor-core product of all R right-hand sides: every column
  within eps of the oracle on the sampled rows;
- the 1-D array keeps a bounded rank as its clusters grow (Sec. II.B: constant
  rank for 1-D geometries), while the 3-D cube's top ranks grow.
"""
import math

import numpy as np
import pytest

import synth
from oracle import h2rows, vie

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GEOMETRIES = ["slab256", "cube64v", "array4096", "cube48"]
NRHS = {"slab256": 128, "cube64v": 256, "array4096": 256, "cube48": 32}
# representation error against the dense VIE, in units of eps: the per-cluster
# truncation at eps (Eqs. 11, 15) accumulates over the admissible blocks of a
# row -- up to 94 per cluster over 9 levels on the 64^3 cube, where 11-18 eps
# was measured for two Stage I tolerances (a tighter one did not lower it);
# 10 eps elsewhere
REPR_BOUND = {"cube64v": 25}


@pytest.fixture(scope="module", params=GEOMETRIES)
def geom(request):
    from paper_1703_01175_gb300 import build, construct_gpu, h2
    build.build_all()
    w = synth.workload(request.param)
    v = w.voxels
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps,
                                        verbose=True)
    a = dh.to_host()
    A = h2.H2Matrix.from_device(dh)
    perm = dh.perm
    info = dh.info
    dh.free()
    del dh
    torch.cuda.empty_cache()
    yield request.param, w, a, perm, A, info
    A.close()
    torch.cuda.empty_cache()


def _rows(n, count, seed):
    return np.sort(np.random.default_rng(seed).choice(n, count, replace=False))


def test_fp32_product_sampled_rows(geom):
    name, w, a, perm, A, info = geom
    x = synth.random_complex(a.n, 41)
    y = A.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    rows = _rows(a.n, 48, 1)
    y_or = h2rows.matvec_rows(a, x, rows)
    assert np.linalg.norm(y[rows] - y_or) <= 1e-5 * np.linalg.norm(y_or)
    # the dense operator Z = I - K diag(chi), natural order
    v = w.voxels
    unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    x_nat = np.empty_like(x)
    x_nat[unk] = x
    exact = vie.z_rows(v.centres, v.dv, v.eps_r, 2 * math.pi, unk[rows]) @ x_nat
    bound = REPR_BOUND.get(name, 10) * w.eps
    assert np.linalg.norm(y[rows] - exact) <= bound * np.linalg.norm(exact)
    assert np.abs(y[rows] - exact).max() <= bound * np.abs(exact).max()


def test_split_bf16_all_columns(geom):
    name, w, a, perm, A, info = geom
    R = NRHS[name]
    X = synth.random_complex(a.n, 43, cols=R).astype(np.complex64)
    Xt = torch.from_numpy(np.asfortranarray(X)).cuda().t().contiguous().t()
    Y = A.matvec(Xt, prec="splitbf16")
    assert A.device_status() == 0
    rows = _rows(a.n, 32, 2)
    Ys = Y.cpu().numpy()[rows]
    del Y, Xt
    ref = h2rows.matvec_rows(a, X.astype(np.complex128), rows)
    err = np.linalg.norm(Ys - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= w.eps, (name, float(err.max()))


def test_rank_growth(geom):
    """Largest rank per level from the leaves up: bounded on the 1-D array
    (within 1.5 x its leaf-level maximum at every level), growing on the 3-D
    cube (its largest rank at least 1.5 x its leaf-level maximum; measured
    69 at the leaves, 136 four levels up)."""
    name, w, a, perm, A, info = geom
    lp = a.level_ptr
    per_level = [int(a.rank[lp[l]:lp[l + 1]].max()) for l in range(len(lp) - 1)]
    nz = [r for r in per_level if r > 0]
    leaf_max = per_level[-1] if per_level[-1] > 0 else nz[-1]
    if name == "array4096":
        assert max(nz) <= 1.5 * leaf_max, per_level
    if name == "cube64v":
        assert max(nz) >= 1.5 * leaf_max, per_level
