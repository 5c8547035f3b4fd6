"""What the trained network gains over the method without it.

The network in paper_1703_01175_gb300/weights/vie_cube48.npz was trained on
residual -> correction pairs from the method's own batched GMRES solves of the
48^3 smooth-permittivity cube (2,000 pairs). Here, on held-out plane waves
(seed 6) of the same cube, batched flexible GMRES(50) with the network as
right preconditioner is run beside batched GMRES(50) without it (split-bf16
products, c64-basis Arnoldi, double-float restart residuals), and:

- every solution of both arms meets the tolerance by the FP64-accumulated H^2
  residual (h2_matvec with H2_PREC_FP64ACC on the c128 solution), the judge
  of the learned path's error;
- the gain is measured and printed (iterations and time of both arms); with
  these weights it is a loss, and the test bounds that loss: a right-hand side
  whose preconditioned cycle does not cut its true residual by 5 % falls back
  to plain GMRES, so the learned arm takes at most a few restart cycles more
  than the plain one.
"""
import json
import os
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_1703_01175_gb300", "weights", "vie_cube48.npz")
NRHS, RESTART, MAXIT = 4, 50, 3000


@pytest.fixture(scope="module")
def cube48():
    from paper_1703_01175_gb300 import build, construct_gpu, h2, precond as P
    build.build_all()
    w = synth.workload("cube48")
    v = w.voxels
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps)
    perm = dh.perm
    A = h2.H2Matrix.from_device(dh)
    dh.free()
    del dh
    torch.cuda.empty_cache()
    z = np.load(WEIGHTS)
    layers = [tuple(int(q) for q in x) for x in z["layers"]]
    P.load_into(A, layers, [z[f"W{i}"] for i in range(len(layers))], [z[f"b{i}"] for i in range(len(layers))],
                P.GridMap(v.shape, perm, v.eps_r))
    unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    yield w, A, unk, json.loads(str(z["record"]))
    A.close()
    torch.cuda.empty_cache()


def _solve(A, B, precond):
    A.gmres_batched(B, tol=1e-12, restart=4, maxit=4, refine=True, prec="splitbf16", arnoldi="fp32",
                    reorth_eta=0.1, precond=precond, check=False)   # workspace
    torch.cuda.synchronize()
    t = time.time()
    X, info = A.gmres_batched(B, tol=1e-4, restart=RESTART, maxit=MAXIT, refine=True, prec="splitbf16",
                              arnoldi="fp32", reorth_eta=0.1, precond=precond, check=False)
    torch.cuda.synchronize()
    return X, info, time.time() - t


def _fp64_residual(A, B, X):
    """||b - A x|| / ||b|| per column with the FP64-accumulated product."""
    out = []
    for j in range(B.shape[1]):
        x = X[:, j].contiguous()
        r = B[:, j] - A.matvec(x, prec="fp64acc")
        out.append(float(torch.linalg.norm(r) / torch.linalg.norm(B[:, j])))
    return out


def test_learned_preconditioner_gain_is_measured_and_bounded(cube48):
    w, A, unk, rec = cube48
    assert rec.get("solve_pairs", 0) >= 2000 and rec.get("train_workload") == "cube48"
    Bm = synth.random_plane_waves(w.voxels, NRHS, seed=6)[unk]
    B = torch.from_numpy(np.asfortranarray(Bm)).cuda().t().contiguous().t()
    Xp, ip, tp = _solve(A, B, False)
    Xl, il, tl = _solve(A, B, True)
    assert A.device_status() == 0
    for label, X, info in (("plain", Xp, ip), ("learned", Xl, il)):
        assert all(i["status"] == 0 for i in info), (label, info)
        res = _fp64_residual(A, B, X)
        assert max(res) <= 1.05e-4, (label, res)
    it_p = np.array([i["iterations"] for i in ip])
    it_l = np.array([i["iterations"] for i in il])
    gain = {"plain_iterations": it_p.tolist(), "learned_iterations": it_l.tolist(),
            "plain_s": round(tp, 2), "learned_s": round(tl, 2),
            "iteration_ratio_plain_over_learned": float(it_p.mean() / it_l.mean()),
            "time_ratio_plain_over_learned": tp / tl,
            "preconditioned_cycles": [i["precond_cycles"] for i in il]}
    print("learned preconditioner on held-out plane waves:", json.dumps(gain))
    # the fallback bounds a loss: at most a few preconditioned cycles before plain GMRES takes over
    assert all(i["precond_cycles"] >= 1 for i in il)
    assert it_l.mean() <= it_p.mean() + 4 * RESTART, gain
    assert np.all(it_l <= it_p + 8 * RESTART), gain
