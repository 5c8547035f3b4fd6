"""Train the learned preconditioner on the method's own GMRES solves.

    python -m paper_1703_01175_gb300.train_precond [--train cube16r] [--rhs 40]
        [--restart 10] [--epochs 30] [--out weights/vie_u26.npz]

1. Build the H^2 operator of the training geometry (host constructor).
2. Solve it for `rhs` random plane waves with restarted GMRES(restart) to a
   tight tolerance; every restart iterate x_k gives a pair
   (r_k, e_k) = (b - A x_k, x* - x_k); optionally add probe pairs
   (A e, e) for random e through the same product.
3. Fit the convolutional network N so that r + N(r) ~ e (unit-RMS scaling)
   with Adam, using the library's convolution, loss and optimiser kernels.
4. Save the FP32 weights and the training record (.npz).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", default="cube16r")
    ap.add_argument("--rhs", type=int, default=40)
    ap.add_argument("--probes", type=int, default=0, help="probe pairs r = A e with random e")
    ap.add_argument("--restart", type=int, default=10)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--out", default=os.path.join(HERE, "weights", "vie_u26.npz"))
    ap.add_argument("--loss", default="residual", choices=["residual", "error"],
                    help="residual: ||A M(r) - r|| (right approximate inverse); error: ||M(r) - e||")
    ap.add_argument("--gpu-construct", action="store_true",
                    help="build the operator on the GPU and collect the pairs from batched solves")
    ap.add_argument("--pairs-per-rhs", type=int, default=50)
    ap.add_argument("--eval-rhs", type=int, default=0, help="held-out plane waves (seed 6) for an evaluation solve")
    ap.add_argument("--eval-restart", type=int, default=50)
    a = ap.parse_args(argv)
    if a.gpu_construct:
        return main_gpu(a)

    import torch
    import synth
    from paper_1703_01175_gb300 import build, construct, h2 as h2py, precond as P

    build.build_all()
    w = synth.workload(a.train)
    v = w.voxels
    t0 = time.time()
    arrs, perm = construct.build_vie_h2_cached(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps)
    A = h2py.H2Matrix(arrs)
    unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    gm = P.GridMap(v.shape, perm, v.eps_r)
    rhs = synth.random_plane_waves(v, a.rhs, seed=a.seed)
    t1 = time.time()
    R, E = (None, None)
    if a.rhs > 0:
        R, E = P.collect_pairs(A, gm, [rhs[unk, j] for j in range(a.rhs)], restart=a.restart, tol=a.tol)
    n_solve = 0 if R is None else int(R.shape[0])
    if a.probes > 0:
        Rp, Ep = P.probe_pairs(A, a.probes, seed=a.seed + 100)
        R = Rp if R is None else torch.cat([R, Rp])
        E = Ep if E is None else torch.cat([E, Ep])
    torch.cuda.synchronize()
    t2 = time.time()
    net = P.ConvNet(v.shape, a.batch, seed=11)
    if a.loss == "residual":
        At = h2py.H2Matrix(P.transpose_arrays(arrs))
        hist = P.train_residual(net, gm, A, At, R, epochs=a.epochs, lr=a.lr, log=lambda s: print(s, flush=True))
        At.close()
    else:
        hist = P.train(net, gm, R, E, epochs=a.epochs, lr=a.lr, log=lambda s: print(s, flush=True))
    torch.cuda.synchronize()
    t3 = time.time()
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    params = net.parameters_numpy()
    record = {"loss": a.loss, "train_workload": a.train, "pairs": int(R.shape[0]), "solve_pairs": n_solve,
              "probe_pairs": int(R.shape[0]) - n_solve, "rhs": a.rhs, "restart": a.restart,
              "epochs": a.epochs, "batch": a.batch, "lr": a.lr, "loss_history": hist, "n_params": net.n_params(),
              "seconds": {"operator": t1 - t0, "pairs": t2 - t1, "training": t3 - t2}}
    np.savez(a.out, record=json.dumps(record), **params)
    print(json.dumps({k: record[k] for k in ("pairs", "n_params", "seconds")}), flush=True)
    print("final relative loss", hist[-1], flush=True)
    A.close()


def evaluate(A, v, unk, count, restart, tol, log=print, maxit=4000):
    """Batched solves of `count` held-out plane waves (seed 6) with and without
    the loaded preconditioner (split-bf16 products, c64-basis Arnoldi):
    iterations, time and true residuals of both."""
    import torch
    import synth
    B = synth.random_plane_waves(v, count, seed=6)[unk]
    Bt = torch.from_numpy(np.asfortranarray(B)).cuda().t().contiguous().t()
    out = {}
    for label, pc in (("plain", False), ("learned", True)):
        A.gmres_batched(Bt, tol=1e-12, restart=4, maxit=4, refine=True, prec="splitbf16", arnoldi="fp32",
                        reorth_eta=0.1, precond=pc, check=False)   # workspace
        torch.cuda.synchronize()
        t = time.time()
        X, info = A.gmres_batched(Bt, tol=tol, restart=restart, maxit=maxit, refine=True, prec="splitbf16",
                                  arnoldi="fp32", reorth_eta=0.1, precond=pc, check=False)
        torch.cuda.synchronize()
        el = time.time() - t
        out[label] = {"seconds": el, "converged": sum(1 for i in info if i["status"] == 0),
                      "mean_iterations": float(np.mean([i["iterations"] for i in info])),
                      "max_rel_res": max(i["rel_res"] for i in info),
                      "mean_precond_cycles": float(np.mean([i["precond_cycles"] for i in info]))}
        log(f"eval {label}: {out[label]}")
    return out


def main_gpu(a):
    """Config-4 recipe: operator built on the GPU, pairs from batched solves of
    `rhs` random plane waves (seed `seed`), training on the GPU, optional
    evaluation on held-out plane waves."""
    import torch
    import synth
    from paper_1703_01175_gb300 import build, construct_gpu, h2 as h2py, precond as P

    build.build_all()
    w = synth.workload(a.train)
    v = w.voxels
    t0 = time.time()
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps)
    perm = dh.perm
    arrs = dh.to_host() if a.loss == "residual" else None
    A = h2py.H2Matrix.from_device(dh)
    dh.free()
    torch.cuda.empty_cache()
    unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    gm = P.GridMap(v.shape, perm, v.eps_r)
    rhs = synth.random_plane_waves(v, a.rhs, seed=a.seed)[unk]
    Bt = torch.from_numpy(np.asfortranarray(rhs)).cuda().t().contiguous().t()
    t1 = time.time()
    # FP32 products with double-float restart residuals: the targets x* - x_k need
    # x* well below the split-bf16 products' 1e-5 accuracy
    R, E, srec = P.collect_pairs_batched(A, Bt, restart=a.restart, tol=a.tol, pairs_per_rhs=a.pairs_per_rhs,
                                         prec="fp32", arnoldi="df")
    del Bt
    torch.cuda.synchronize()
    t2 = time.time()
    print(f"pairs: {0 if R is None else R.shape[0]} from {srec}, {t2 - t1:.1f} s", flush=True)
    net = P.ConvNet(v.shape, a.batch, seed=11)
    if a.loss == "residual":
        At = h2py.H2Matrix(P.transpose_arrays(arrs))
        hist = P.train_residual(net, gm, A, At, R, epochs=a.epochs, lr=a.lr, log=lambda s: print(s, flush=True))
        At.close()
    else:
        hist = P.train(net, gm, R, E, epochs=a.epochs, lr=a.lr, log=lambda s: print(s, flush=True))
    torch.cuda.synchronize()
    t3 = time.time()
    params = net.parameters_numpy()
    record = {"loss": a.loss, "train_workload": a.train, "pairs": int(R.shape[0]), "solve_pairs": int(R.shape[0]),
              "probe_pairs": 0, "rhs": a.rhs, "restart": a.restart, "solve_record": srec,
              "epochs": a.epochs, "batch": a.batch, "lr": a.lr, "loss_history": hist, "n_params": net.n_params(),
              "seconds": {"operator": t1 - t0, "pairs": t2 - t1, "training": t3 - t2}}
    del R, E
    torch.cuda.empty_cache()
    if a.eval_rhs > 0:
        P.load_net(A, net, gm)
        record["evaluation"] = evaluate(A, v, unk, a.eval_rhs, a.eval_restart, w.tol,
                                        log=lambda s: print(s, flush=True))
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    np.savez(a.out, record=json.dumps(record), **params)
    print(json.dumps({k: record[k] for k in ("pairs", "n_params", "seconds")}), flush=True)
    print("final relative loss", hist[-1], flush=True)
    A.close()


if __name__ == "__main__":
    main()
