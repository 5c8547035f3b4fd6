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
    a = ap.parse_args(argv)

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


if __name__ == "__main__":
    main()
