"""Pins of the oracle's GMRES against LAPACK's dense solve and the Arnoldi
relation."""
import math

import numpy as np

import synth
from oracle import h2build, h2mv, krylov, tree as otree, vie

K = 2.0 * math.pi


def test_gmres_matches_dense_solve_cube8():
    w = synth.workload("cube8")
    v = w.voxels
    Z = vie.assemble_Z(v.centres, v.dv, v.eps_r, K)
    b = synth.default_rhs(w)
    x, it, hist = krylov.gmres(lambda q: Z @ q, b, 1e-10, restart=50)
    xd = np.linalg.solve(Z, b)
    assert hist[-1] <= 1e-10
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_gmres_small_restart_and_tiny_brute_force():
    v = synth.random_eps_grid((2, 2, 2), (1 / 16,) * 3, 2.0, 6.0, seed=1)
    Z = vie.assemble_Z(v.centres, v.dv, v.eps_r, K)
    b = synth.random_complex(v.n, 8)
    x, it, hist = krylov.gmres(lambda q: Z @ q, b, 1e-12, restart=3, maxit=500)
    assert np.linalg.norm(Z @ x - b) <= 1e-11 * np.linalg.norm(b)


def test_fgmres_with_exact_inverse_takes_one_step():
    v = synth.random_eps_grid((3, 3, 2), (1 / 16,) * 3, 2.0, 6.0, seed=4)
    Z = vie.assemble_Z(v.centres, v.dv, v.eps_r, K)
    Zi = np.linalg.inv(Z)
    b = synth.random_complex(v.n, 2)
    x, it, hist = krylov.gmres(lambda q: Z @ q, b, 1e-10, restart=10, precond=lambda q: Zi @ q)
    assert it == 1
    assert np.linalg.norm(Z @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_arnoldi_relation():
    v = synth.uniform_grid((4, 4, 2), (1 / 16,) * 3, 4.0)
    Z = vie.assemble_Z(v.centres, v.dv, v.eps_r, K)
    V, H = krylov.arnoldi(lambda q: Z @ q, synth.random_complex(v.n, 6), 12)
    assert np.abs(Z @ V[:, :12] - V @ H).max() <= 1e-12 * np.abs(Z).max()
    assert np.abs(V.conj().T @ V - np.eye(13)).max() <= 1e-10


def test_h2_gmres_residual_cube8():
    w = synth.workload("cube8")
    v = w.voxels
    Kd = vie.assemble_K(v.centres, v.dv, K)
    tr = otree.build_tree(v.centres, w.n_min)
    pa = otree.partition(tr, w.eta)
    Kt = h2build.to_tree_order(Kd, tr)
    chi = vie.chi_unknowns(v.eps_r)[tr.unknown_perm()]
    hZ = h2build.system_h2(h2build.build_h2_K(Kt, tr, pa, w.eps), chi)
    Zt = np.eye(tr.n) - Kt * chi[None, :]
    b = synth.default_rhs(w)[tr.unknown_perm()]
    x, it, hist = krylov.gmres(lambda q: h2mv.h2_matvec(hZ, q), b, w.tol, restart=50)
    assert hist[-1] <= w.tol
    # the H^2 solution solves the dense system to about the representation error
    assert np.linalg.norm(Zt @ x - b) <= 1e-4 * np.linalg.norm(b)
