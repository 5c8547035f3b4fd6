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


def test_bicgstab_matches_dense_solve_cube8():
    w = synth.workload("cube8")
    v = w.voxels
    Z = vie.assemble_Z(v.centres, v.dv, v.eps_r, K)
    b = synth.default_rhs(w)
    x, it, hist = krylov.bicgstab(lambda q: Z @ q, b, 1e-10, maxit=500)
    xd = np.linalg.solve(Z, b)
    assert hist[-1] <= 1e-10
    assert np.linalg.norm(Z @ x - b) <= 2e-10 * np.linalg.norm(b)   # recursive and true residual agree
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_bicgstab_exact_on_two_eigenvalues():
    """A = Q diag(l1, l2) Q^-1 has a minimal polynomial of degree 2: the
    BiCG part terminates after two steps, so BiCGStab converges in at most 2
    iterations (in exact arithmetic; here to rounding)."""
    rng = np.random.default_rng(3)
    n = 12
    Q = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    d = np.where(np.arange(n) < 5, 2.0 + 1.0j, 0.5 - 0.25j)
    A = Q @ np.diag(d) @ np.linalg.inv(Q)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist = krylov.bicgstab(lambda q: A @ q, b, 1e-9, maxit=50)
    assert it <= 2
    assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)


def test_bicgstab_identity_and_zero_rhs():
    b = synth.random_complex(10, 4)
    x, it, hist = krylov.bicgstab(lambda q: 3.0 * q, b, 1e-12)
    assert it == 1 and np.allclose(x, b / 3.0)
    x, it, hist = krylov.bicgstab(lambda q: q, np.zeros(5, complex), 1e-12)
    assert it == 0 and not np.any(x)
