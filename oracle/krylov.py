"""Restarted GMRES(m) with modified Gram-Schmidt (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper solves with BiCGStab (Sec. V); the solver around the H^2 product
here is restarted GMRES(m) (Saad & Schultz 1986): Arnoldi with modified
Gram-Schmidt, Givens rotations on the Hessenberg matrix, x0 = 0, and the
relative residual ||b - A x|| / ||b|| recomputed with the operator itself at
every restart. With a right preconditioner M the flexible variant (FGMRES,
Saad 1993) stores the preconditioned directions z_j = M(v_j) and updates
x += Z y.

Pin (tests/test_oracle_krylov.py): the solution agrees with LAPACK's dense
solve, and the Arnoldi relation A V_m = V_{m+1} H_m holds. The paper's own
solver, BiCGStab, is here too (`bicgstab`), pinned the same way and by its
exact termination on operators with few distinct eigenvalues.
"""
from __future__ import annotations

import numpy as np


def _givens(a: complex, b: complex):
    """c, s with [c s; -conj(s) c] [a; b] = [r; 0], c real."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    na = abs(a)
    nr = np.hypot(na, abs(b))
    c = na / nr
    s = (a / na) * np.conj(b) / nr
    return c, s


def gmres(apply_A, b: np.ndarray, tol: float, restart: int = 50, maxit: int = 1000,
          precond=None, x0=None):
    """Solve A x = b. Returns (x, iterations, history of relative residuals).

    apply_A(v) -> A v; precond(v) -> M v (right preconditioner, FGMRES) or None.
    Convergence: the recomputed true residual <= tol * ||b||.
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return np.zeros_like(b), 0, [0.0]
    it = 0
    r = b - apply_A(x)
    beta = np.linalg.norm(r)
    hist.append(beta / bnorm)
    while beta / bnorm > tol and it < maxit:
        m = restart
        V = np.zeros((n, m + 1), dtype=np.complex128)
        Zs = np.zeros((n, m), dtype=np.complex128) if precond is not None else None
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        j_done = 0
        for j in range(m):
            zj = precond(V[:, j]) if precond is not None else V[:, j]
            if Zs is not None:
                Zs[:, j] = zj
            w = apply_A(zj)
            for i in range(j + 1):            # modified Gram-Schmidt
                H[i, j] = np.vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) / bnorm <= tol or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        basis = Zs if Zs is not None else V
        x = x + basis[:, :j_done] @ y
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
    return x, it, hist


def arnoldi(apply_A, v0: np.ndarray, m: int):
    """m steps of Arnoldi with modified Gram-Schmidt: returns V (n x m+1) and
    the Hessenberg H (m+1 x m) with A V[:, :m] = V H."""
    n = v0.shape[0]
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    V[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(m):
        w = apply_A(V[:, j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


def bicgstab(apply_A, b: np.ndarray, tol: float, maxit: int = 1000, x0=None):
    """BiCGStab (van der Vorst 1992), the paper's solver (Sec. V), for complex
    systems: the shadow residual is r0, inner products (u, v) = u^H v.

    Each iteration takes two products: v = A p, then t = A s. The iterate
    stops when the recursive residual r falls below tol * ||b|| (the returned
    history holds ||r|| / ||b|| per iteration); breakdown (rho = 0,
    (r0, v) = 0 or (t, t) = 0) ends the solve. Returns (x, iterations, history).
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = b - apply_A(x)
    rhat = r.copy()
    hist = [np.linalg.norm(r) / bnorm]
    rho_old = alpha = omega = 1.0 + 0.0j
    v = np.zeros(n, dtype=np.complex128)
    p = np.zeros(n, dtype=np.complex128)
    it = 0
    while hist[-1] > tol and it < maxit:
        rho = np.vdot(rhat, r)
        if rho == 0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_A(p)
        d = np.vdot(rhat, v)
        if d == 0:
            break
        alpha = rho / d
        s = r - alpha * v
        t = apply_A(s)
        tt = np.vdot(t, t).real
        omega = np.vdot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        if omega == 0:
            break
    return x, it, hist
