"""GPU BiCGStab (the paper's solver, Sec. V) against the oracle's.

Bar: the oracle's FP64 H^2 residual of the GPU solution is within the
tolerance (refined runs exactly, recursive-residual runs within 1.05 tol plus
the FP32 product's rounding), the solution agrees with the oracle's BiCGStab
solution to the accuracy the residual allows, and the outcome codes of
non-convergence and a zero right-hand side are right.
"""
import numpy as np
import pytest

import cases
import synth
from oracle import krylov

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mats():
    from paper_1703_01175_gb300 import build, h2
    build.build_all()
    out = {name: h2.H2Matrix(cases.get(name).arrays()) for name in ("cube8", "cube12", "ragged")}
    yield out
    for m in out.values():
        m.close()


def _oracle_res(c, x, b):
    return np.linalg.norm(b - c.oracle_matvec(x)) / np.linalg.norm(b)


@pytest.mark.parametrize("refine,arnoldi", [(True, "fp64"), (True, "df"), (False, "fp64")])
def test_bicgstab_cube8_matches_oracle(mats, refine, arnoldi):
    c = cases.get("cube8")
    w = synth.workload("cube8")
    b = synth.default_rhs(w)[c.tree.unknown_perm()]
    tol = 1e-6 if refine else 1e-5
    xg, info = mats["cube8"].bicgstab(torch.from_numpy(b).cuda(), tol=tol, maxit=500, refine=refine, arnoldi=arnoldi)
    xg = xg.cpu().numpy()
    assert info[0]["status"] == 0, info
    assert _oracle_res(c, xg, b) <= tol * (1.0 if refine else 1.05) + 2e-7
    xo, it, hist = krylov.bicgstab(c.oracle_matvec, b, tol, maxit=500)
    assert np.linalg.norm(xg - xo) <= 50 * tol * np.linalg.norm(xo)
    assert abs(info[0]["iterations"] - it) <= max(3, it // 5)


def test_bicgstab_multi_rhs_and_ragged(mats):
    for name in ("cube12", "ragged"):
        c = cases.get(name)
        B = np.asfortranarray(synth.random_complex(c.n, 41, cols=2))
        Bt = torch.from_numpy(B).cuda().t().contiguous().t()
        X, info = mats[name].bicgstab(Bt, tol=1e-6, maxit=2000, refine=True)
        X = X.cpu().numpy()
        for j in range(2):
            assert info[j]["status"] == 0, info[j]
            assert _oracle_res(c, X[:, j], B[:, j]) <= 1e-6


def test_bicgstab_not_converged_and_zero_rhs(mats):
    c = cases.get("ragged")
    b = synth.random_complex(c.n, 43)
    x, info = mats["ragged"].bicgstab(torch.from_numpy(b).cuda(), tol=1e-14, maxit=3)
    assert info[0]["status"] == 4 and info[0]["iterations"] == 3   # H2_ERR_NOT_CONVERGED
    assert info[0]["rel_res"] < 1.0
    z = torch.zeros(c.n, dtype=torch.complex128, device="cuda")
    x, info = mats["ragged"].bicgstab(z, tol=1e-6)
    assert info[0]["status"] == 0 and torch.count_nonzero(x).item() == 0
