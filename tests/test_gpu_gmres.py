"""GPU restarted GMRES against the oracle.

Bar: the oracle's FP64 H^2 residual ||b - A x_gpu|| / ||b|| is at most the
requested tolerance (times 1.05 for the plain FP32 restart residual), the GPU
solution agrees with the oracle's GMRES solution to the accuracy the residual
allows, and the outcome codes for non-convergence, zero right-hand sides and
initial guesses are right.
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
    out = {}
    for name in ("cube8", "cube12", "ragged", "odd"):
        out[name] = h2.H2Matrix(cases.get(name).arrays())
    yield out
    for m in out.values():
        m.close()


def _oracle_res(c, x, b):
    return np.linalg.norm(b - c.oracle_matvec(x)) / np.linalg.norm(b)


@pytest.mark.parametrize("refine", [True, False])
def test_gmres_cube8_matches_oracle(mats, refine):
    c = cases.get("cube8")
    w = synth.workload("cube8")
    b = synth.default_rhs(w)[c.tree.unknown_perm()]
    tol = 1e-6 if refine else 1e-5
    xg, info = mats["cube8"].gmres(torch.from_numpy(b).cuda(), tol=tol, restart=50, refine=refine)
    xg = xg.cpu().numpy()
    assert info[0]["status"] == 0, info
    res = _oracle_res(c, xg, b)
    assert res <= tol * (1.0 if refine else 1.05) + 2e-7
    xo, it, hist = krylov.gmres(c.oracle_matvec, b, tol, restart=50)
    assert np.linalg.norm(xg - xo) <= 50 * tol * np.linalg.norm(xo)
    assert abs(info[0]["iterations"] - it) <= 3


def test_gmres_restart_and_multi_rhs(mats):
    c = cases.get("cube12")
    B = np.asfortranarray(synth.random_complex(c.n, 7, cols=2))
    Bt = torch.from_numpy(B).cuda().t().contiguous().t()
    X, info = mats["cube12"].gmres(Bt, tol=1e-4, restart=8, maxit=2000, refine=True)
    X = X.cpu().numpy()
    for j in range(2):
        assert info[j]["status"] == 0
        assert info[j]["restarts"] >= 2
        assert _oracle_res(c, X[:, j], B[:, j]) <= 1e-4


def test_gmres_not_converged_and_zero_rhs(mats):
    c = cases.get("ragged")
    b = synth.random_complex(c.n, 3)
    x, info = mats["ragged"].gmres(torch.from_numpy(b).cuda(), tol=1e-12, restart=4, maxit=6)
    assert info[0]["status"] == 4 and info[0]["iterations"] == 6  # H2_ERR_NOT_CONVERGED
    assert info[0]["rel_res"] < 1.0
    z = torch.zeros(c.n, dtype=torch.complex128, device="cuda")
    x, info = mats["ragged"].gmres(z, tol=1e-6)
    assert info[0]["status"] == 0 and torch.count_nonzero(x).item() == 0


def test_gmres_initial_guess(mats):
    c = cases.get("ragged")
    b = synth.random_complex(c.n, 4)
    bt = torch.from_numpy(b).cuda()
    x, info = mats["ragged"].gmres(bt, tol=1e-8, restart=30, refine=True)
    assert info[0]["status"] == 0
    x2, info2 = mats["ragged"].gmres(bt, x=x.clone(), tol=1e-6, restart=30, refine=True, x0_given=True)
    assert info2[0]["iterations"] == 0 and info2[0]["status"] == 0
    assert torch.allclose(x, x2)


@pytest.mark.parametrize("refine", [True, False])
def test_gmres_double_float_arnoldi(mats, refine):
    """Double-float Gram-Schmidt on the FP32 pipes: same convergence as the
    FP64 one and an oracle residual within the tolerance."""
    c = cases.get("cube8")
    w = synth.workload("cube8")
    b = synth.default_rhs(w)[c.tree.unknown_perm()]
    tol = 1e-6 if refine else 1e-5
    bt = torch.from_numpy(b).cuda()
    x1, i1 = mats["cube8"].gmres(bt, tol=tol, restart=50, refine=refine)
    x2, i2 = mats["cube8"].gmres(bt, tol=tol, restart=50, refine=refine, arnoldi="df")
    assert i2[0]["status"] == 0, i2
    assert abs(i1[0]["iterations"] - i2[0]["iterations"]) <= 1
    x2 = x2.cpu().numpy()
    assert _oracle_res(c, x2, b) <= tol * (1.0 if refine else 1.05) + 2e-7
    xo, it, hist = krylov.gmres(c.oracle_matvec, b, tol, restart=50)
    assert np.linalg.norm(x2 - xo) <= 50 * tol * np.linalg.norm(xo)


@pytest.mark.parametrize("name,tol", [("ragged", 1e-4), ("ragged", 1e-6), ("odd", 1e-5)])
def test_gmres_fp32_basis_arnoldi(mats, name, tol):
    """c64 basis with FP32 products and compensated sums: converges to the
    tolerance against the oracle's FP64 residual, in about the iterations of
    the FP64 Arnoldi (ragged: 630 unknowns, row segments with tails; odd: 525
    unknowns, the update pass's two-strided-rows path)."""
    c = cases.get(name)
    b = synth.random_complex(c.n, 19)
    bt = torch.from_numpy(b).cuda()
    x1, i1 = mats[name].gmres(bt, tol=tol, restart=40, maxit=2000, refine=True)
    x2, i2 = mats[name].gmres(bt, tol=tol, restart=40, maxit=2000, refine=True, arnoldi="fp32", reorth_eta=0.1)
    assert i2[0]["status"] == 0, i2
    assert _oracle_res(c, x2.cpu().numpy(), b) <= tol * 1.05
    assert i2[0]["iterations"] <= i1[0]["iterations"] * 1.1 + 3, (i1, i2)


def test_batched_gmres_fp32_basis_odd_n(mats):
    """Batched solve with the c64 basis on an odd number of unknowns: every
    column's oracle FP64 residual within the tolerance."""
    c = cases.get("odd")
    R = 3
    B = np.asfortranarray(synth.random_complex(c.n, 29, cols=R))
    Bt = torch.from_numpy(B).cuda().t().contiguous().t()
    X, info = mats["odd"].gmres_batched(Bt, tol=1e-4, restart=30, maxit=2000, refine=True, prec="splitbf16",
                                        arnoldi="fp32", reorth_eta=0.1)
    X = X.cpu().numpy()
    for j in range(R):
        assert info[j]["status"] == 0, info[j]
        assert _oracle_res(c, X[:, j], B[:, j]) <= 1.05e-4


@pytest.mark.parametrize("arnoldi", ["fp64", "df", "fp32"])
@pytest.mark.parametrize("prec", ["splitbf16", "fp32"])
def test_batched_gmres_matches_oracle(mats, prec, arnoldi):
    """Batched GMRES (one multi-RHS product per Arnoldi step): every column's
    oracle FP64 residual within the tolerance."""
    c = cases.get("cube12")
    R = 5
    B = np.asfortranarray(synth.random_complex(c.n, 17, cols=R))
    Bt = torch.from_numpy(B).cuda().t().contiguous().t()
    X, info = mats["cube12"].gmres_batched(Bt, tol=1e-4, restart=30, maxit=2000, refine=True, prec=prec,
                                           arnoldi=arnoldi)
    X = X.cpu().numpy()
    for j in range(R):
        assert info[j]["status"] == 0, info[j]
        assert _oracle_res(c, X[:, j], B[:, j]) <= 1.05e-4
    # same Krylov method as the single-RHS solver: similar iteration counts
    x1, i1 = mats["cube12"].gmres(torch.from_numpy(np.ascontiguousarray(B[:, 0])).cuda(), tol=1e-4, restart=30,
                                  refine=True)
    assert abs(info[0]["iterations"] - i1[0]["iterations"]) <= 10


def test_reorthogonalisation_threshold(mats):
    """eta = 1 reprojects at every step (CGS2), eta = 0.1 only under heavy
    cancellation; both converge like the default, and eta outside [0, 1] is
    rejected."""
    c = cases.get("cube12")
    b = synth.random_complex(c.n, 31)
    bt = torch.from_numpy(b).cuda()
    its = {}
    for eta in (0.0, 1.0, 0.1):
        x, info = mats["cube12"].gmres(bt, tol=1e-6, restart=30, maxit=2000, refine=True, reorth_eta=eta)
        assert info[0]["status"] == 0
        assert _oracle_res(c, x.cpu().numpy(), b) <= 1e-6 + 2e-7
        its[eta] = info[0]
    assert its[1.0]["reorth_steps"] == its[1.0]["iterations"]
    assert its[0.1]["reorth_steps"] <= its[0.0]["reorth_steps"]
    assert abs(its[0.1]["iterations"] - its[0.0]["iterations"]) <= 2
    from paper_1703_01175_gb300 import h2 as h2py
    with pytest.raises(h2py.H2Error):
        mats["cube12"].gmres(bt, tol=1e-6, restart=30, reorth_eta=1.5)
