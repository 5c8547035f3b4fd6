"""Pulse-basis, point-matched E-field volume integral equation (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's Eq. 1 is the D-field VIE discretised with SWG functions (Eqs. 2-3);
its H^2 algorithms are stated to be kernel independent (Sec. I, Sec. VI), so the
same construction is applied here to the simpler pulse-basis E-field form on
box voxels:

    E^i(r_m) = E_m - sum_n K_mn chi_n E_n,     chi_n = eps_r,n - 1,

i.e. the system matrix is Z = I - K diag(chi), with 3x3 blocks

    K_mn = dV (k^2 I + grad grad) g(r_m - r_n)          (m != n)
         = dV k^2 g(R) [ (1 - j/(kR) - 1/(kR)^2) I + (-1 + 3j/(kR) + 3/(kR)^2) R^R^ ]
    K_mm = [ (2/3) ((1 + j k a) e^{-j k a} - 1) - 1/3 ] I

with g(R) = e^{-j k R} / (4 pi R) (Sec. II.A) and a = (3 dV / 4 pi)^{1/3} the
radius of the sphere of the voxel's volume. The self term is the principal
volume integral of (k^2 + grad grad) g over that sphere, which by symmetry is
(2/3) k^2 int g dv, plus the -I/3 depolarisation dyad of a spherical exclusion
volume; k^2 int_sphere g dv = (1 + j k a) e^{-j k a} - 1 in closed form.

Unknowns are ordered voxel-major, component-minor: index 3 n + c.

Pins (tests/test_oracle_vie.py): the dyad against a finite-difference Hessian
of g, its far- and near-zone limits, the sphere integral against quadrature,
the radiation-reaction term and Clausius-Mossotti limit of the self term,
complex symmetry of K, and that a void voxel scatters nothing.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def green_scalar(R: np.ndarray, k: float) -> np.ndarray:
    """g(R) = exp(-j k R) / (4 pi R), Sec. II.A below Eq. 1."""
    return np.exp(-1j * k * R) / (4.0 * math.pi * R)


def green_dyad(Rvec: np.ndarray, k: float) -> np.ndarray:
    """k^{-2} (k^2 I + grad grad) g at separation vectors Rvec (..., 3).

    Returns (..., 3, 3) complex128: g [a I + b R^R^] with
    a = 1 - j/(kR) - 1/(kR)^2 and b = -1 + 3j/(kR) + 3/(kR)^2.
    """
    Rvec = np.asarray(Rvec, dtype=np.float64)
    R = np.sqrt(np.sum(Rvec * Rvec, axis=-1))
    kR = k * R
    g = green_scalar(R, k)
    a = 1.0 - 1j / kR - 1.0 / kR**2
    b = -1.0 + 3j / kR + 3.0 / kR**2
    Rh = Rvec / R[..., None]
    out = (b * g)[..., None, None] * (Rh[..., :, None] * Rh[..., None, :])
    idx = np.arange(3)
    out[..., idx, idx] += (a * g)[..., None]
    return out


def sphere_integral(a: float, k: float) -> complex:
    """k^2 * integral of g over a ball of radius a centred on the source point:
    k^2 int_0^a r e^{-j k r} dr = (1 + j k a) e^{-j k a} - 1."""
    ka = k * a
    return (1.0 + 1j * ka) * np.exp(-1j * ka) - 1.0


def equivalent_radius(dv: float) -> float:
    return (3.0 * dv / (4.0 * math.pi)) ** (1.0 / 3.0)


def self_term(dv: float, k: float) -> complex:
    """Scalar s with K_mm = s I: (2/3) k^2 int_sphere g - 1/3."""
    return (2.0 / 3.0) * sphere_integral(equivalent_radius(dv), k) - 1.0 / 3.0


def k_block(rm: np.ndarray, rn: np.ndarray, dv: float, k: float) -> np.ndarray:
    """The 3x3 block K_mn between voxel centres rm and rn."""
    if np.array_equal(rm, rn):
        return self_term(dv, k) * np.eye(3, dtype=np.complex128)
    return dv * k * k * green_dyad(np.asarray(rm) - np.asarray(rn), k)


def assemble_K(centres: np.ndarray, dv: float, k: float) -> np.ndarray:
    """Dense K (3 nv x 3 nv) in natural voxel order, entry by 3x3 block."""
    nv = centres.shape[0]
    K = np.zeros((nv, 3, nv, 3), dtype=np.complex128)
    for m in range(nv):
        Rvec = centres[m][None, :] - centres
        Rvec[m] = 1.0  # placeholder, overwritten below
        blk = dv * k * k * green_dyad(Rvec, k)  # (nv, 3, 3)
        blk[m] = self_term(dv, k) * np.eye(3)
        K[m] = blk.transpose(1, 0, 2)
    return K.reshape(3 * nv, 3 * nv)


def chi_unknowns(eps_r: np.ndarray) -> np.ndarray:
    """chi per unknown: eps_r - 1 repeated for the three components."""
    return np.repeat(np.asarray(eps_r, dtype=np.complex128) - 1.0, 3)


def assemble_Z(centres: np.ndarray, dv: float, eps_r: np.ndarray, k: float) -> np.ndarray:
    """System matrix Z = I - K diag(chi) (natural order)."""
    K = assemble_K(centres, dv, k)
    chi = chi_unknowns(eps_r)
    return np.eye(K.shape[0], dtype=np.complex128) - K * chi[None, :]


def k_rows(centres: np.ndarray, dv: float, k: float, rows) -> np.ndarray:
    """Selected rows of K (natural order): rows[i] = 3 m + c.
    Returns (len(rows), 3 nv), one row at a time."""
    nv = centres.shape[0]
    out = np.empty((len(rows), 3 * nv), dtype=np.complex128)
    for i, r in enumerate(rows):
        m, c = divmod(int(r), 3)
        Rvec = centres[m][None, :] - centres
        Rvec[m] = 1.0
        blk = dv * k * k * green_dyad(Rvec, k)
        blk[m] = self_term(dv, k) * np.eye(3)
        out[i] = blk[:, c, :].reshape(-1)
    return out


def z_rows(centres, dv, eps_r, k, rows) -> np.ndarray:
    """Selected rows of Z = I - K diag(chi) (natural order)."""
    R = -k_rows(centres, dv, k, rows) * chi_unknowns(eps_r)[None, :]
    for i, r in enumerate(rows):
        R[i, int(r)] += 1.0
    return R
