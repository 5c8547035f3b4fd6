"""Pins of the oracle's VIE operator against facts it does not itself define.

- splitmix64 reproduces the published test vector (tests/golden/splitmix64.txt);
- the dyad g [a I + b R^R^] equals (k^2 + grad grad) g / k^2 evaluated by
  finite differences of the scalar g (Sec. II.A, Eq. 1 kernel);
- far zone: the dyad tends to g (I - R^R^) (transverse radiation field);
- near zone: k^2 times the dyad tends to the static dipole kernel
  (3 R^R^ - I) / (4 pi R^3);
- the sphere integral closed form against adaptive quadrature;
- the self term's imaginary part is the radiation reaction -k^3 dV / (6 pi)
  of a small dipole to leading order, and its static limit -1/3 gives the
  Clausius-Mossotti internal field 3 E^i / (eps_r + 2);
- K is complex symmetric;
- a void voxel (chi = 0) scatters nothing: the other voxels' fields do not
  change when it is added, and its own field is the incident plus the
  scattered field of the others.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import vie

K = 2.0 * math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    got = synth.splitmix64_sequence(1234567, len(vals))
    assert [int(v) for v in got] == vals


def test_uniform_range_and_independence():
    u = synth.uniform(7, 20000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert not np.array_equal(synth.uniform(7, 10, 0), synth.uniform(7, 10, 1))


def _fd_dyad(Rvec, k, h=1e-4):
    """(k^2 I + grad grad) g / k^2 by central differences of the scalar g."""
    def g(r):
        R = np.linalg.norm(r)
        return np.exp(-1j * k * R) / (4 * math.pi * R)
    H = np.zeros((3, 3), dtype=np.complex128)
    E = np.eye(3) * h
    for i in range(3):
        for j in range(3):
            H[i, j] = (g(Rvec + E[i] + E[j]) - g(Rvec + E[i] - E[j])
                       - g(Rvec - E[i] + E[j]) + g(Rvec - E[i] - E[j])) / (4 * h * h)
    return g(Rvec) * np.eye(3) + H / (k * k)


@pytest.mark.parametrize("Rvec", [(0.3, -0.2, 0.5), (0.05, 0.07, -0.02), (1.7, 0.4, 0.9)])
def test_dyad_matches_finite_difference_hessian(Rvec):
    Rvec = np.array(Rvec)
    G = vie.green_dyad(Rvec, K)
    F = _fd_dyad(Rvec, K, h=1e-4 * np.linalg.norm(Rvec))
    assert np.abs(G - F).max() <= 1e-5 * np.abs(G).max()


def test_dyad_far_zone_is_transverse():
    d = np.array([1.0, 2.0, -2.0]) / 3.0
    R = 1e4 / K
    G = vie.green_dyad(R * d, K)
    g = np.exp(-1j * K * R) / (4 * math.pi * R)
    Gt = g * (np.eye(3) - np.outer(d, d))
    assert np.abs(G - Gt).max() <= 2e-4 * abs(g)


def test_dyad_near_zone_is_static_dipole():
    d = np.array([2.0, -1.0, 2.0]) / 3.0
    R = 1e-4 / K
    G = K * K * vie.green_dyad(R * d, K)
    S = (3 * np.outer(d, d) - np.eye(3)) / (4 * math.pi * R**3)
    assert np.abs(G - S).max() <= 1e-6 * np.abs(S).max()


@pytest.mark.parametrize("a", [0.01, 0.04, 0.2, 0.5])
def test_sphere_integral_quadrature(a):
    from scipy.integrate import quad
    re = quad(lambda r: K * K * r * math.cos(K * r), 0, a, epsabs=1e-14, epsrel=1e-13)[0]
    im = quad(lambda r: -K * K * r * math.sin(K * r), 0, a, epsabs=1e-14, epsrel=1e-13)[0]
    assert abs(vie.sphere_integral(a, K) - (re + 1j * im)) <= 1e-12 * max(1.0, abs(re + 1j * im))


def test_self_term_radiation_reaction():
    for dv in (1e-6, 1e-5, (1 / 16) ** 3):
        s = vie.self_term(dv, K)
        ka = K * vie.equivalent_radius(dv)
        rr = -K**3 * dv / (6 * math.pi)
        assert abs(s.imag - rr) <= 0.2 * ka**2 * abs(rr) + 1e-15


def test_clausius_mossotti_static_limit():
    dv = 1e-9  # k a ~ 4e-3
    for eps_r in (2.0, 4.0, 9.5):
        Z = vie.assemble_Z(np.zeros((1, 3)), dv, np.array([eps_r]), K)
        Ei = np.array([1.0, -0.5, 0.25j])
        E = np.linalg.solve(Z, Ei)
        cm = 3.0 * Ei / (eps_r + 2.0)
        assert np.abs(E - cm).max() <= 1e-4 * np.abs(cm).max()


def test_K_is_complex_symmetric():
    v = synth.uniform_grid((4, 3, 5), (1 / 16, 1 / 16, 1 / 16), 3.0)
    Km = vie.assemble_K(v.centres, v.dv, K)
    assert np.abs(Km - Km.T).max() <= 1e-15 * np.abs(Km).max()
    assert np.abs(Km - Km.conj().T).max() > 1e-3 * np.abs(Km).max()  # not Hermitian


def test_void_voxel_scatters_nothing():
    c = np.array([[0.0, 0.0, 0.0], [0.07, 0.02, 0.0], [0.0, 0.09, 0.05]])
    dv = (1 / 16) ** 3
    eps = np.array([4.0, 2.5, 1.0])  # the third voxel is void
    v = synth.VoxelSet("t", c, np.array([1 / 16] * 3), eps.astype(complex))
    Ei = synth.plane_wave(v, (0, 0, 1), (1, 0, 0))
    E3 = np.linalg.solve(vie.assemble_Z(c, dv, eps, K), Ei)
    E2 = np.linalg.solve(vie.assemble_Z(c[:2], dv, eps[:2], K), Ei[:6])
    assert np.abs(E3[:6] - E2).max() <= 1e-12 * np.abs(E2).max()
    scat = sum(vie.k_block(c[2], c[n], dv, K) @ ((eps[n] - 1) * E2[3 * n:3 * n + 3]) for n in range(2))
    assert np.abs(E3[6:] - (Ei[6:] + scat)).max() <= 1e-12 * np.abs(E3[6:]).max()


def test_rows_match_dense():
    v = synth.random_eps_grid((3, 4, 2), (1 / 16,) * 3, 2.0, 6.0, seed=9)
    Zd = vie.assemble_Z(v.centres, v.dv, v.eps_r, K)
    rows = [0, 5, 17, 3 * v.nv - 1]
    assert np.abs(vie.z_rows(v.centres, v.dv, v.eps_r, K, rows) - Zd[rows]).max() == 0.0
