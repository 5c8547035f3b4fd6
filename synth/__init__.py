"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the H^2 method: it only produces the
inputs the method is applied to -- voxel geometries, relative permittivity
fields, incident plane waves and random vectors -- from a counter-based
generator (splitmix64), so that both sides of every comparison see bit-equal
inputs.

Units: the free-space wavelength is 1, so the wavenumber is k0 = 2*pi.
Voxel n of an (nx, ny, nz) grid has the linear index n = ix + nx*(iy + ny*iz)
and its centre at origin + ((ix+1/2) hx, (iy+1/2) hy, (iz+1/2) hz).
Incident fields use the e^{+j omega t} time convention of the paper's Green's
function g = e^{-j k0 R} / (4 pi R) (Sec. II.A, Eq. 1): a plane wave
travelling along the unit vector d is p * exp(-j k0 d.r).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

K0 = 2.0 * math.pi  # free-space wavenumber for wavelength 1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """The splitmix64 output function (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64_sequence(state: int, count: int) -> np.ndarray:
    """The plain sequential splitmix64: state += golden gamma, output the mix."""
    with np.errstate(over="ignore"):
        ctr = np.arange(1, count + 1, dtype=np.uint64)
        return _mix64(np.uint64(state & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN)


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """`count` consecutive splitmix64 outputs of the generator keyed by
    (seed, stream). Counter-based: element i depends only on (seed, stream, i)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
                               ^ _mix64(np.array([np.uint64(stream)]))[0]],
                              dtype=np.uint64))[0]
        ctr = np.arange(1, count + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GOLDEN)


def uniform(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of splitmix64 / 2^53."""
    u = splitmix64(seed, count, stream) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class VoxelSet:
    """A set of equal-size box voxels (the pulse-basis cells).

    centres: (nv, 3) float64 voxel centres, natural order.
    h:       (3,) voxel edge lengths.
    eps_r:   (nv,) complex128 relative permittivity per voxel.
    shape:   (nx, ny, nz) for a full grid, or None for other layouts.
    """
    name: str
    centres: np.ndarray
    h: np.ndarray
    eps_r: np.ndarray
    shape: tuple | None = None

    @property
    def nv(self) -> int:
        return int(self.centres.shape[0])

    @property
    def n(self) -> int:
        """Number of unknowns: three field components per voxel."""
        return 3 * self.nv

    @property
    def dv(self) -> float:
        return float(np.prod(self.h))


def grid_centres(shape, h, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    nx, ny, nz = shape
    ix = np.arange(nx, dtype=np.float64)
    iy = np.arange(ny, dtype=np.float64)
    iz = np.arange(nz, dtype=np.float64)
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")  # x fastest
    c = np.stack([(X.ravel() + 0.5) * h[0] + origin[0],
                  (Y.ravel() + 0.5) * h[1] + origin[1],
                  (Z.ravel() + 0.5) * h[2] + origin[2]], axis=1)
    return np.ascontiguousarray(c)


def uniform_grid(shape, h, eps_r, name="grid") -> VoxelSet:
    h = np.asarray(h, dtype=np.float64)
    c = grid_centres(shape, h)
    eps = np.full(c.shape[0], complex(eps_r), dtype=np.complex128)
    return VoxelSet(name, c, h, eps, tuple(shape))


def random_eps_grid(shape, h, lo, hi, seed, name="grid") -> VoxelSet:
    """Grid with eps_r drawn i.i.d. uniform in [lo, hi] per voxel."""
    v = uniform_grid(shape, h, 1.0, name)
    u = uniform(seed, v.nv, stream=1)
    v.eps_r = (lo + (hi - lo) * u).astype(np.complex128)
    return v


def bump_eps_grid(shape, h, lo, hi, seed, n_bumps=16, name="grid") -> VoxelSet:
    """Smooth random eps_r in [lo, hi]: f = sum_i A_i exp(-|r-c_i|^2 / 2 s_i^2)
    with c_i uniform in the grid's box, s_i ~ U[0.25, 0.75], A_i ~ U[0, 1],
    rescaled linearly so that min f -> lo and max f -> hi."""
    v = uniform_grid(shape, h, 1.0, name)
    box = np.asarray(shape, dtype=np.float64) * v.h
    u = uniform(seed, 5 * n_bumps, stream=2).reshape(n_bumps, 5)
    f = np.zeros(v.nv)
    for i in range(n_bumps):
        c = u[i, 0:3] * box
        s = 0.25 + 0.5 * u[i, 3]
        a = u[i, 4]
        d2 = np.sum((v.centres - c) ** 2, axis=1)
        f += a * np.exp(-d2 / (2.0 * s * s))
    f = (f - f.min()) / (f.max() - f.min())
    v.eps_r = (lo + (hi - lo) * f).astype(np.complex128)
    return v


def void_grid(shape, h, eps_r, void_frac, seed, name="grid") -> VoxelSet:
    """Uniform eps_r with a Bernoulli(void_frac) set of voxels at eps_r = 1
    (kept as unknowns)."""
    v = uniform_grid(shape, h, eps_r, name)
    u = uniform(seed, v.nv, stream=3)
    v.eps_r[u < void_frac] = 1.0
    return v


def cube_array_1d(n_cubes, cube_vox, h, pitch, eps_r, name="array") -> VoxelSet:
    """n_cubes cubes of cube_vox^3 voxels each, centred on the x axis with the
    given pitch (cube edge + gap)."""
    one = grid_centres((cube_vox,) * 3, (h, h, h))
    offs = np.zeros((n_cubes, 3))
    offs[:, 0] = np.arange(n_cubes) * pitch
    c = (offs[:, None, :] + one[None, :, :]).reshape(-1, 3)
    eps = np.full(c.shape[0], complex(eps_r), dtype=np.complex128)
    return VoxelSet(name, np.ascontiguousarray(c), np.array([h, h, h]), eps, None)


def plane_wave(v: VoxelSet, direction, polarisation, k0: float = K0) -> np.ndarray:
    """Incident field p exp(-j k0 d.r) sampled at the voxel centres, as a
    length-3*nv complex128 vector ordered voxel-major, component-minor."""
    d = np.asarray(direction, dtype=np.float64)
    p = np.asarray(polarisation, dtype=np.complex128)
    ph = np.exp(-1j * k0 * (v.centres @ d))
    return (ph[:, None] * p[None, :]).reshape(-1)


def random_plane_waves(v: VoxelSet, count: int, seed: int, k0: float = K0):
    """`count` plane waves with directions uniform on the sphere
    (cos(theta) ~ U[-1,1], phi ~ U[0,2pi)) and a polarisation angle
    psi ~ U[0,2pi) in the plane orthogonal to the direction.
    Returns an (3*nv, count) complex128 array (column-major use)."""
    u = uniform(seed, 3 * count, stream=4).reshape(count, 3)
    out = np.empty((v.n, count), dtype=np.complex128)
    for i in range(count):
        ct = 2.0 * u[i, 0] - 1.0
        st = math.sqrt(max(0.0, 1.0 - ct * ct))
        ph = 2.0 * math.pi * u[i, 1]
        psi = 2.0 * math.pi * u[i, 2]
        d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
        th_hat = np.array([ct * math.cos(ph), ct * math.sin(ph), -st])
        ph_hat = np.array([-math.sin(ph), math.cos(ph), 0.0])
        p = math.cos(psi) * th_hat + math.sin(psi) * ph_hat
        out[:, i] = plane_wave(v, d, p, k0)
    return out


def random_complex(n: int, seed: int, stream: int = 5, cols: int = 1) -> np.ndarray:
    """Complex vector(s) with real and imaginary parts uniform in [-1, 1)."""
    u = uniform(seed, 2 * n * cols, stream=stream).reshape(2, n, cols)
    z = (2.0 * u[0] - 1.0) + 1j * (2.0 * u[1] - 1.0)
    return z[:, 0] if cols == 1 else z


# ---------------------------------------------------------------------------
# Workload recipes (sizes, permittivity fields, seeds, H^2 parameters).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    voxels: VoxelSet
    n_min: int        # leaf size in unknowns
    eta: float        # admissibility parameter, Eq. 4
    eps: float        # truncation accuracy
    nrhs: int
    rhs_seed: int | None  # None: the single x-polarised +z plane wave
    tol: float        # Krylov tolerance


def workload(name: str) -> Workload:
    """Named synthetic workloads.

    cube8    : 8^3 cube, side 0.5, eps_r 4, N = 1,536, leaf 64, eps 1e-4.
    cube32   : 32^3 cube, side 2, eps_r ~ U[2,6] (seed 2), N = 98,304, leaf 96.
    slab256  : 256x256x2 slab, 8 x 8 x 0.06, eps_r 3, N = 393,216, 128 RHS.
    cube48   : 48^3 cube, side 3, smooth eps_r in [2,8] (seed 4), N = 331,776.
    cube64v  : 64^3 cube, side 4, eps_r 4 with 10% void voxels (seed 7).
    array4096: 4096 cubes of 4^3 voxels on the x axis, pitch 0.5, eps_r 2.54.
    cube16r  : 16^3 cube, side 1, eps_r ~ U[2,6] (seed 2): the training geometry
               of the learned preconditioner (cube32's voxel size and eps_r law).
    Smaller grids "cubeNN" (uniform eps_r 4, side NN/16) are test cases, and
    "arrayNNN" is the array4096 family with NNN cubes (the 1-D scaling series).
    """
    h16 = 1.0 / 16.0
    if name == "cube8":
        v = uniform_grid((8, 8, 8), (h16,) * 3, 4.0, name)
        return Workload(v, 64, 1.0, 1e-4, 1, None, 1e-6)
    if name == "cube32":
        v = random_eps_grid((32, 32, 32), (h16,) * 3, 2.0, 6.0, seed=2, name=name)
        return Workload(v, 96, 1.0, 1e-4, 1, None, 1e-4)
    if name == "slab256":
        v = uniform_grid((256, 256, 2), (1.0 / 32, 1.0 / 32, 0.03), 3.0, name)
        return Workload(v, 96, 1.0, 1e-4, 128, 3, 1e-4)
    if name == "cube48":
        v = bump_eps_grid((48, 48, 48), (h16,) * 3, 2.0, 8.0, seed=4, name=name)
        return Workload(v, 96, 1.0, 1e-4, 1, None, 1e-4)
    if name == "cube64v":
        v = void_grid((64, 64, 64), (h16,) * 3, 4.0, 0.10, seed=7, name=name)
        return Workload(v, 96, 1.0, 1e-4, 256, 8, 1e-4)
    if name == "array4096":
        v = cube_array_1d(4096, 4, h16, 0.5, 2.54, name)
        return Workload(v, 96, 1.0, 1e-4, 256, 8, 1e-4)
    if name == "cube16r":
        # same voxel size and eps_r distribution as cube32, 16^3 voxels
        v = random_eps_grid((16, 16, 16), (h16,) * 3, 2.0, 6.0, seed=2, name=name)
        return Workload(v, 96, 1.0, 1e-4, 1, None, 1e-4)
    if name.startswith("array") and name[5:].isdigit():
        v = cube_array_1d(int(name[5:]), 4, h16, 0.5, 2.54, name)
        return Workload(v, 96, 1.0, 1e-4, 256, 8, 1e-4)
    if name.startswith("cube") and name[4:].isdigit():
        m = int(name[4:])
        v = uniform_grid((m, m, m), (h16,) * 3, 4.0, name)
        return Workload(v, 96 if m >= 16 else 64, 1.0, 1e-4, 1, None, 1e-4)
    raise KeyError(name)


def default_rhs(w: Workload) -> np.ndarray:
    """The workload's right-hand side(s): the x-polarised plane wave incident
    along +z, or `nrhs` random plane waves."""
    if w.rhs_seed is None:
        return plane_wave(w.voxels, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0))
    return random_plane_waves(w.voxels, w.nrhs, w.rhs_seed)
