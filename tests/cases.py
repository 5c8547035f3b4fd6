"""Shared test cases: oracle-built H^2 operators and their C-ABI arrays.

The H^2 data of these cases is produced by the oracle's truncated-SVD build;
the CUDA library receives it only as input (h2_load) and its products are
compared with the oracle's FP64 products on the same data.
"""
from __future__ import annotations

import functools
import math

import numpy as np

import synth
from oracle import h2build, h2mv, tree as otree, vie
from paper_1703_01175_gb300 import h2 as h2py

K = 2.0 * math.pi


class Case:
    def __init__(self, name, v, n_min, eps, eta=1.0):
        self.name = name
        self.v = v
        Kd = vie.assemble_K(v.centres, v.dv, K)
        self.tree = otree.build_tree(v.centres, n_min)
        self.part = otree.partition(self.tree, eta)
        Kt = h2build.to_tree_order(Kd, self.tree)
        hK = h2build.build_h2_K(Kt, self.tree, self.part, eps)
        self.chi = vie.chi_unknowns(v.eps_r)[self.tree.unknown_perm()]
        self.hZ = h2build.system_h2(hK, self.chi)
        self.Zt = np.eye(self.tree.n) - Kt * self.chi[None, :]
        self.n = self.tree.n

    def arrays(self, dtype=np.complex128, symmetric=False) -> h2py.H2Arrays:
        tr, hZ = self.tree, self.hZ
        W = None if symmetric else hZ.W
        return h2py.arrays_from_blocks(tr.n, tr.level_ptr, tr.child, tr.begin, tr.size, hZ.rank,
                                       hZ.U, W, hZ.T, hZ.S, hZ.Z, dtype=dtype)

    def oracle_matvec(self, x):
        if x.ndim == 1:
            return h2mv.h2_matvec(self.hZ, x)
        return np.stack([h2mv.h2_matvec(self.hZ, x[:, j]) for j in range(x.shape[1])], axis=1)

    @functools.cached_property
    def hZ32(self):
        """The same H^2 data rounded to complex64, as the device stores it."""
        def rnd(d):
            return None if d is None else {k: v.astype(np.complex64).astype(np.complex128) for k, v in d.items()}
        h = self.hZ
        return h2build.H2(h.tree, h.part, h.rank, rnd(h.U), rnd(h.W), rnd(h.T), rnd(h.S), rnd(h.Z))

    def oracle_matvec_stored(self, x):
        """FP64 product with the complex64-rounded data: the exact result an
        accumulation of the stored data should reproduce."""
        return h2mv.h2_matvec(self.hZ32, x)


@functools.lru_cache(maxsize=None)
def get(name: str) -> Case:
    if name == "cube8":
        w = synth.workload("cube8")
        return Case(name, w.voxels, w.n_min, w.eps)
    if name == "ragged":
        v = synth.random_eps_grid((7, 5, 6), (1 / 16,) * 3, 2.0, 6.0, seed=3)
        return Case(name, v, 40, 1e-4)
    if name == "odd":  # 175 voxels: an odd number of unknowns (525)
        v = synth.random_eps_grid((7, 5, 5), (1 / 16,) * 3, 2.0, 6.0, seed=9)
        return Case(name, v, 40, 1e-4)
    if name == "cube12":
        v = synth.random_eps_grid((12, 12, 12), (1 / 16,) * 3, 2.0, 6.0, seed=12)
        return Case(name, v, 96, 1e-4)
    if name == "slab":
        v = synth.uniform_grid((24, 20, 2), (1 / 32, 1 / 32, 0.03), 3.0)
        return Case(name, v, 60, 1e-4)
    if name == "array":
        v = synth.cube_array_1d(40, 2, 1 / 16, 0.25, 2.54)
        return Case(name, v, 24, 1e-4)
    if name == "single_leaf":
        v = synth.uniform_grid((2, 2, 2), (1 / 16,) * 3, 4.0)
        return Case(name, v, 24, 1e-4)
    if name == "tiny_leaves":
        v = synth.random_eps_grid((4, 3, 3), (1 / 16,) * 3, 2.0, 6.0, seed=6)
        return Case(name, v, 3, 1e-4)
    raise KeyError(name)
