"""Host-side construction of the minimal-rank H^2 representation of the
pulse-basis E-field VIE matrix Z = I - K diag(chi) (setup; not on the timed
path). Produces the arrays that h2_load takes.

Operator (the paper's kernel-independent construction applied to the voxel
E-field VIE): K_mn = dV k^2 g(R) [(1 - j/kR - 1/kR^2) I + (-1 + 3j/kR + 3/kR^2) R^R^]
for m != n with g = e^{-jkR}/(4 pi R) (Sec. II.A), and the equivalent-sphere
self term K_mm = [(2/3)((1 + jka) e^{-jka} - 1) - 1/3] I, a = (3 dV / 4 pi)^{1/3}.

Steps (Omar & Jiao):
  * cluster tree by balanced bisection of the voxels and strong-admissibility
    block partition, Sec. III.A, Eq. 4 (voxel centres' bounding boxes; split
    along the longest box edge at the median voxel; leaf when 3 * #voxels <=
    n_min);
  * Stage I, Sec. III.B: for every cluster t the admissible blocks of its own
    level are grouped into G^t (Eq. 5), approximated by adaptive cross
    approximation with partial pivoting to eps_A (Eq. 6) and recompressed by a
    reduced SVD to eps_acc (Eq. 7): G^t ~ A_t B_t^T;
  * Stage II, Sec. III.C: leaf bases from the Gram matrix of the leaf's rows of
    its own and all its ancestors' A B^T factors (Eqs. 10-12), non-leaf
    transfer matrices from the Gram matrix projected on the children's bases
    (Eqs. 13-16), couplings S = V^{tH} A B^T conj(V^s) (Eqs. 17-18);
  * the system matrix takes row basis U = V, column basis W = diag(chi) V,
    couplings -S and near blocks delta_ts I - K^{(t,s)} diag(chi_s).

Truncation reading: singular values (eigenvalues of a Gram matrix) above
eps * sigma_1 (eps^2 * lambda_1) of the matrix being decomposed.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .h2 import H2Arrays, arrays_from_blocks

_LIBB = None


def _libb():
    """The native constructor helpers (include/h2build.h)."""
    global _LIBB
    if _LIBB is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libh2build.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1703_01175_gb300.build.build_all()")
        L = ctypes.CDLL(path)
        dp, i64p = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
        L.h2c_aca_vie.restype = ctypes.c_int
        L.h2c_aca_vie.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  i64p, ctypes.c_int32, i64p, ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_int32, dp, dp, ctypes.POINTER(ctypes.c_int32), i64p, dp]
        L.h2c_block_vie.restype = ctypes.c_int
        L.h2c_block_vie.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    i64p, ctypes.c_int32, i64p, ctypes.c_int32, dp, ctypes.c_double,
                                    ctypes.c_double, dp]
        _LIBB = L
    return _LIBB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class _BlasThreads:
    """Context manager pinning every loaded OpenBLAS (numpy and scipy each
    bring their own) to n threads (no-op for a library whose thread-control
    symbol cannot be found), so that a pool of Python worker threads does not
    oversubscribe the cores."""
    _cache = {}   # library path -> (set, get) or None

    def __init__(self, n):
        self.n = n
        self.old = []

    @classmethod
    def _lookup(cls):
        """(set, get) function pairs of every OpenBLAS mapped into the process."""
        try:
            with open("/proc/self/maps") as f:
                libs = sorted({line.split()[-1] for line in f
                               if "openblas" in line and (line.strip().endswith(".so") or ".so." in line)})
        except OSError:
            libs = []
        out = []
        for path in libs:
            if path not in cls._cache:
                cls._cache[path] = None
                try:
                    L = ctypes.CDLL(path)
                except OSError:
                    continue
                for sset, sget in (("scipy_openblas_set_num_threads64_", "scipy_openblas_get_num_threads64_"),
                                   ("scipy_openblas_set_num_threads", "scipy_openblas_get_num_threads"),
                                   ("openblas_set_num_threads64_", "openblas_get_num_threads64_"),
                                   ("openblas_set_num_threads", "openblas_get_num_threads")):
                    if hasattr(L, sset) and hasattr(L, sget):
                        fs, fg = getattr(L, sset), getattr(L, sget)
                        fs.argtypes, fs.restype = [ctypes.c_int], None
                        fg.argtypes, fg.restype = [], ctypes.c_int
                        cls._cache[path] = (fs, fg)
                        break
            if cls._cache[path] is not None:
                out.append(cls._cache[path])
        return out

    @classmethod
    def threads(cls) -> int:
        """Threads of the first pinned library (os.cpu_count() if none is found)."""
        fns = cls._lookup()
        return fns[0][1]() if fns else (os.cpu_count() or 1)

    def __enter__(self):
        self.old = []
        for fs, fg in self._lookup():
            self.old.append((fs, fg()))
            fs(self.n)
        return self

    def __exit__(self, *exc):
        for fs, n in self.old:
            fs(n)

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# kernel entries
# ---------------------------------------------------------------------------

class VieKernel:
    """Entries of K for voxel centres `c` (nv, 3) of volume dv at wavenumber k."""

    def __init__(self, centres, dv, k=TWO_PI):
        self.c = np.ascontiguousarray(centres, dtype=np.float64)
        self.dv = float(dv)
        self.k = float(k)
        a = (3.0 * self.dv / (4.0 * math.pi)) ** (1.0 / 3.0)
        ka = self.k * a
        self.self_val = (2.0 / 3.0) * ((1.0 + 1j * ka) * np.exp(-1j * ka) - 1.0) - 1.0 / 3.0

    def blocks(self, vi, vj) -> np.ndarray:
        """K[(vi, a), (vj, b)] as an array (len(vi), 3, len(vj), 3)."""
        ci = self.c[np.asarray(vi)]
        cj = self.c[np.asarray(vj)]
        R = ci[:, None, :] - cj[None, :, :]
        r2 = np.einsum("ijk,ijk->ij", R, R)
        same = r2 == 0.0
        r = np.sqrt(np.where(same, 1.0, r2))
        kr = self.k * r
        inv = 1.0 / kr
        g = np.exp(-1j * kr) / (4.0 * math.pi * r)
        pre = self.dv * self.k * self.k * g
        ca = pre * (1.0 - 1j * inv - inv * inv)
        cb = pre * (-1.0 + 3j * inv + 3.0 * inv * inv)
        Rh = R / r[..., None]
        out = cb[:, :, None, None] * (Rh[:, :, :, None] * Rh[:, :, None, :])
        for a in range(3):
            out[:, :, a, a] += ca
        if same.any():
            ii, jj = np.nonzero(same)
            out[ii, jj] = 0.0
            for a in range(3):
                out[ii, jj, a, a] = self.self_val
        return out.transpose(0, 2, 1, 3)

    def matrix(self, vi, vj) -> np.ndarray:
        b = self.blocks(vi, vj)
        return b.reshape(3 * len(vi), 3 * len(vj))

    def unknown_row(self, i_vox, comp, vj) -> np.ndarray:
        """Row (i_vox, comp) of K against voxels vj (all components)."""
        return self.blocks([i_vox], vj)[0, comp].reshape(-1)

    def aca_native(self, rows_vox, cols_vox, eps, kmax0=128):
        """Stage-I ACA of K[rows, cols] in native code.

        Returns (U, V, piv_rows, piv_vals): K[rows, cols] ~ U V^T, and row
        piv_rows[l] of the block equals piv_vals[l] v_l + sum_{p<l} U[piv_rows[l], p] v_p."""
        L = _libb()
        rv = np.ascontiguousarray(rows_vox, dtype=np.int64)
        cv = np.ascontiguousarray(cols_vox, dtype=np.int64)
        m, n = 3 * len(rv), 3 * len(cv)
        kmax = min(kmax0, m, n)
        while True:
            U = np.empty((kmax, m), dtype=np.complex128)
            V = np.empty((kmax, n), dtype=np.complex128)
            pr = np.empty(kmax, dtype=np.int64)
            pvv = np.empty(kmax, dtype=np.complex128)
            kk = ctypes.c_int32(0)
            st = L.h2c_aca_vie(_dp(self.c), self.dv, self.k, self.self_val.real, self.self_val.imag,
                               _i64p(rv), len(rv), _i64p(cv), len(cv), eps, kmax,
                               _dp(U), _dp(V), ctypes.byref(kk), _i64p(pr), _dp(pvv))
            if st < 0:
                raise ValueError("h2c_aca_vie: bad arguments")
            if st == 0 or kmax >= min(m, n):
                k = kk.value
                return U[:k].T, V[:k].T, pr[:k], pvv[:k]
            kmax = min(2 * kmax, m, n)

    def block_native(self, rows_vox, cols_vox, colscale=None, alpha=1.0):
        """alpha * K[rows, cols] * diag(colscale per column voxel), native."""
        L = _libb()
        rv = np.ascontiguousarray(rows_vox, dtype=np.int64)
        cv = np.ascontiguousarray(cols_vox, dtype=np.int64)
        out = np.empty((3 * len(cv), 3 * len(rv)), dtype=np.complex128)  # column-major storage
        cs = None if colscale is None else np.ascontiguousarray(colscale, dtype=np.complex128)
        L.h2c_block_vie(_dp(self.c), self.dv, self.k, self.self_val.real, self.self_val.imag,
                        _i64p(rv), len(rv), _i64p(cv), len(cv),
                        _dp(cs) if cs is not None else None, complex(alpha).real, complex(alpha).imag,
                        _dp(out))
        return out.T


# ---------------------------------------------------------------------------
# tree and partition
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class ClusterTree:
    perm: np.ndarray        # tree position -> voxel
    level_ptr: np.ndarray
    child: np.ndarray       # (nc, 2)
    parent: np.ndarray
    level: np.ndarray
    vbegin: np.ndarray
    vsize: np.ndarray
    lo: np.ndarray
    hi: np.ndarray

    @property
    def nc(self):
        return len(self.vsize)

    def leaf(self, t):
        return self.child[t, 0] < 0


def cluster_tree(centres: np.ndarray, n_min: int) -> ClusterTree:
    """Balanced binary bisection of the voxels (Sec. III.A), numbered level by
    level, each cluster a contiguous range of the tree order."""
    c = np.asarray(centres, dtype=np.float64)
    nv = c.shape[0]
    # level-synchronous construction keeps breadth-first numbering
    cur = [np.arange(nv)]
    cur_parent = [-1]
    levels, parents, childs, sets = [], [], [], []
    lev = 0
    while cur:
        nxt, nxt_parent = [], []
        base = len(sets)
        for i, vox in enumerate(cur):
            idx = base + i
            sets.append(vox)
            parents.append(cur_parent[i])
            levels.append(lev)
            if 3 * len(vox) <= n_min or len(vox) < 2:
                childs.append((-1, -1))
                continue
            p = c[vox]
            ext = p.max(0) - p.min(0)
            ax = int(np.nonzero(ext >= ext.max() * (1.0 - 1e-12))[0][0])
            order = np.lexsort((vox, p[:, ax]))
            srt = vox[order]
            h = (len(vox) + 1) // 2
            childs.append((len(nxt), len(nxt) + 1))  # relative, fixed below
            nxt.extend([srt[:h], srt[h:]])
            nxt_parent.extend([idx, idx])
        nbase = base + len(cur)
        for i in range(len(cur)):
            a, b = childs[base + i]
            if a >= 0:
                childs[base + i] = (nbase + a, nbase + b)
        cur, cur_parent = nxt, nxt_parent
        lev += 1
    nc = len(sets)
    child = np.array(childs, dtype=np.int64).reshape(nc, 2)
    parent = np.array(parents, dtype=np.int64)
    level = np.array(levels, dtype=np.int64)
    vsize = np.array([len(s) for s in sets], dtype=np.int64)
    vbegin = np.zeros(nc, dtype=np.int64)
    for t in range(nc):  # parents precede children in BFS order
        a, b = child[t]
        if a >= 0:
            vbegin[a] = vbegin[t]
            vbegin[b] = vbegin[t] + vsize[a]
    perm = np.empty(nv, dtype=np.int64)
    lo = np.empty((nc, 3))
    hi = np.empty((nc, 3))
    for t in range(nc):
        if child[t, 0] < 0:
            perm[vbegin[t]:vbegin[t] + vsize[t]] = sets[t]
        p = c[sets[t]]
        lo[t] = p.min(0)
        hi[t] = p.max(0)
    level_ptr = np.searchsorted(level, np.arange(level.max() + 2))
    return ClusterTree(perm, level_ptr, child, parent, level, vbegin, vsize, lo, hi)


def block_partition(tr: ClusterTree, eta: float):
    """Admissible and near pairs from (root, root) down (Sec. III.A, Eq. 4).
    A pair is admissible when its box distance d > 0 and
    max(diam_t, diam_s) <= eta * d."""
    diam = np.sqrt(np.sum((tr.hi - tr.lo) ** 2, axis=1))
    adm, near = [], []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        gap = np.maximum(0.0, np.maximum(tr.lo[t] - tr.hi[s], tr.lo[s] - tr.hi[t]))
        d = math.sqrt(float(gap @ gap))
        if d > 0.0 and max(diam[t], diam[s]) <= eta * d:
            adm.append((t, s))
            continue
        lt, ls = tr.child[t, 0] < 0, tr.child[s, 0] < 0
        if lt and ls:
            near.append((t, s))
        elif lt:
            stack.extend((t, int(x)) for x in tr.child[s])
        elif ls:
            stack.extend((int(x), s) for x in tr.child[t])
        else:
            stack.extend((int(a), int(b)) for a in tr.child[t] for b in tr.child[s])
    adm.sort()
    near.sort()
    return adm, near


# ---------------------------------------------------------------------------
# Stage I: grouped ACA + reduced SVD
# ---------------------------------------------------------------------------

def aca(row_fn, col_fn, m: int, n: int, eps: float, kmax: int):
    """Adaptive cross approximation with partial pivoting: M ~ U V^T.
    Stops when |u_k||v_k| <= eps ||U V^T||_F on two consecutive steps."""
    kcap = max(8, min(kmax, 64))
    U = np.zeros((m, kcap), dtype=np.complex128)
    V = np.zeros((n, kcap), dtype=np.complex128)
    used = np.zeros(m, dtype=bool)
    i, k, norm2, small = 0, 0, 0.0, 0
    while k < kmax:
        r = row_fn(i)
        if k:
            r = r - V[:, :k] @ U[i, :k]
        used[i] = True
        j = int(np.argmax(np.abs(r)))
        piv = r[j]
        if piv == 0.0:
            free = np.nonzero(~used)[0]
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v = r / piv
        u = col_fn(j)
        if k:
            u = u - U[:, :k] @ V[j, :k]
        nu2 = float(np.vdot(u, u).real)
        nv2 = float(np.vdot(v, v).real)
        if k:
            cross = (U[:, :k].conj().T @ u) * np.conj(V[:, :k].conj().T @ v)
            norm2 += 2.0 * float(cross.sum().real)
        norm2 += nu2 * nv2
        if k == kcap:
            kcap = min(kmax, 2 * kcap)
            U = np.concatenate([U, np.zeros((m, kcap - k), dtype=U.dtype)], axis=1)
            V = np.concatenate([V, np.zeros((n, kcap - k), dtype=V.dtype)], axis=1)
        U[:, k] = u
        V[:, k] = v
        k += 1
        if math.sqrt(nu2 * nv2) <= eps * math.sqrt(max(norm2, 0.0)):
            small += 1
            if small >= 2:
                break
        else:
            small = 0
        au = np.abs(u)
        au[used] = -1.0
        i = int(np.argmax(au))
        if au[i] < 0.0:
            break
    return U[:, :k], V[:, :k]


def reduced_svd(U: np.ndarray, V: np.ndarray, eps: float):
    """Recompress U V^T to A B^T with sigma_i > eps sigma_1 (Eq. 7).

    U = Q_U R_U and V = Q_V R_V are orthogonalised through the eigen-
    decompositions of their k' x k' Gram matrices (R = Lambda^{1/2} E^H); the
    SVD R_U R_V^T = X Sigma Y^H then gives A = Q_U X Sigma and
    B = Q_V conj(Y), so that B^T conj(B) = I. Returns (A, C) with B = V C."""
    k = U.shape[1]
    if k == 0:
        return U, np.zeros((0, 0), dtype=np.complex128)
    lu, Eu = np.linalg.eigh(U.conj().T @ U)
    lv, Ev = np.linalg.eigh(V.conj().T @ V)
    if lu[-1] <= 0.0 or lv[-1] <= 0.0:
        return U[:, :0], np.zeros((k, 0), dtype=np.complex128)
    mu = lu > 1e-13 * lu[-1]
    mv = lv > 1e-13 * lv[-1]
    Eu, lu = Eu[:, mu], np.sqrt(lu[mu])
    Ev, lv = Ev[:, mv], np.sqrt(lv[mv])
    Ru = lu[:, None] * Eu.conj().T
    Rv = lv[:, None] * Ev.conj().T
    X, sv, Yh = np.linalg.svd(Ru @ Rv.T)
    kk = int(np.count_nonzero(sv > eps * sv[0]))
    A = U @ ((Eu / lu[None, :]) @ (X[:, :kk] * sv[:kk]))
    C = (Ev / lv[None, :]) @ Yh[:kk, :].T
    return A, C


def _trunc_eig(G: np.ndarray, eps: float) -> np.ndarray:
    """Eigenvectors of the Hermitian PSD G with eigenvalue > eps^2 lambda_max
    (Eqs. 11, 15), in decreasing order."""
    G = 0.5 * (G + G.conj().T)
    w, Q = np.linalg.eigh(G)
    w, Q = w[::-1], Q[:, ::-1]
    if w.size == 0 or w[0] <= 0.0:
        return Q[:, :0]
    kk = int(np.count_nonzero(w > eps * eps * w[0]))
    return np.ascontiguousarray(Q[:, :kk])


@dataclasses.dataclass
class BuildInfo:
    seconds: dict
    stage1_rank: dict
    adm: list
    near: list


def build_vie_h2(centres, dv, eps_r, n_min=96, eta=1.0, eps=1e-4, k=TWO_PI,
                 eps_aca=None, eps_stage1=None, near_dtype=np.complex64,
                 out_dtype=np.complex64, threads=None, verbose=False):
    """Build the H^2 arrays of Z = I - K diag(chi) for voxels at `centres`.

    Returns (arrays, tree, info). `arrays` is an H2Arrays in tree order
    (unknown 3 p + c is component c of the voxel at tree position p;
    tree.perm maps tree positions to voxel indices).
    """
    t_all = time.time()
    secs = {}
    threads = threads or os.cpu_count() or 4
    eps_aca = eps / 10.0 if eps_aca is None else eps_aca
    eps_stage1 = eps / 3.0 if eps_stage1 is None else eps_stage1
    kern = VieKernel(centres, dv, k)
    chi_vox = np.asarray(eps_r, dtype=np.complex128) - 1.0

    t0 = time.time()
    tr = cluster_tree(centres, n_min)
    adm, near = block_partition(tr, eta)
    secs["tree_partition"] = time.time() - t0
    nc = tr.nc
    vox = [tr.perm[tr.vbegin[t]:tr.vbegin[t] + tr.vsize[t]] for t in range(nc)]
    partners = [[] for _ in range(nc)]
    for t, s in adm:
        partners[t].append(s)

    # ---- Stage I -----------------------------------------------------------------
    # G^t ~ A_t B_t^T with B_t = V_aca C_t. ACA with partial pivoting is a cross
    # approximation: V_aca^T = L^{-1} G^t[I, :] for the pivot rows I and the
    # lower-triangular L (L_ll = pivot, L_lp = U[I_l, p]), so
    # B_t = G^t[I, :]^T D_t with D_t = L^{-T} C_t: only the k' pivot rows of
    # K are needed later to re-form any block of B_t.
    import scipy.linalg
    t0 = time.time()
    fac = {}     # t -> (A_t, pivot voxels, pivot components, D_t)
    s1rank = {}
    cols_of = {t: np.concatenate([vox[s] for s in partners[t]]) for t in range(nc) if partners[t]}

    def stage1(t):
        Ua, Va, prow, pval = kern.aca_native(vox[t], cols_of[t], eps_aca)
        A, C = reduced_svd(Ua, Va, eps_stage1)
        kp = Ua.shape[1]
        Lm = np.tril(Ua[prow, :], -1) + np.diag(pval)
        D = scipy.linalg.solve_triangular(Lm.T, C, lower=False) if kp else C
        return t, A, vox[t][prow // 3], prow % 3, D, kp

    work = sorted(cols_of, key=lambda t: -len(vox[t]) * len(cols_of[t]))
    with _BlasThreads(1), ThreadPoolExecutor(threads) as ex:
        for t, A, pvox, pcomp, D, kp in ex.map(stage1, work):
            fac[t] = (A, pvox, pcomp, D)
            s1rank[t] = (kp, A.shape[1])
    secs["stage1"] = time.time() - t0
    if verbose:
        print(f"construct: stage I {secs['stage1']:.1f} s ({len(fac)} clusters)", flush=True)

    # ---- Stage II: bases and transfers, bottom-up ---------------------------------
    t0 = time.time()
    # B_j^T conj(B_j) of Eq. 10: the identity for the reduced-SVD normalisation above
    M = {t: np.eye(f[0].shape[1], dtype=np.complex128) for t, f in fac.items()}
    anc_f = []
    for t in range(nc):
        lst, a = [], t
        while a >= 0:
            if a in fac:
                lst.append(a)
            a = int(tr.parent[a])
        anc_f.append(lst)
    rank = np.zeros(nc, dtype=np.int64)
    V_leaf, T = {}, {}
    P = {}       # P[c][j] = V^{cH} A_j|_c for j in anc_f(c)
    PT = {}      # P[t][t]
    nlev = len(tr.level_ptr) - 1
    for lev in range(nlev - 1, -1, -1):
        for t in range(int(tr.level_ptr[lev]), int(tr.level_ptr[lev + 1])):
            if tr.leaf(t):
                n_t = 3 * int(tr.vsize[t])
                if anc_f[t]:
                    G2 = np.zeros((n_t, n_t), dtype=np.complex128)
                    rows = {}
                    for j in anc_f[t]:
                        r0 = 3 * int(tr.vbegin[t] - tr.vbegin[j])
                        Aj = fac[j][0][r0:r0 + n_t]
                        rows[j] = Aj
                        G2 += Aj @ M[j] @ Aj.conj().T
                    V = _trunc_eig(G2, eps)
                    P[t] = {j: V.conj().T @ rows[j] for j in anc_f[t]}
                else:
                    V = np.zeros((n_t, 0), dtype=np.complex128)
                    P[t] = {}
                V_leaf[t] = V
                rank[t] = V.shape[1]
            else:
                c1, c2 = (int(x) for x in tr.child[t])
                k1, k2 = int(rank[c1]), int(rank[c2])
                if anc_f[t] and k1 + k2 > 0:
                    G2 = np.zeros((k1 + k2, k1 + k2), dtype=np.complex128)
                    small = {}
                    for j in anc_f[t]:
                        As = np.vstack([P[c1][j], P[c2][j]])
                        small[j] = As
                        G2 += As @ M[j] @ As.conj().T
                    Pm = _trunc_eig(G2, eps)
                else:
                    Pm = np.zeros((k1 + k2, 0), dtype=np.complex128)
                    small = {}
                T[c1] = Pm[:k1]
                T[c2] = Pm[k1:]
                rank[t] = Pm.shape[1]
                P[t] = {j: Pm.conj().T @ small[j] for j in anc_f[t]} if small else {}
                del P[c1], P[c2]
            if t in fac:
                PT[t] = P[t][t]
    P.clear()
    secs["stage2_bases"] = time.time() - t0
    if verbose:
        print(f"construct: stage II bases {secs['stage2_bases']:.1f} s", flush=True)

    # ---- couplings (Eq. 18) with expanded bases, level by level ---------------------
    # S^{t,s} = V^{tH} A_t B_{t,s}^T conj(V^s) = P_{t,t} (V^{sH} B_{t,s})^T, with
    # B_{t,s} = K[I_t, s]^T D_t re-formed from the pivot rows of G^t.
    t0 = time.time()
    S = {}
    below = {}

    def couple(args):
        t, lst, cur = args
        A, pvox, pcomp, D = fac[t]
        out = []
        for s in lst:
            # K[s, I_t]: rows of s against the pivot unknowns of G^t (K symmetric)
            Kb = kern.block_native(vox[s], pvox)
            KsI = Kb[:, 3 * np.arange(len(pvox)) + pcomp]
            Q = (cur[s].conj().T @ KsI) @ D               # V^{sH} B_{t,s}
            out.append(((t, s), -(PT[t] @ Q.T)))           # system matrix: -K
        return out

    for lev in range(nlev - 1, -1, -1):
        cur = {}
        for c in range(int(tr.level_ptr[lev]), int(tr.level_ptr[lev + 1])):
            if tr.leaf(c):
                cur[c] = V_leaf[c]
            else:
                c1, c2 = (int(x) for x in tr.child[c])
                cur[c] = np.vstack([below[c1] @ T[c1], below[c2] @ T[c2]])
        rows_here = {}
        for t, s in adm:
            if int(tr.level[s]) == lev and int(rank[t]) > 0 and int(rank[s]) > 0:
                rows_here.setdefault(t, set()).add(s)
        jobs = [(t, lst, cur) for t, lst in rows_here.items()]
        with _BlasThreads(1), ThreadPoolExecutor(threads) as ex:
            for lst in ex.map(couple, jobs):
                for key, blk in lst:
                    S[key] = blk
        below = cur
    for t, s in adm:  # zero-rank couplings
        if (t, s) not in S:
            S[(t, s)] = np.zeros((int(rank[t]), int(rank[s])), dtype=np.complex128)
    # K is complex symmetric and both sides use the same basis, so Eq. 18 gives
    # S^{s,t} = (S^{t,s})^T; the two skeleton estimates above agree only to the
    # truncation accuracy, and their mean restores the symmetry exactly
    for t, s in adm:
        if t < s:
            m = 0.5 * (S[(t, s)] + S[(s, t)].T)
            S[(t, s)] = m
            S[(s, t)] = m.T.copy()
    secs["couplings"] = time.time() - t0
    if verbose:
        print(f"construct: couplings {secs['couplings']:.1f} s", flush=True)

    # ---- near field ----------------------------------------------------------------
    t0 = time.time()
    Z = {}
    chi_tree_vox = chi_vox[tr.perm]
    near_by_row = {}
    for t, s in near:
        near_by_row.setdefault(t, []).append(s)

    def near_row(t):
        lst = near_by_row[t]
        cols = np.concatenate([vox[s] for s in lst])
        Zb = kern.block_native(vox[t], cols, colscale=chi_vox[cols], alpha=-1.0)
        out, off = [], 0
        for s in lst:
            ns = 3 * len(vox[s])
            blk = Zb[:, off:off + ns]
            if s == t:
                blk = blk + np.eye(ns)
            out.append(((t, s), blk.astype(near_dtype)))
            off += ns
        return out

    with _BlasThreads(1), ThreadPoolExecutor(threads) as ex:
        for lst in ex.map(near_row, list(near_by_row)):
            for key, blk in lst:
                Z[key] = blk
    secs["near"] = time.time() - t0
    if verbose:
        print(f"construct: near field {secs['near']:.1f} s", flush=True)

    # ---- system-matrix bases ---------------------------------------------------------
    U = {t: V for t, V in V_leaf.items()}
    W = {t: np.repeat(chi_tree_vox[tr.vbegin[t]:tr.vbegin[t] + tr.vsize[t]], 3)[:, None] * V
         for t, V in V_leaf.items()}
    t0 = time.time()
    arrs = arrays_from_blocks(3 * len(tr.perm), tr.level_ptr, tr.child, 3 * tr.vbegin,
                              3 * tr.vsize, rank, U, W, T, S, Z, dtype=out_dtype)
    secs["pack"] = time.time() - t0
    secs["total"] = time.time() - t_all
    if verbose:
        print("construct:", {k: round(v, 2) for k, v in secs.items()})
    return arrs, tr, BuildInfo(secs, s1rank, adm, near)


def _source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    here = os.path.dirname(os.path.abspath(__file__))
    for rel in ("construct.py", "h2.py", os.path.join("csrc_host", "h2_construct.cpp")):
        with open(os.path.join(here, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def build_vie_h2_cached(centres, dv, eps_r, n_min=96, eta=1.0, eps=1e-4, k=TWO_PI,
                        out_dtype=np.complex64, cache_dir=None, verbose=False):
    """build_vie_h2 with an on-disk cache of the resulting arrays, keyed by the
    inputs and the constructor's sources (directory: $H2_CACHE_DIR, default
    /tmp/h2_cache). Returns (arrays, perm)."""
    import hashlib
    cache_dir = cache_dir or os.environ.get("H2_CACHE_DIR") or "/tmp/h2_cache"
    h = hashlib.sha256()
    for a in (np.ascontiguousarray(centres, dtype=np.float64), np.ascontiguousarray(eps_r, dtype=np.complex128)):
        h.update(a.tobytes())
    h.update(repr((float(dv), int(n_min), float(eta), float(eps), float(k), np.dtype(out_dtype).str)).encode())
    h.update(_source_hash().encode())
    path = os.path.join(cache_dir, f"h2_{h.hexdigest()[:24]}.npz")
    fields = [f.name for f in dataclasses.fields(H2Arrays)]
    if os.path.exists(path):
        try:
            z = np.load(path, allow_pickle=False)
            vals = {f: (None if f"{f}__none" in z.files else (int(z[f]) if f == "n" else z[f])) for f in fields}
            return H2Arrays(**vals), z["perm"]
        except Exception:
            pass
    arrs, tr, info = build_vie_h2(centres, dv, eps_r, n_min=n_min, eta=eta, eps=eps, k=k,
                                  out_dtype=out_dtype, verbose=verbose)
    try:
        os.makedirs(cache_dir, exist_ok=True)
        payload = {}
        for f in fields:
            v = getattr(arrs, f)
            if v is None:
                payload[f"{f}__none"] = np.zeros(1)
            else:
                payload[f] = np.asarray(v)
        payload["perm"] = tr.perm
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, **payload)
        os.replace(tmp, path)
    except OSError:
        pass
    return arrs, tr.perm
