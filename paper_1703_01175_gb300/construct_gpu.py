"""GPU construction of the minimal-rank H^2 representation of the pulse-basis
E-field VIE matrix Z = I - K diag(chi) (setup; not on the timed path).

The steps are those of the host constructor (construct.py), in the paper's
order:
  * cluster tree and strong-admissibility partition (Sec. III.A, Eq. 4), on
    the host;
  * Stage I (Sec. III.B, Eqs. 5-7): the admissible blocks of every cluster t at
    its own level grouped into G^t and approximated by adaptive cross
    approximation (GPU, one thread block per cluster), then recompressed by a
    reduced SVD whose Gram matrices are GPU products and whose k' x k'
    eigen- and singular value decompositions run on the host in FP64;
  * Stage II (Sec. III.C, Eqs. 10-16): leaf Gram matrices and projected Gram
    matrices formed on the GPU with FP64 accumulation (their eigenvalues are
    truncated at eps^2 lambda_max), eigen-decomposed on the host, projections
    and transfer products on the GPU;
  * couplings (Eq. 18) S^{t,s} = V^{tH} A_t B_{t,s}^T conj(V^s), with B_t
    re-formed from the pivot rows of G^t (B_t = G^t[I, :]^T D_t), as GPU
    products whose kernel entries are generated inside the product;
  * near-field blocks delta_ts I - K^{t,s} diag(chi_s), generated on the GPU.
The result stays in device memory and is handed to h2_load_device, so the
H^2 data of a large geometry never crosses to the host.

Arithmetic: kernel entries with FP64 geometry and phase, FP32 after it; the
cross approximation, its Gram matrices and every projection product in FP32;
the Stage II Gram matrices with FP64 accumulation; the small factorisations
in FP64. The host constructor (FP64 throughout) and this one agree in every
rank on the test geometries (tests/test_gpu_construct.py).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import construct
from .construct import TWO_PI, _BlasThreads

_LIB = None

H2C_N, H2C_T, H2C_C, H2C_R = 0, 1, 2, 3


class _Vie(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("dv", ctypes.c_double), ("self_re", ctypes.c_double),
                ("self_im", ctypes.c_double)]


NEAR_DESC = np.dtype([("row_v0", "<i4"), ("row_nv", "<i4"), ("col_v0", "<i4"), ("col_nv", "<i4"),
                      ("out_off", "<i8"), ("diag", "<i4"), ("pad_", "<i4")])
ACA_JOB = np.dtype([("row_v0", "<i4"), ("row_nv", "<i4"), ("col_nv", "<i4"), ("kmax", "<i4"),
                    ("col_off", "<i8"), ("u_off", "<i8"), ("v_off", "<i8"), ("used_off", "<i8"),
                    ("piv_off", "<i8")])
GEMM_DESC = np.dtype([("A", "<u8"), ("B", "<u8"), ("C", "<u8"), ("m", "<i4"), ("n", "<i4"), ("k", "<i4"),
                      ("opa", "<i4"), ("opb", "<i4"), ("beta", "<i4"), ("lda", "<i8"), ("ldb", "<i8"),
                      ("ldc", "<i8"), ("alpha_re", "<f4"), ("alpha_im", "<f4")])
COUPLE_DESC = np.dtype([("Vs", "<u8"), ("piv", "<u8"), ("Q", "<u8"), ("ldv", "<i8"), ("ldq", "<i8"),
                        ("s_v0", "<i4"), ("s_nv", "<i4"), ("ks", "<i4"), ("kp", "<i4")])
assert NEAR_DESC.itemsize == 32 and ACA_JOB.itemsize == 56 and GEMM_DESC.itemsize == 80
assert COUPLE_DESC.itemsize == 56
ACA_KMAX = 4096


def lib():
    """libh2con.so (include/h2con.h); raises when it has not been built."""
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libh2con.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1703_01175_gb300.build.build_all()")
        L = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.h2c_near_blocks.argtypes = [vp, _Vie, vp, vp, i64, vp, vp]
        L.h2c_aca.argtypes = [vp, _Vie, vp, vp, i32, ctypes.c_float, vp, vp, vp, vp, vp, vp, vp, vp]
        L.h2c_gemm_grouped.argtypes = [vp, vp, vp, i64, i32, vp]
        L.h2c_couple_grouped.argtypes = [vp, _Vie, vp, vp, vp, i64, vp]
        L.h2c_sym_average.argtypes = [vp, vp, vp, vp, vp, i64, vp]
        for f in (L.h2c_near_blocks, L.h2c_aca, L.h2c_gemm_grouped, L.h2c_couple_grouped, L.h2c_sym_average):
            f.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


@dataclasses.dataclass
class DeviceH2:
    """H^2 arrays of the h2_data layout with the block arrays on the device
    (complex64 torch tensors) and the tree, CSR and offset arrays on the host."""
    n: int
    level_ptr: np.ndarray
    child: np.ndarray
    begin: np.ndarray
    size: np.ndarray
    rank: np.ndarray
    U: object
    U_off: np.ndarray
    W: object
    W_off: np.ndarray
    T: object
    T_off: np.ndarray
    adm_ptr: np.ndarray
    adm_col: np.ndarray
    S: object
    S_off: np.ndarray
    near_ptr: np.ndarray
    near_col: np.ndarray
    Z: object
    Z_off: np.ndarray
    perm: np.ndarray
    info: dict

    @property
    def nc(self) -> int:
        return int(self.size.shape[0])

    def device_bytes(self) -> int:
        return sum(int(x.numel()) * 8 for x in (self.U, self.W, self.T, self.S, self.Z))

    def to_host(self):
        """The same arrays with the blocks copied to host memory (an H2Arrays)."""
        from .h2 import H2Arrays
        blk = {k: getattr(self, k).cpu().numpy() for k in ("U", "W", "T", "S", "Z")}
        return H2Arrays(int(self.n), self.level_ptr, self.child, self.begin, self.size, self.rank,
                        blk["U"], self.U_off, blk["W"], self.W_off, blk["T"], self.T_off,
                        self.adm_ptr, self.adm_col, blk["S"], self.S_off, self.near_ptr, self.near_col,
                        blk["Z"], self.Z_off)

    def free(self):
        """Drop the device blocks (after h2_load_device has packed them)."""
        self.U = self.W = self.T = self.S = self.Z = None


class _Gpu:
    """Device memory, descriptor uploads and launches on one stream."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.stream = torch.cuda.current_stream(self.dev).cuda_stream
        self.L = lib()

    def up(self, arr: np.ndarray):
        """Upload a host array (any dtype) as raw bytes; returns the tensor."""
        t = self.torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).reshape(-1))
        return t.to(self.dev, non_blocking=False)

    def zeros_c64(self, n):
        return self.torch.zeros(max(int(n), 1), dtype=self.torch.complex64, device=self.dev)

    def empty_c64(self, n):
        return self.torch.empty(max(int(n), 1), dtype=self.torch.complex64, device=self.dev)

    def gemm(self, rows, out_f64=False):
        """Grouped products: rows of (A, B, C, m, n, k, opa, opb, beta, lda, ldb, ldc, alpha)."""
        rows = [r for r in rows if r[3] > 0 and r[4] > 0]
        if not rows:
            return
        d = np.zeros(len(rows), dtype=GEMM_DESC)
        a = np.array([(r[0], r[1], r[2]) for r in rows], dtype=np.uint64)
        d["A"], d["B"], d["C"] = a[:, 0], a[:, 1], a[:, 2]
        iv = np.array([r[3:12] for r in rows], dtype=np.int64)
        for i, f in enumerate(("m", "n", "k", "opa", "opb", "beta", "lda", "ldb", "ldc")):
            d[f] = iv[:, i]
        al = np.array([complex(r[12]) for r in rows])
        d["alpha_re"], d["alpha_im"] = al.real, al.imag
        tm = (d["m"].astype(np.int64) + 63) // 64
        tn = (d["n"].astype(np.int64) + 63) // 64
        cnt = tm * tn
        prob = np.repeat(np.arange(len(rows), dtype=np.int32), cnt)
        start = np.repeat(np.cumsum(cnt) - cnt, cnt)
        idx = (np.arange(int(cnt.sum()), dtype=np.int64) - start).astype(np.int32)
        dd, dp, di = self.up(d), self.up(prob), self.up(idx)
        _check(self.L.h2c_gemm_grouped(dd.data_ptr(), dp.data_ptr(), di.data_ptr(), len(prob), int(out_f64),
                                       self.stream), "h2c_gemm_grouped")
        self._keep = (dd, dp, di)

    def gemm_np(self, A, B, C, m, n, k, opa, opb, beta, lda, ldb, ldc, alpha=1.0, out_f64=False):
        """Grouped products from arrays (scalars broadcast), like gemm()."""
        cnt_ = np.broadcast(A, B, C, m, n, k, lda, ldb, ldc).shape
        nprob = cnt_[0] if cnt_ else 1
        d = np.zeros(nprob, dtype=GEMM_DESC)
        for f, v in (("A", A), ("B", B), ("C", C), ("m", m), ("n", n), ("k", k), ("opa", opa), ("opb", opb),
                     ("beta", beta), ("lda", lda), ("ldb", ldb), ("ldc", ldc)):
            d[f] = v
        d["alpha_re"], d["alpha_im"] = complex(alpha).real, complex(alpha).imag
        d = d[(d["m"] > 0) & (d["n"] > 0)]
        if len(d) == 0:
            return
        tm = (d["m"].astype(np.int64) + 63) // 64
        tn = (d["n"].astype(np.int64) + 63) // 64
        cnt = tm * tn
        prob = np.repeat(np.arange(len(d), dtype=np.int32), cnt)
        start = np.repeat(np.cumsum(cnt) - cnt, cnt)
        idx = (np.arange(int(cnt.sum()), dtype=np.int64) - start).astype(np.int32)
        dd, dp, di = self.up(d), self.up(prob), self.up(idx)
        _check(self.L.h2c_gemm_grouped(dd.data_ptr(), dp.data_ptr(), di.data_ptr(), len(prob), int(out_f64),
                                       self.stream), "h2c_gemm_grouped")
        self._keep = (dd, dp, di)

    def sync(self):
        self.torch.cuda.synchronize(self.dev)


def _ptr(t, elem_off=0, elem_bytes=8):
    return int(t.data_ptr()) + int(elem_off) * elem_bytes


def _trunc_eig_many(items, eps, pool, threads):
    """_trunc_eig for many Hermitian matrices: items is a list of (key, G);
    matrices of one size are stacked and decomposed in chunks across the host
    threads. Returns {key: eigenvectors with eigenvalue > eps^2 lambda_max}."""
    by_n = {}
    for key, G in items:
        by_n.setdefault(G.shape[0], []).append((key, G))
    chunks = []
    for n_, lst in by_n.items():
        step = max(4, -(-len(lst) // threads))
        chunks += [lst[c:c + step] for c in range(0, len(lst), step)]

    def run(lst):
        St = np.stack([G for _, G in lst])
        St = 0.5 * (St + np.conj(np.swapaxes(St, 1, 2)))
        w, Q = np.linalg.eigh(St)
        out = []
        for b, (key, _) in enumerate(lst):
            wb, Qb = w[b, ::-1], Q[b, :, ::-1]
            kk = 0 if wb.size == 0 or wb[0] <= 0.0 else int(np.count_nonzero(wb > eps * eps * wb[0]))
            out.append((key, np.ascontiguousarray(Qb[:, :kk])))
        return out

    with _BlasThreads(1):
        return dict(r for part in pool.map(run, chunks) for r in part)


def _reduced_svd_from_grams(Gu, Gv, eps):
    """Eq. 7 from the Gram matrices of the cross approximation's factors:
    U = Q_U R_U, V = Q_V R_V with R = Lambda^{1/2} E^H of each Gram matrix, the
    SVD R_U R_V^T = X Sigma Y^H truncated at sigma_i > eps sigma_1, so that
    A = U W_u with W_u = (E_u / lambda_u^{1/2}) X Sigma and B = V C with
    C = (E_v / lambda_v^{1/2}) conj(Y), B^T conj(B) = I. Returns (W_u, C)."""
    k = Gu.shape[0]
    du = np.sqrt(np.maximum(np.real(np.diag(Gu)), 0.0))
    dvv = np.sqrt(np.maximum(np.real(np.diag(Gv)), 0.0))
    if k == 0 or du.max() <= 0.0 or dvv.max() <= 0.0:
        return np.zeros((k, 0)), np.zeros((k, 0))
    su = np.where(du > 0, 1.0 / np.where(du > 0, du, 1.0), 0.0)
    sv = np.where(dvv > 0, 1.0 / np.where(dvv > 0, dvv, 1.0), 0.0)
    # Gram matrices of the column-normalised factors (FP32 products keep a
    # relative error per entry, so normalising after the product is exact)
    Gu_h = (Gu * su[:, None]) * su[None, :]
    Gv_h = (Gv * sv[:, None]) * sv[None, :]
    lu, Eu = np.linalg.eigh(0.5 * (Gu_h + Gu_h.conj().T))
    lv, Ev = np.linalg.eigh(0.5 * (Gv_h + Gv_h.conj().T))
    if lu[-1] <= 0.0 or lv[-1] <= 0.0:
        return np.zeros((k, 0)), np.zeros((k, 0))
    mu = lu > 1e-13 * lu[-1]
    mv = lv > 1e-13 * lv[-1]
    Eu, lu = Eu[:, mu], np.sqrt(lu[mu])
    Ev, lv = Ev[:, mv], np.sqrt(lv[mv])
    # factors of the unnormalised U = Uh diag(du): R_u = lambda^{1/2} E^H diag(du)
    Ru = (lu[:, None] * Eu.conj().T) * du[None, :]
    Rv = (lv[:, None] * Ev.conj().T) * dvv[None, :]
    X, s, Yh = np.linalg.svd(Ru @ Rv.T)
    kk = int(np.count_nonzero(s > eps * s[0]))
    Wu = su[:, None] * ((Eu / lu[None, :]) @ (X[:, :kk] * s[:kk]))
    C = sv[:, None] * ((Ev / lv[None, :]) @ Yh[:kk, :].T)
    return Wu, C


def _reduced_svd_stack(Gu, Gv, Lm, k, eps):
    """Eq. 7 for a stack of cross approximations padded to one size K.

    Gu, Gv: (B, K, K) Gram matrices U^H U and V^H V of the factors (the first
    k[b] rows and columns used); Lm: (B, K, K) lower-triangular pivot matrices
    (L_ll = pivot, L_lp = U[I_l, p]) of the cross approximations. With the
    Cholesky factors of the column-normalised Gram matrices, U = Q_U R_U and
    V = Q_V R_V (R = L^H diag(column norms)); the singular values and left
    vectors of M = R_U R_V^T come from the Hermitian eigenproblem of M M^H in
    FP64 (singular values above eps sigma_1, a relative threshold well inside
    FP64's range), and Y = M^H X Sigma^{-1}. Returns per b: W_u = R_U^{-1} X
    Sigma (A = U W_u) and D = L^{-T} R_V^{-1} conj(Y) (B_t = G^t[I, :]^T D),
    both k[b] x kk[b], or None for a matrix whose Cholesky factorisation fails
    (the caller then takes the eigen-decomposition route)."""
    B, K = Gu.shape[0], Gu.shape[1]
    pad = np.arange(K)[None, :] >= np.asarray(k)[:, None]          # (B, K): padded columns
    eye = np.eye(K)

    def factor(G):
        d = np.sqrt(np.maximum(np.real(np.diagonal(G, axis1=1, axis2=2)), 0.0))
        d = np.where(pad | (d <= 0.0), 1.0, d)
        Gh = G / d[:, :, None] / d[:, None, :]
        Gh = np.where(pad[:, :, None] | pad[:, None, :], 0.0, Gh) + pad[:, :, None] * eye[None]
        Gh = 0.5 * (Gh + np.conj(np.swapaxes(Gh, 1, 2)))
        ok = np.ones(B, dtype=bool)
        L = np.zeros_like(Gh)
        try:
            L = np.linalg.cholesky(Gh)
        except np.linalg.LinAlgError:
            for b in range(B):
                try:
                    L[b] = np.linalg.cholesky(Gh[b])
                except np.linalg.LinAlgError:
                    ok[b] = False
                    L[b] = eye
        R = np.conj(np.swapaxes(L, 1, 2)) * d[:, None, :]                 # upper triangular, identity padding
        return R, ok

    Ru, oku = factor(Gu)
    Rv, okv = factor(Gv)
    keep = ~pad
    Rum = Ru * keep[:, :, None]
    Rvm = Rv * keep[:, :, None]
    M = Rum @ np.swapaxes(Rvm, 1, 2)
    w, X = np.linalg.eigh(M @ np.conj(np.swapaxes(M, 1, 2)))
    w, X = w[:, ::-1], X[:, :, ::-1]
    sig = np.sqrt(np.maximum(w, 0.0))
    kk = np.array([int(np.count_nonzero(sig[b] > eps * sig[b, 0])) if sig[b, 0] > 0 else 0 for b in range(B)])
    inv = np.where(np.arange(K)[None, :] < kk[:, None], 1.0 / np.where(sig > 0, sig, 1.0), 0.0)
    Y = (np.conj(np.swapaxes(M, 1, 2)) @ X) * inv[:, None, :]
    Wu = np.linalg.solve(Ru, X * sig[:, None, :])
    C = np.linalg.solve(Rv, np.conj(Y))
    D = np.linalg.solve(np.swapaxes(Lm, 1, 2), C)
    out = []
    for b in range(B):
        if not (oku[b] and okv[b]):
            out.append(None)
        else:
            out.append((Wu[b, :k[b], :kk[b]], D[b, :k[b], :kk[b]]))
    return out


def build_vie_h2_gpu(centres, dv, eps_r, n_min=96, eta=1.0, eps=1e-4, k=TWO_PI, eps_aca=None,
                     eps_stage1=None, device=0, batch_bytes=None, threads=None, verbose=False) -> DeviceH2:
    """Build the H^2 arrays of Z = I - K diag(chi) for voxels at `centres` on
    GPU `device`. Returns a DeviceH2 in tree order (unknown 3 p + c is
    component c of the voxel at tree position p; perm maps tree positions to
    voxel indices)."""
    g = _Gpu(device)
    torch = g.torch
    t_all = time.time()
    secs = {}
    threads = threads or os.cpu_count() or 4
    eps_aca = eps / 10.0 if eps_aca is None else eps_aca
    eps_stage1 = eps / 3.0 if eps_stage1 is None else eps_stage1
    if batch_bytes is None:
        free, total = torch.cuda.mem_get_info(g.dev)
        batch_bytes = int(min(96e9, 0.4 * free))
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    chi_vox = np.asarray(eps_r, dtype=np.complex128) - 1.0
    a_eq = (3.0 * float(dv) / (4.0 * math.pi)) ** (1.0 / 3.0)
    ka = k * a_eq
    self_val = (2.0 / 3.0) * ((1.0 + 1j * ka) * np.exp(-1j * ka) - 1.0) - 1.0 / 3.0
    vie = _Vie(float(k), float(dv), float(self_val.real), float(self_val.imag))

    t0 = time.time()
    tr = construct.cluster_tree(centres, n_min)
    adm, near = construct.block_partition(tr, eta)
    secs["tree_partition"] = time.time() - t0
    nc = tr.nc
    vb = tr.vbegin.astype(np.int64)
    vs = tr.vsize.astype(np.int64)
    lev = tr.level.astype(np.int64)
    child = tr.child
    parent = tr.parent
    nlev = len(tr.level_ptr) - 1
    is_leaf = child[:, 0] < 0
    n = 3 * len(tr.perm)
    cen = torch.from_numpy(centres[tr.perm].reshape(-1)).to(g.dev)
    chi_t = torch.from_numpy(chi_vox[tr.perm].astype(np.complex64)).to(g.dev)
    partners = [[] for _ in range(nc)]
    for t, s in adm:
        partners[t].append(s)

    # ---- near field --------------------------------------------------------------
    t0 = time.time()
    near_t = np.array([p[0] for p in near], dtype=np.int64)
    near_s = np.array([p[1] for p in near], dtype=np.int64)
    zsz = 9 * vs[near_t] * vs[near_s]
    Z_off = np.concatenate([[0], np.cumsum(zsz)[:-1]]).astype(np.int64)
    Z = g.empty_c64(int(zsz.sum()))
    nd = np.zeros(len(near), dtype=NEAR_DESC)
    nd["row_v0"], nd["row_nv"] = vb[near_t], vs[near_t]
    nd["col_v0"], nd["col_nv"] = vb[near_s], vs[near_s]
    nd["out_off"], nd["diag"] = Z_off, (near_t == near_s)
    dnd = g.up(nd)
    _check(g.L.h2c_near_blocks(cen.data_ptr(), vie, chi_t.data_ptr(), dnd.data_ptr(), len(nd), Z.data_ptr(),
                               g.stream), "h2c_near_blocks")
    near_ptr = np.zeros(nc + 1, dtype=np.int64)
    np.add.at(near_ptr, near_t + 1, 1)
    near_ptr = np.cumsum(near_ptr).astype(np.int32)
    g.sync()
    del dnd
    secs["near"] = time.time() - t0

    # ---- Stage I: ACA of G^t per cluster, reduced SVD ------------------------------
    t0 = time.time()
    fac = {}        # t -> dict(A=tensor (kk x m, col-major), kk, kp, piv=int32 tensor, D=np (kp x kk))
    s1rank = {}
    fac_clusters = [t for t in range(nc) if partners[t]]
    by_level = {}
    for t in fac_clusters:
        by_level.setdefault(int(lev[t]), []).append(t)
    prev_max = 0
    pool = ThreadPoolExecutor(threads)
    tsub = {"aca_kernel": 0.0, "grams": 0.0, "host_svd": 0.0, "factor_gemm": 0.0, "prep": 0.0}
    for L_ in sorted(by_level, reverse=True):
        queue = []
        for t in by_level[L_]:
            m = 3 * int(vs[t])
            ncols = 3 * int(sum(vs[s] for s in partners[t]))
            cap = min(ACA_KMAX, m, ncols, max(128, 2 * prev_max + 32))
            queue.append((t, m, ncols, int(cap)))
        level_max = 0
        while queue:
            # one batch: jobs until the factor memory reaches batch_bytes
            queue.sort(key=lambda x: -(x[1] + x[2]) * x[3])
            batch, used_b = [], 0
            rest = []
            for job in queue:
                need = (job[1] + job[2]) * job[3] * 8 + job[1]
                if not batch or used_b + need <= batch_bytes:
                    batch.append(job)
                    used_b += need
                else:
                    rest.append(job)
            queue = rest
            nj = len(batch)
            jobs = np.zeros(nj, dtype=ACA_JOB)
            colv = []
            co = uo = vo = qo = po = 0
            for i, (t, m, ncols, cap) in enumerate(batch):
                cv = np.concatenate([np.arange(vb[s], vb[s] + vs[s]) for s in partners[t]]).astype(np.int32)
                colv.append(cv)
                jobs[i] = (vb[t], vs[t], ncols // 3, cap, co, uo, vo, qo, po)
                co += len(cv)
                uo += cap * m
                vo += cap * ncols
                qo += m
                po += cap
            tq = time.time()
            dcol = g.up(np.concatenate(colv))
            djobs = g.up(jobs)
            U = g.empty_c64(uo)
            V = g.empty_c64(vo)
            used = torch.empty(max(qo, 1), dtype=torch.uint8, device=g.dev)
            prow = torch.empty(max(po, 1), dtype=torch.int32, device=g.dev)
            pval = g.empty_c64(po)
            kout = torch.empty(nj, dtype=torch.int32, device=g.dev)
            stat = torch.empty(nj, dtype=torch.int32, device=g.dev)
            g.sync()
            tsub["prep"] += time.time() - tq
            tq = time.time()
            _check(g.L.h2c_aca(cen.data_ptr(), vie, dcol.data_ptr(), djobs.data_ptr(), nj, float(eps_aca),
                               U.data_ptr(), V.data_ptr(), used.data_ptr(), prow.data_ptr(), pval.data_ptr(),
                               kout.data_ptr(), stat.data_ptr(), g.stream), "h2c_aca")
            kk_h = kout.cpu().numpy()
            tsub["aca_kernel"] += time.time() - tq
            tq = time.time()
            st_h = stat.cpu().numpy()
            done = []
            for i, (t, m, ncols, cap) in enumerate(batch):
                if st_h[i] == 1 and cap < min(ACA_KMAX, m, ncols):
                    queue.append((t, m, ncols, int(min(ACA_KMAX, m, ncols, 2 * cap))))
                else:
                    done.append(i)
            # Gram matrices of the factors (FP32 products) and the pivot rows of U
            rows, goff, go = [], {}, 0
            for i in done:
                t, m, ncols, cap = batch[i]
                kp = int(kk_h[i])
                if kp == 0:
                    continue
                goff[i] = go
                go += 2 * kp * kp
            G = g.empty_c64(go)
            for i in goff:
                t, m, ncols, cap = batch[i]
                kp = int(kk_h[i])
                up_, vp_ = _ptr(U, jobs[i]["u_off"]), _ptr(V, jobs[i]["v_off"])
                rows.append((up_, up_, _ptr(G, goff[i]), kp, kp, m, H2C_C, H2C_N, 0, m, m, kp, 1.0))
                rows.append((vp_, vp_, _ptr(G, goff[i] + kp * kp), kp, kp, ncols, H2C_C, H2C_N, 0, ncols, ncols,
                             kp, 1.0))
            g.gemm(rows)
            prow_h = prow.cpu().numpy()
            pval_h = pval.cpu().numpy()
            # U[piv_row[a], l] for a, l < k'
            gidx, gpos, go2 = [], {}, 0
            for i in goff:
                kp = int(kk_h[i])
                m = batch[i][1]
                pr = prow_h[jobs[i]["piv_off"]:jobs[i]["piv_off"] + kp].astype(np.int64)
                gidx.append((jobs[i]["u_off"] + np.arange(kp)[None, :] * m + pr[:, None]).reshape(-1))
                gpos[i] = go2
                go2 += kp * kp
            Upiv = (U[torch.from_numpy(np.concatenate(gidx)).to(g.dev)].cpu().numpy() if gidx
                    else np.zeros(0, np.complex64))
            G_h = G.cpu().numpy()
            tsub["grams"] += time.time() - tq
            tq = time.time()

            # the reduced SVDs, stacked by padded size and split across host threads
            groups = {}
            for i in done:
                kp = int(kk_h[i])
                if kp > 0:
                    groups.setdefault((kp + 7) // 8 * 8, []).append(i)
            chunks = []
            for K_, idxs in groups.items():
                step = max(8, -(-len(idxs) // threads))
                chunks += [(K_, idxs[c:c + step]) for c in range(0, len(idxs), step)]

            def host_chunk(arg):
                K_, idxs = arg
                nb = len(idxs)
                Gu = np.zeros((nb, K_, K_), dtype=np.complex128)
                Gv = np.zeros((nb, K_, K_), dtype=np.complex128)
                Lm = np.tile(np.eye(K_, dtype=np.complex128), (nb, 1, 1))
                ks = np.zeros(nb, dtype=np.int64)
                prs = []
                for b_, i in enumerate(idxs):
                    kp = int(kk_h[i])
                    ks[b_] = kp
                    o = goff[i]
                    Gu[b_, :kp, :kp] = G_h[o:o + kp * kp].reshape(kp, kp, order="F")
                    Gv[b_, :kp, :kp] = G_h[o + kp * kp:o + 2 * kp * kp].reshape(kp, kp, order="F")
                    up = Upiv[gpos[i]:gpos[i] + kp * kp].reshape(kp, kp)
                    pv = pval_h[jobs[i]["piv_off"]:jobs[i]["piv_off"] + kp]
                    Lm[b_, :kp, :kp] = np.tril(up, -1) + np.diag(pv)
                    prs.append(prow_h[jobs[i]["piv_off"]:jobs[i]["piv_off"] + kp].astype(np.int64))
                out = _reduced_svd_stack(Gu, Gv, Lm, ks, eps_stage1)
                res_ = []
                for b_, i in enumerate(idxs):
                    kp = int(ks[b_])
                    if out[b_] is None:   # Cholesky failed: eigen-decomposition route
                        Wu, C = _reduced_svd_from_grams(Gu[b_, :kp, :kp], Gv[b_, :kp, :kp], eps_stage1)
                        D = np.linalg.solve(Lm[b_, :kp, :kp].T, C) if C.shape[1] else C
                    else:
                        Wu, D = out[b_]
                    res_.append((i, Wu, D, prs[b_]))
                return res_

            with _BlasThreads(1):
                res = [r for part in pool.map(host_chunk, chunks) for r in part]
            for i in done:
                if int(kk_h[i]) == 0:
                    s1rank[batch[i][0]] = (0, 0)
            tsub["host_svd"] += time.time() - tq
            tq = time.time()
            # A_t = U W_u, stored (kk x m) column-major, i.e. row-major m x kk
            rows = []
            for i, Wu, D, pr in res:
                t, m, ncols, cap = batch[i]
                kp = int(kk_h[i])
                kk = Wu.shape[1]
                s1rank[t] = (kp, kk)
                level_max = max(level_max, kp)
                if kk == 0:
                    continue
                Wd = torch.from_numpy(np.asfortranarray(Wu).astype(np.complex64).reshape(-1, order="F")).to(g.dev)
                A = g.empty_c64(kk * m)
                rows.append((_ptr(Wd), _ptr(U, jobs[i]["u_off"]), _ptr(A), kk, m, kp, H2C_T, H2C_T, 0, kp, m, kk,
                             1.0))
                piv_u = torch.from_numpy((3 * vb[t] + pr).astype(np.int32)).to(g.dev)
                fac[t] = {"A": A, "kk": kk, "kp": kp, "piv": piv_u, "D": D, "Wd": Wd}
            g.gemm(rows)
            g.sync()
            tsub["factor_gemm"] += time.time() - tq
            for t in fac:
                fac[t].pop("Wd", None)
            del U, V, used, prow, pval, G, dcol, djobs
            if verbose:
                print(f"construct_gpu:   batch of {nj} jobs (level {L_}), {used_b / 1e9:.1f} GB of factors, "
                      f"max rank {int(kk_h.max()) if nj else 0}; cumulative {tsub}", flush=True)
        prev_max = max(prev_max, level_max)
        if verbose:
            print(f"construct_gpu: stage I level {L_}: {len(by_level[L_])} clusters, max ACA rank {level_max}",
                  flush=True)
    secs["stage1"] = time.time() - t0
    secs.update({"stage1_" + k_: v_ for k_, v_ in tsub.items()})

    # ---- Stage II: bases and transfers, bottom-up ------------------------------------
    t0 = time.time()
    anc_f = []
    for t in range(nc):
        lst, a = [], t
        while a >= 0:
            if a in fac:
                lst.append(a)
            a = int(parent[a])
        anc_f.append(lst[::-1])          # root first: t itself (if any) last
    Kc = np.array([sum(fac[j]["kk"] for j in anc_f[t]) for t in range(nc)], dtype=np.int64)
    rank = np.zeros(nc, dtype=np.int64)
    Vleaf = {}        # leaf -> tensor (n_t x k_t col-major)
    Pm_dev = {}       # non-leaf -> tensor ((k1+k2) x k_t col-major): transfers of both children
    T_host = {}       # child -> (k_c x k_parent) complex128
    P = {}            # cluster -> tensor (k_t x K_t col-major)
    PT = {}           # cluster with fac -> tensor (k_t x kk_t)

    def col_off(t, j):
        o = 0
        for a in anc_f[t]:
            if a == j:
                return o
            o += fac[a]["kk"]
        raise KeyError(j)

    for L_ in range(nlev - 1, -1, -1):
        cl = list(range(int(tr.level_ptr[L_]), int(tr.level_ptr[L_ + 1])))
        leaves = [t for t in cl if is_leaf[t] and anc_f[t]]
        inner = [t for t in cl if not is_leaf[t]]
        # leaf Gram matrices G_(t) G_(t)^H = sum_j A_j|_t A_j|_t^H (Eq. 10), FP64 accumulation
        if leaves:
            nt = {t: 3 * int(vs[t]) for t in leaves}
            goff, go = {}, 0
            for t in leaves:
                goff[t] = go
                go += nt[t] ** 2
            G2 = torch.empty(max(go, 1), dtype=torch.complex128, device=g.dev)
            depth = max(len(anc_f[t]) for t in leaves)
            for idx in range(depth):
                rows = []
                for t in leaves:
                    if idx >= len(anc_f[t]):
                        continue
                    j = anc_f[t][idx]
                    kk = fac[j]["kk"]
                    r0 = 3 * int(vb[t] - vb[j])
                    X = _ptr(fac[j]["A"], r0 * kk)
                    beta = 1 if idx > 0 else 0
                    rows.append((X, X, _ptr(G2, goff[t], 16), nt[t], nt[t], kk, H2C_T, H2C_R, beta, kk, kk, nt[t],
                                 1.0))
                g.gemm(rows, out_f64=True)
            G2h = G2.cpu().numpy()
            del G2

            bases = _trunc_eig_many([(t, G2h[goff[t]:goff[t] + nt[t] ** 2].reshape(nt[t], nt[t], order="F"))
                                     for t in leaves], eps, pool, threads)
            res = [(t, bases[t]) for t in leaves]
            rows = []
            for t, Vt in res:
                rank[t] = Vt.shape[1]
                if rank[t] == 0:
                    continue
                Vd = torch.from_numpy(np.asfortranarray(Vt).astype(np.complex64).reshape(-1, order="F")).to(g.dev)
                Vleaf[t] = Vd
                kt = int(rank[t])
                Pt = g.empty_c64(kt * Kc[t])
                P[t] = Pt
                o = 0
                for j in anc_f[t]:
                    kk = fac[j]["kk"]
                    r0 = 3 * int(vb[t] - vb[j])
                    X = _ptr(fac[j]["A"], r0 * kk)
                    rows.append((_ptr(Vd), X, _ptr(Pt, o * kt), kt, kk, nt[t], H2C_C, H2C_T, 0, nt[t], kk, kt, 1.0))
                    o += kk
            g.gemm(rows)
        # projected Gram matrices of the non-leaf clusters (Eqs. 13-15), FP64 accumulation
        work = []
        for t in inner:
            c1, c2 = int(child[t, 0]), int(child[t, 1])
            k1, k2 = int(rank[c1]), int(rank[c2])
            if not anc_f[t] or k1 + k2 == 0 or Kc[t] == 0:
                T_host[c1] = np.zeros((k1, 0))
                T_host[c2] = np.zeros((k2, 0))
                continue
            work.append((t, c1, c2, k1, k2))
        if work:
            goff, go = {}, 0
            for w in work:
                goff[w[0]] = go
                go += (w[3] + w[4]) ** 2
            G2 = torch.empty(max(go, 1), dtype=torch.complex128, device=g.dev)
            rows = []
            for t, c1, c2, k1, k2 in work:
                K_ = int(Kc[t])
                ld = k1 + k2
                base = goff[t]
                blocks = [(c1, c1, 0, 0, k1, k1), (c1, c2, 0, k1, k1, k2), (c2, c1, k1, 0, k2, k1),
                          (c2, c2, k1, k1, k2, k2)]
                for a, b, ro, co_, mm, nn in blocks:
                    if mm == 0 or nn == 0:
                        continue
                    rows.append((_ptr(P[a]), _ptr(P[b]), _ptr(G2, base + ro + co_ * ld, 16), mm, nn, K_, H2C_N,
                                 H2C_C, 0, int(rank[a]), int(rank[b]), ld, 1.0))
            g.gemm(rows, out_f64=True)
            G2h = G2.cpu().numpy()
            del G2

            bases = _trunc_eig_many([(w_[0], G2h[goff[w_[0]]:goff[w_[0]] + (w_[3] + w_[4]) ** 2]
                                      .reshape(w_[3] + w_[4], w_[3] + w_[4], order="F")) for w_ in work],
                                    eps, pool, threads)
            res = [(w_, bases[w_[0]]) for w_ in work]
            rows1, rows2 = [], []
            for (t, c1, c2, k1, k2), Pm in res:
                kt = Pm.shape[1]
                rank[t] = kt
                T_host[c1] = Pm[:k1]
                T_host[c2] = Pm[k1:]
                if kt == 0:
                    continue
                Pd = torch.from_numpy(np.asfortranarray(Pm).astype(np.complex64).reshape(-1, order="F")).to(g.dev)
                Pm_dev[t] = Pd
                K_ = int(Kc[t])
                Pt = g.empty_c64(kt * K_)
                P[t] = Pt
                ld = k1 + k2
                if k1 > 0:
                    rows1.append((_ptr(Pd), _ptr(P[c1]), _ptr(Pt), kt, K_, k1, H2C_C, H2C_N, 0, ld, k1, kt, 1.0))
                if k2 > 0:
                    rows2.append((_ptr(Pd, k1), _ptr(P[c2]), _ptr(Pt), kt, K_, k2, H2C_C, H2C_N,
                                  1 if k1 > 0 else 0, ld, k2, kt, 1.0))
            g.gemm(rows1)
            g.gemm(rows2)
        g.sync()
        for t in cl:
            if t in fac and int(rank[t]) > 0:
                kt, kk = int(rank[t]), fac[t]["kk"]
                o = col_off(t, t)
                PT[t] = P[t][o * kt:(o + kk) * kt].clone()
        for t in inner:
            for c in child[t]:
                P.pop(int(c), None)
    P.clear()
    secs["stage2_bases"] = time.time() - t0
    if verbose:
        print(f"construct_gpu: stage II {secs['stage2_bases']:.1f} s, max rank {int(rank.max())}", flush=True)

    # ---- couplings (Eq. 18), level by level of the column cluster -------------------
    t0 = time.time()
    adm_t = np.array([p[0] for p in adm], dtype=np.int64)
    adm_s = np.array([p[1] for p in adm], dtype=np.int64)
    ssz = rank[adm_t] * rank[adm_s]
    S_off = np.concatenate([[0], np.cumsum(ssz)[:-1]]).astype(np.int64)
    S = g.zeros_c64(int(ssz.sum()))
    adm_ptr = np.zeros(nc + 1, dtype=np.int64)
    np.add.at(adm_ptr, adm_t + 1, 1)
    adm_ptr = np.cumsum(adm_ptr).astype(np.int32)
    # F_t = P_tt D_t^T (k_t x k'_t)
    F = {}
    rows = []
    for t in fac:
        kt = int(rank[t])
        if kt == 0:
            continue
        kp, kk = fac[t]["kp"], fac[t]["kk"]
        Dd = torch.from_numpy(np.asfortranarray(fac[t]["D"]).astype(np.complex64).reshape(-1, order="F")).to(g.dev)
        fac[t]["Dd"] = Dd
        F[t] = g.empty_c64(kt * kp)
        rows.append((_ptr(PT[t]), _ptr(Dd), _ptr(F[t]), kt, kp, kk, H2C_N, H2C_T, 0, kt, kp, kt, 1.0))
    g.gemm(rows)
    g.sync()
    for t in fac:
        fac[t].pop("Dd", None)
    kp_of = np.zeros(nc, dtype=np.int64)
    piv_ptr = np.zeros(nc, dtype=np.uint64)
    F_ptr = np.zeros(nc, dtype=np.uint64)
    for t in fac:
        kp_of[t] = fac[t]["kp"]
        piv_ptr[t] = fac[t]["piv"].data_ptr()
    for t, X_ in F.items():
        F_ptr[t] = X_.data_ptr()
    pairs_by_level = {}
    for j in range(len(adm)):
        t, s = int(adm_t[j]), int(adm_s[j])
        if rank[t] > 0 and rank[s] > 0:
            pairs_by_level.setdefault(int(lev[s]), []).append(j)
    cur_below = {}
    for L_ in range(nlev - 1, -1, -1):
        cl = list(range(int(tr.level_ptr[L_]), int(tr.level_ptr[L_ + 1])))
        cur = {}
        rows = []
        for c in cl:
            kc = int(rank[c])
            if kc == 0:
                continue
            if is_leaf[c]:
                cur[c] = Vleaf[c]
                continue
            c1, c2 = int(child[c, 0]), int(child[c, 1])
            n1, n2 = 3 * int(vs[c1]), 3 * int(vs[c2])
            k1, k2 = int(rank[c1]), int(rank[c2])
            X = g.zeros_c64((n1 + n2) * kc)
            cur[c] = X
            ld = k1 + k2
            if k1 > 0:
                rows.append((_ptr(cur_below[c1]), _ptr(Pm_dev[c]), _ptr(X), n1, kc, k1, H2C_N, H2C_N, 0, n1, ld,
                             n1 + n2, 1.0))
            if k2 > 0:
                rows.append((_ptr(cur_below[c2]), _ptr(Pm_dev[c], k1), _ptr(X, n1), n2, kc, k2, H2C_N, H2C_N, 0, n2,
                             ld, n1 + n2, 1.0))
        g.gemm(rows)
        plist = np.asarray(pairs_by_level.get(L_, []), dtype=np.int64)
        cur_ptr = np.zeros(nc, dtype=np.uint64)
        for c_, X_ in cur.items():
            cur_ptr[c_] = X_.data_ptr()
        # batches of pairs whose products Q fit in batch_bytes
        qsz = rank[adm_s[plist]] * kp_of[adm_t[plist]] if len(plist) else np.zeros(0, dtype=np.int64)
        cum = np.cumsum(8 * qsz)
        i0 = 0
        while i0 < len(plist):
            base = int(cum[i0 - 1]) if i0 else 0
            i1 = max(i0 + 1, int(np.searchsorted(cum, base + batch_bytes, side="right")))
            sel = plist[i0:i1]
            ts_, ss_ = adm_t[sel], adm_s[sel]
            qoff = np.concatenate([[0], np.cumsum(qsz[i0:i1])[:-1]]).astype(np.int64)
            Q = g.empty_c64(int(qsz[i0:i1].sum()))
            cd = np.zeros(len(sel), dtype=COUPLE_DESC)
            cd["Vs"], cd["piv"] = cur_ptr[ss_], piv_ptr[ts_]
            cd["Q"] = np.uint64(Q.data_ptr()) + (8 * qoff).astype(np.uint64)
            cd["ldv"], cd["ldq"] = 3 * vs[ss_], rank[ss_]
            cd["s_v0"], cd["s_nv"], cd["ks"], cd["kp"] = vb[ss_], vs[ss_], rank[ss_], kp_of[ts_]
            tm = (cd["ks"].astype(np.int64) + 63) // 64
            tn = (cd["kp"].astype(np.int64) + 63) // 64
            cnt = tm * tn
            prob = np.repeat(np.arange(len(sel), dtype=np.int32), cnt)
            start = np.repeat(np.cumsum(cnt) - cnt, cnt)
            tidx = (np.arange(int(cnt.sum()), dtype=np.int64) - start).astype(np.int32)
            dcd, dp, di = g.up(cd), g.up(prob), g.up(tidx)
            _check(g.L.h2c_couple_grouped(cen.data_ptr(), vie, dcd.data_ptr(), dp.data_ptr(), di.data_ptr(),
                                          len(prob), g.stream), "h2c_couple_grouped")
            # S^{t,s} = -F_t Q^T (the system matrix carries -K)
            g.gemm_np(F_ptr[ts_], cd["Q"], np.uint64(S.data_ptr()) + (8 * S_off[sel]).astype(np.uint64),
                      rank[ts_], rank[ss_], kp_of[ts_], H2C_N, H2C_T, 0, rank[ts_], rank[ss_], rank[ts_], alpha=-1.0)
            g.sync()
            del Q, dcd, dp, di
            i0 = i1
        cur_below = cur
    del cur_below, F, PT
    # S^{s,t} = (S^{t,s})^T exactly: the mean of the two skeleton estimates
    keys = adm_t * nc + adm_s                       # increasing: the pairs are sorted
    j_ts = np.nonzero((adm_t < adm_s) & (ssz > 0))[0]
    j_st = np.searchsorted(keys, adm_s[j_ts] * nc + adm_t[j_ts])
    assert np.array_equal(keys[j_st], adm_s[j_ts] * nc + adm_t[j_ts]), "partition is not symmetric"
    if len(j_ts):
        a = np.stack([j_ts, j_st], axis=1).astype(np.int64)
        sel = a
        d_ts, d_st = g.up(S_off[a[:, 0]]), g.up(S_off[a[:, 1]])
        d_kt = g.up(rank[adm_t[a[:, 0]]].astype(np.int32))
        d_ks = g.up(rank[adm_s[a[:, 0]]].astype(np.int32))
        _check(g.L.h2c_sym_average(S.data_ptr(), d_ts.data_ptr(), d_st.data_ptr(), d_kt.data_ptr(), d_ks.data_ptr(),
                                   len(sel), g.stream), "h2c_sym_average")
        g.sync()
    secs["couplings"] = time.time() - t0

    # ---- system-matrix bases -------------------------------------------------------------
    t0 = time.time()
    leaf_ids = [t for t in range(nc) if is_leaf[t] and rank[t] > 0]
    U_off = np.zeros(nc, dtype=np.int64)
    o = 0
    for t in leaf_ids:
        U_off[t] = o
        o += 3 * int(vs[t]) * int(rank[t])
    Uf = g.empty_c64(o)
    Wf = g.empty_c64(o)
    chi_u = chi_t.repeat_interleave(3)
    for t in leaf_ids:
        nt, kt = 3 * int(vs[t]), int(rank[t])
        Vt = Vleaf[t].view(kt, nt).t()          # (nt x kt) view of the column-major basis
        Uf[U_off[t]:U_off[t] + nt * kt] = Vleaf[t]
        Wf[U_off[t]:U_off[t] + nt * kt].view(kt, nt).copy_((chi_u[3 * vb[t]:3 * vb[t] + nt][:, None] * Vt).t())
    T_off = np.zeros(nc, dtype=np.int64)
    tparts, o = [], 0
    for c in range(1, nc):
        p = int(parent[c])
        if rank[c] > 0 and rank[p] > 0:
            T_off[c] = o
            tparts.append(np.asfortranarray(T_host[c]).astype(np.complex64).reshape(-1, order="F"))
            o += int(rank[c]) * int(rank[p])
    Tf = torch.from_numpy(np.concatenate(tparts) if tparts else np.zeros(1, np.complex64)).to(g.dev)
    g.sync()
    secs["bases"] = time.time() - t0
    pool.shutdown()
    secs["total"] = time.time() - t_all
    if verbose:
        print("construct_gpu:", {k_: round(v, 2) for k_, v in secs.items()}, flush=True)
    info = {"seconds": secs, "stage1_rank": s1rank, "n_adm": len(adm), "n_near": len(near)}
    return DeviceH2(n, tr.level_ptr.astype(np.int32), child.astype(np.int32).reshape(-1),
                    (3 * vb).astype(np.int32), (3 * vs).astype(np.int32), rank.astype(np.int32),
                    Uf, U_off, Wf, U_off.copy(), Tf, T_off, adm_ptr, adm_s.astype(np.int32), S, S_off,
                    near_ptr, near_s.astype(np.int32), Z, Z_off, tr.perm.copy(), info)
