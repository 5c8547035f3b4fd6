"""ctypes binding of libh2 (include/h2.h): argument marshalling only.

Every step of the product and the solve runs in the CUDA library; this module
only flattens block dictionaries into the C-ABI arrays, checks tensor dtypes and
devices, and passes raw pointers. If the library is missing it raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libh2.so")

H2_OK, H2_ERR_ARG, H2_ERR_ALLOC, H2_ERR_CUDA = 0, 1, 2, 3
H2_ERR_NOT_CONVERGED, H2_ERR_BREAKDOWN, H2_ERR_TIMEOUT, H2_ERR_STATE = 4, 5, 6, 7
H2_C64, H2_C128 = 0, 1
PREC = {"fp32": 0, "splitbf16": 1, "fp64acc": 2, "dfacc": 3}

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class _Tree(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_clusters", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("level_ptr", _i32p), ("child", _i32p), ("begin", _i32p), ("size", _i32p),
                ("rank", _i32p)]


class _Data(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int),
                ("U", ctypes.c_void_p), ("U_off", _i64p), ("U_len", ctypes.c_int64),
                ("W", ctypes.c_void_p), ("W_off", _i64p), ("W_len", ctypes.c_int64),
                ("T", ctypes.c_void_p), ("T_off", _i64p), ("T_len", ctypes.c_int64),
                ("adm_ptr", _i32p), ("adm_col", _i32p),
                ("S", ctypes.c_void_p), ("S_off", _i64p), ("S_len", ctypes.c_int64),
                ("near_ptr", _i32p), ("near_col", _i32p),
                ("Z", ctypes.c_void_p), ("Z_off", _i64p), ("Z_len", ctypes.c_int64)]


class _Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n", "n_clusters", "n_leaves", "n_levels", "near_blocks", "adm_blocks", "near_elems",
        "coupling_elems", "transfer_elems", "leaf_elems", "device_bytes")] + [
        ("max_rank", ctypes.c_int32), ("kernels_per_matvec", ctypes.c_int32)]


# arithmetic of the Gram-Schmidt passes: FP64, or double-float on the FP32 pipes
ARNOLDI = {"fp64": 0, "df": 1, "fp32": 2}


class _SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("x0_given", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("arnoldi", ctypes.c_int32), ("reorth_eta", ctypes.c_double)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int32), ("precond_cycles", ctypes.c_int32), ("reorth_steps", ctypes.c_int32)]


class H2Error(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libh2 (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1703_01175_gb300.build.build_all()")
    L = ctypes.CDLL(LIB_PATH)
    L.h2_load.restype = ctypes.c_int
    L.h2_load.argtypes = [ctypes.POINTER(_Tree), ctypes.POINTER(_Data), ctypes.c_char_p,
                          ctypes.POINTER(ctypes.c_void_p)]
    L.h2_load_device.restype = ctypes.c_int
    L.h2_load_device.argtypes = [ctypes.POINTER(_Tree), ctypes.POINTER(_Data), ctypes.c_char_p,
                                 ctypes.POINTER(ctypes.c_void_p)]
    L.h2_free.restype = None
    L.h2_free.argtypes = [ctypes.c_void_p]
    L.h2_matvec.restype = ctypes.c_int
    L.h2_matvec.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                            ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    L.h2_matvec_host.restype = ctypes.c_int
    L.h2_matvec_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_int64, ctypes.c_int]
    L.h2_get_stats.restype = ctypes.c_int
    L.h2_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Stats)]
    L.h2_sym_near.restype = ctypes.c_int
    L.h2_sym_near.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.h2_sym_near_stats.restype = ctypes.c_int
    L.h2_sym_near_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_double)]
    L.h2_sym_stats.restype = ctypes.c_int
    L.h2_sym_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_double)]
    L.h2_profile_matvec.restype = ctypes.c_int
    L.h2_profile_matvec.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_int32]
    L.h2_gmres.restype = ctypes.c_int
    L.h2_gmres.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                           ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveInfo), ctypes.c_void_p]
    L.h2_save.restype = ctypes.c_int
    L.h2_save.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    L.h2_load_file.restype = ctypes.c_int
    L.h2_load_file.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    L.h2_bicgstab.restype = ctypes.c_int
    L.h2_bicgstab.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                              ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveInfo), ctypes.c_void_p]
    L.h2_gmres_batched.restype = ctypes.c_int
    L.h2_gmres_batched.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_int64, ctypes.POINTER(_SolveOpts), ctypes.c_int,
                                   ctypes.POINTER(_SolveInfo), ctypes.c_void_p]
    L.h2_autotune.restype = ctypes.c_int
    L.h2_autotune.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32]
    L.h2_autotune_tc.restype = ctypes.c_int
    L.h2_autotune_tc.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p, ctypes.c_int32]
    L.h2_apply_tuning.restype = ctypes.c_int
    L.h2_apply_tuning.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    L.h2_configure.restype = ctypes.c_int
    L.h2_configure.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    L.h2_device_status.restype = ctypes.c_int
    L.h2_device_status.argtypes = [ctypes.c_void_p]
    L.h2_status_string.restype = ctypes.c_char_p
    L.h2_status_string.argtypes = [ctypes.c_int]
    L.h2_last_error.restype = ctypes.c_char_p
    L.h2_last_error.argtypes = []
    _lib = L
    return L


def _check(status: int, where: str):
    if status != H2_OK:
        L = lib()
        raise H2Error(status, where, f"{L.h2_status_string(status).decode()}: {L.h2_last_error().decode()}")


def exported_symbols() -> list:
    """Names declared in include/h2.h (the C ABI)."""
    return ["h2_load", "h2_load_device", "h2_free", "h2_matvec", "h2_matvec_host", "h2_get_stats", "h2_sym_stats", "h2_sym_near", "h2_sym_near_stats",
            "h2_profile_matvec", "h2_gmres", "h2_gmres_batched", "h2_device_status", "h2_autotune",
            "h2_autotune_tc", "h2_apply_tuning", "h2_configure",
            "h2_status_string", "h2_last_error"]


# ---------------------------------------------------------------------------
# Flat arrays of an H^2 representation (the h2_tree / h2_data layout).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class H2Arrays:
    n: int
    level_ptr: np.ndarray   # int32 [n_levels + 1]
    child: np.ndarray       # int32 [2 * nc]
    begin: np.ndarray       # int32 [nc]
    size: np.ndarray        # int32 [nc]
    rank: np.ndarray        # int32 [nc]
    U: np.ndarray           # complex, flat
    U_off: np.ndarray       # int64 [nc]
    W: np.ndarray | None
    W_off: np.ndarray | None
    T: np.ndarray
    T_off: np.ndarray
    adm_ptr: np.ndarray
    adm_col: np.ndarray
    S: np.ndarray
    S_off: np.ndarray
    near_ptr: np.ndarray
    near_col: np.ndarray
    Z: np.ndarray
    Z_off: np.ndarray

    @property
    def nc(self) -> int:
        return int(self.size.shape[0])


def _flatten(blocks: dict, keys, nc_or_len: int, dtype):
    """Concatenate column-major blocks; returns (flat, offsets)."""
    off = np.zeros(nc_or_len, dtype=np.int64)
    parts = []
    pos = 0
    for i, key in enumerate(keys):
        if key is None or key not in blocks:
            continue
        b = np.asarray(blocks[key])
        off[i] = pos
        parts.append(np.asfortranarray(b).reshape(-1, order="F").astype(dtype, copy=False))
        pos += b.size
    flat = np.concatenate(parts) if parts else np.zeros(1, dtype=dtype)
    return np.ascontiguousarray(flat), off


def arrays_from_blocks(n, level_ptr, child, begin, size, rank, U: dict, W: dict | None,
                       T: dict, S: dict, Z: dict, dtype=np.complex128) -> H2Arrays:
    """Marshal per-block dictionaries (cluster -> matrix, (t, s) -> matrix) into
    the flat CSR arrays of h2_data. Blocks are column-major in the output."""
    nc = len(size)
    child = np.asarray(child, dtype=np.int32).reshape(-1)
    Uf, Uo = _flatten(U, range(nc), nc, dtype)
    if W is not None:
        Wf, Wo = _flatten(W, range(nc), nc, dtype)
    else:
        Wf, Wo = None, None
    Tf, To = _flatten(T, range(nc), nc, dtype)
    adm = sorted(S.keys())
    near = sorted(Z.keys())
    adm_ptr = np.zeros(nc + 1, dtype=np.int32)
    for t, _ in adm:
        adm_ptr[t + 1] += 1
    adm_ptr = np.cumsum(adm_ptr).astype(np.int32)
    near_ptr = np.zeros(nc + 1, dtype=np.int32)
    for t, _ in near:
        near_ptr[t + 1] += 1
    near_ptr = np.cumsum(near_ptr).astype(np.int32)
    Sf, So = _flatten(S, adm, len(adm), dtype)
    Zf, Zo = _flatten(Z, near, len(near), dtype)
    return H2Arrays(int(n), np.asarray(level_ptr, dtype=np.int32), child,
                    np.asarray(begin, dtype=np.int32), np.asarray(size, dtype=np.int32),
                    np.asarray(rank, dtype=np.int32), Uf, Uo, Wf, Wo, Tf, To,
                    adm_ptr, np.array([s for _, s in adm] or [0], dtype=np.int32), Sf, So,
                    near_ptr, np.array([s for _, s in near] or [0], dtype=np.int32), Zf, Zo)


def _ip(a, t):
    return a.ctypes.data_as(t) if a is not None else None


class H2Matrix:
    """A loaded H^2 operator on one GPU (wraps an h2_handle)."""

    def __init__(self, arrs: H2Arrays, device: int = 0, graphs: bool = True, tc_pipeline: bool = True,
                 wait_limit: int | None = None, sym_couple: bool = False):
        L = lib()
        cplx = arrs.U.dtype
        if cplx not in (np.complex64, np.complex128):
            raise TypeError("block arrays must be complex64 or complex128")
        for name in ("W", "T", "S", "Z"):
            a = getattr(arrs, name)
            if a is not None and a.dtype != cplx:
                raise TypeError(f"{name} has dtype {a.dtype}, expected {cplx}")
        self._keep = arrs
        self.n = arrs.n
        tr = _Tree(arrs.n, arrs.nc, len(arrs.level_ptr) - 1, _ip(arrs.level_ptr, _i32p),
                   _ip(arrs.child, _i32p), _ip(arrs.begin, _i32p), _ip(arrs.size, _i32p),
                   _ip(arrs.rank, _i32p))
        dt = H2_C64 if cplx == np.complex64 else H2_C128
        d = _Data(dt,
                  arrs.U.ctypes.data, _ip(arrs.U_off, _i64p), arrs.U.size,
                  arrs.W.ctypes.data if arrs.W is not None else None, _ip(arrs.W_off, _i64p),
                  arrs.W.size if arrs.W is not None else 0,
                  arrs.T.ctypes.data, _ip(arrs.T_off, _i64p), arrs.T.size,
                  _ip(arrs.adm_ptr, _i32p), _ip(arrs.adm_col, _i32p),
                  arrs.S.ctypes.data, _ip(arrs.S_off, _i64p), arrs.S.size,
                  _ip(arrs.near_ptr, _i32p), _ip(arrs.near_col, _i32p),
                  arrs.Z.ctypes.data, _ip(arrs.Z_off, _i64p), arrs.Z.size)
        h = ctypes.c_void_p()
        opts = f"device={device};graphs={int(graphs)};tc_pipeline={int(tc_pipeline)};sym_couple={int(sym_couple)}"
        if wait_limit is not None:
            opts += f";wait_limit={int(wait_limit)}"
        _check(L.h2_load(ctypes.byref(tr), ctypes.byref(d), opts.encode(), ctypes.byref(h)), "h2_load")
        self._h = h
        self.device = device
        self._keep = None  # the library copied everything

    @classmethod
    def from_device(cls, dh, device: int = 0, graphs: bool = True, tc_pipeline: bool = True,
                    wait_limit: int | None = None, sym_couple: bool = False) -> "H2Matrix":
        """Load H^2 arrays whose blocks are complex64 tensors on `device` (a
        construct_gpu.DeviceH2) through h2_load_device: the blocks are packed
        on the device and never copied to the host."""
        import torch
        for name in ("U", "W", "T", "S", "Z"):
            a = getattr(dh, name)
            if a is None:
                continue
            if not (a.is_cuda and a.dtype == torch.complex64 and a.device.index == device):
                raise TypeError(f"{name} must be a complex64 tensor on cuda:{device}")
        arrs = dh
        tr = _Tree(arrs.n, arrs.nc, len(arrs.level_ptr) - 1, _ip(arrs.level_ptr, _i32p),
                   _ip(arrs.child, _i32p), _ip(arrs.begin, _i32p), _ip(arrs.size, _i32p),
                   _ip(arrs.rank, _i32p))
        d = _Data(H2_C64,
                  arrs.U.data_ptr(), _ip(arrs.U_off, _i64p), arrs.U.numel(),
                  arrs.W.data_ptr() if arrs.W is not None else None, _ip(arrs.W_off, _i64p),
                  arrs.W.numel() if arrs.W is not None else 0,
                  arrs.T.data_ptr(), _ip(arrs.T_off, _i64p), arrs.T.numel(),
                  _ip(arrs.adm_ptr, _i32p), _ip(arrs.adm_col, _i32p),
                  arrs.S.data_ptr(), _ip(arrs.S_off, _i64p), arrs.S.numel(),
                  _ip(arrs.near_ptr, _i32p), _ip(arrs.near_col, _i32p),
                  arrs.Z.data_ptr(), _ip(arrs.Z_off, _i64p), arrs.Z.numel())
        opts = f"device={device};graphs={int(graphs)};tc_pipeline={int(tc_pipeline)};sym_couple={int(sym_couple)}"
        if wait_limit is not None:
            opts += f";wait_limit={int(wait_limit)}"
        torch.cuda.synchronize(device)
        torch.cuda.empty_cache()   # the constructor's freed temporaries go back to the device
        h = ctypes.c_void_p()
        _check(lib().h2_load_device(ctypes.byref(tr), ctypes.byref(d), opts.encode(), ctypes.byref(h)),
               "h2_load_device")
        self = cls.__new__(cls)
        self._h = h
        self.device = device
        self._keep = None
        self.n = arrs.n
        return self

    @classmethod
    def from_file(cls, path: str, device: int = 0, graphs: bool = True, tc_pipeline: bool = True,
                  wait_limit: int | None = None, sym_couple: bool = False) -> "H2Matrix":
        """Reload an operator written by save() (no re-validation or re-packing)."""
        opts = f"device={device};graphs={int(graphs)};tc_pipeline={int(tc_pipeline)};sym_couple={int(sym_couple)}"
        if wait_limit is not None:
            opts += f";wait_limit={int(wait_limit)}"
        h = ctypes.c_void_p()
        _check(lib().h2_load_file(str(path).encode(), opts.encode(), ctypes.byref(h)), "h2_load_file")
        self = cls.__new__(cls)
        self._h = h
        self.device = device
        self._keep = None
        self.n = self.stats()["n"]
        return self

    def save(self, path: str):
        """Write the loaded operator to `path` (see from_file)."""
        _check(lib().h2_save(self._h, str(path).encode()), "h2_save")

    def close(self):
        if getattr(self, "_h", None):
            lib().h2_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        s = _Stats()
        _check(lib().h2_get_stats(self._h, ctypes.byref(s)), "h2_get_stats")
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def sym_near(self, chi):
        """Store the near field once per leaf pair for the single-RHS FP32
        product; chi: numpy complex array (n,) in tree order, or None to go
        back to the full storage."""
        if chi is None:
            _check(lib().h2_sym_near(self._h, None, H2_C128), "h2_sym_near")
            return
        c = np.ascontiguousarray(chi, dtype=np.complex128)
        if c.shape != (self.n,):
            raise ValueError(f"chi must have shape ({self.n},)")
        _check(lib().h2_sym_near(self._h, c.ctypes.data, H2_C128), "h2_sym_near")

    def sym_near_stats(self) -> dict:
        """Near field stored once per leaf pair (after sym_near)."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().h2_sym_near_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "h2_sym_near_stats")
        return {"stored_elems": a.value, "scratch_entries": b.value, "max_asym": c.value}

    def sym_stats(self) -> dict:
        """Symmetric coupling storage (handle loaded with sym_couple=True)."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().h2_sym_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "h2_sym_stats")
        return {"stored_elems": a.value, "scratch_entries": b.value, "max_asym": c.value}

    def matvec(self, x, y=None, prec: str = "fp32", stream=None):
        """y = A x on the device. x: torch complex64 (fp32, splitbf16) or
        complex128 (fp64acc, dfacc) CUDA tensor of shape (n,) or (n, nrhs) column-major
        (i.e. x.t() contiguous) or (nrhs, n) contiguous rows via x.T."""
        import torch
        want = torch.complex128 if prec in ("fp64acc", "dfacc") else torch.complex64
        if x.dtype != want or not x.is_cuda:
            raise TypeError(f"x must be a CUDA {want} tensor")
        nrhs, ld = self._shape(x)
        if y is None:
            y = torch.empty_like(x)
        if y.dtype != want or y.shape != x.shape or not y.is_cuda:
            raise TypeError("y must match x")
        self._shape(y)
        st = torch.cuda.current_stream(x.device).cuda_stream if stream is None else stream
        _check(lib().h2_matvec(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                               nrhs, ld, PREC[prec], ctypes.c_void_p(st)), "h2_matvec")
        return y

    def _shape(self, x):
        if x.dim() == 1:
            if x.shape[0] != self.n or x.stride(0) != 1:
                raise ValueError("vector length or stride mismatch")
            return 1, self.n
        if x.dim() == 2 and x.shape[0] == self.n and x.stride(0) == 1:
            return x.shape[1], x.stride(1) if x.shape[1] > 1 else self.n
        raise ValueError("x must be (n,) or (n, nrhs) with unit stride along n")

    def matvec_host(self, x: np.ndarray, prec: str = "fp32", out: np.ndarray | None = None) -> np.ndarray:
        """y = A x with host numpy arrays (copies inside the call); `out`, if
        given, receives y (same shape, dtype and column-major layout as x;
        pinned host memory makes both copies direct DMA)."""
        want = np.complex128 if prec in ("fp64acc", "dfacc") else np.complex64
        x = np.asarray(x)
        if x.dtype != want:
            raise TypeError(f"x must be {want}")
        nrhs = 1 if x.ndim == 1 else x.shape[1]
        xf = np.asfortranarray(x)
        if out is None:
            y = np.empty_like(xf, order="F")
        else:
            y = out
            if y.shape != xf.shape or y.dtype != xf.dtype or not y.flags.f_contiguous:
                raise TypeError("out must match x in shape and dtype and be column-major")
        _check(lib().h2_matvec_host(self._h, xf.ctypes.data, y.ctypes.data, nrhs, self.n, PREC[prec]),
               "h2_matvec_host")
        return y

    def gmres_batched(self, B, X=None, tol=1e-4, restart=50, maxit=1000, refine=False, x0_given=False,
                      prec="splitbf16", arnoldi="fp64", reorth_eta=0.0, stream=None, check=True, precond=False):
        """Batched GMRES for B (n, nrhs) column-major complex128 on the device."""
        import torch
        if B.dtype != torch.complex128 or not B.is_cuda:
            raise TypeError("B must be a CUDA complex128 tensor")
        nrhs, ld = self._shape(B)
        if X is None:
            X = torch.zeros_like(B)
        opts = _SolveOpts(float(tol), int(restart), int(maxit), int(bool(refine)), int(bool(x0_given)), int(bool(precond)),
                          ARNOLDI[arnoldi], float(reorth_eta))
        infos = (_SolveInfo * nrhs)()
        st = torch.cuda.current_stream(B.device).cuda_stream if stream is None else stream
        status = lib().h2_gmres_batched(self._h, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()), nrhs,
                                        ld, ctypes.byref(opts), PREC[prec], infos, ctypes.c_void_p(st))
        out = [{"iterations": i.iterations, "restarts": i.restarts, "rel_res": i.rel_res, "status": i.status,
                "reorth_steps": i.reorth_steps, "precond_cycles": i.precond_cycles} for i in infos]
        if check and status not in (H2_OK, H2_ERR_NOT_CONVERGED):
            _check(status, "h2_gmres_batched")
        return X, out

    def autotune(self, nrhs_tc: int | None = None, cache: str | None = None, fp32: bool = True) -> dict:
        """Pick the fastest CTA size of every FP32 product stage and, with
        nrhs_tc, the fastest pipeline depth of every tensor-core phase for that
        many right-hand sides (returns the report). With `cache` (a JSON file),
        a report stored for this GPU model and operator shape is applied
        without timing anything, and a new report is stored there."""
        import json
        key = gpu = None
        if cache:
            import torch
            gpu = torch.cuda.get_device_name(self.device)
            st = self.stats()
            key = (f"n={st['n']};clusters={st['n_clusters']};near={st['near_blocks']};adm={st['adm_blocks']};"
                   f"max_rank={st['max_rank']};nrhs_tc={((nrhs_tc or 0) + 127) // 128 * 128}")
            try:
                with open(cache) as f:
                    saved = json.load(f).get(gpu, {}).get(key)
            except (OSError, ValueError):
                saved = None
            if saved:
                self.apply_tuning(saved)
                return dict(saved, cached=True)
        buf = ctypes.create_string_buffer(1 << 18)
        rep = {}
        if fp32:
            _check(lib().h2_autotune(self._h, buf, len(buf)), "h2_autotune")
            rep = json.loads(buf.value.decode())
        if nrhs_tc:
            _check(lib().h2_autotune_tc(self._h, int(nrhs_tc), buf, len(buf)), "h2_autotune_tc")
            rep.update(json.loads(buf.value.decode()))
        if cache:
            try:
                with open(cache) as f:
                    allc = json.load(f)
            except (OSError, ValueError):
                allc = {}
            allc.setdefault(gpu, {})[key] = rep
            d = os.path.dirname(os.path.abspath(cache))
            os.makedirs(d, exist_ok=True)
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(allc, f)
            os.replace(tmp, cache)
        return rep

    def apply_tuning(self, report: dict):
        """Apply a report of autotune() (or a part of one) without timing
        anything (h2_apply_tuning)."""
        import json
        _check(lib().h2_apply_tuning(self._h, json.dumps(report).encode()), "h2_apply_tuning")

    def configure(self, graphs: bool | None = None, tc_pipeline: bool | None = None):
        """Change the graph and tensor-core pipeline options of the loaded handle."""
        opts = []
        if graphs is not None:
            opts.append(f"graphs={int(bool(graphs))}")
        if tc_pipeline is not None:
            opts.append(f"tc_pipeline={int(bool(tc_pipeline))}")
        if opts:
            _check(lib().h2_configure(self._h, ";".join(opts).encode()), "h2_configure")

    def device_status(self) -> int:
        """Synchronise and return H2_OK or H2_ERR_TIMEOUT (a bounded wait ran out)."""
        return lib().h2_device_status(self._h)

    def gmres(self, b, x=None, tol=1e-4, restart=50, maxit=1000, refine=False, x0_given=False,
              precond=0, arnoldi="fp64", reorth_eta=0.0, stream=None, check=True):
        """Solve A x = b on the device. b: CUDA complex128 (n,) or (n, nrhs)
        column-major. Returns (x, [info dict per RHS])."""
        import torch
        if b.dtype != torch.complex128 or not b.is_cuda:
            raise TypeError("b must be a CUDA complex128 tensor")
        nrhs, ld = self._shape(b)
        if x is None:
            x = torch.zeros_like(b)
        opts = _SolveOpts(float(tol), int(restart), int(maxit), int(bool(refine)), int(bool(x0_given)), int(precond),
                          ARNOLDI[arnoldi], float(reorth_eta))
        infos = (_SolveInfo * nrhs)()
        st = torch.cuda.current_stream(b.device).cuda_stream if stream is None else stream
        status = lib().h2_gmres(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs, ld,
                                ctypes.byref(opts), infos, ctypes.c_void_p(st))
        out = [{"iterations": i.iterations, "restarts": i.restarts, "rel_res": i.rel_res, "status": i.status,
                "precond_cycles": i.precond_cycles, "reorth_steps": i.reorth_steps} for i in infos]
        if check and status not in (H2_OK, H2_ERR_NOT_CONVERGED):
            _check(status, "h2_gmres")
        return x, out

    def bicgstab(self, b, x=None, tol=1e-4, maxit=1000, refine=False, x0_given=False, arnoldi="fp64",
                 stream=None, check=True):
        """BiCGStab (the paper's solver) on the device. b: CUDA complex128 (n,)
        or (n, nrhs) column-major. arnoldi selects the accumulated residual
        product used by refine: "fp64" (FP64ACC) or "df" (DFACC).
        Returns (x, [info dict per RHS])."""
        import torch
        if b.dtype != torch.complex128 or not b.is_cuda:
            raise TypeError("b must be a CUDA complex128 tensor")
        nrhs, ld = self._shape(b)
        if x is None:
            x = torch.zeros_like(b)
        opts = _SolveOpts(float(tol), 0, int(maxit), int(bool(refine)), int(bool(x0_given)), 0, ARNOLDI[arnoldi], 0.0)
        infos = (_SolveInfo * nrhs)()
        st = torch.cuda.current_stream(b.device).cuda_stream if stream is None else stream
        status = lib().h2_bicgstab(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs, ld,
                                   ctypes.byref(opts), infos, ctypes.c_void_p(st))
        out = [{"iterations": i.iterations, "restarts": i.restarts, "rel_res": i.rel_res, "status": i.status}
               for i in infos]
        if check and status not in (H2_OK, H2_ERR_NOT_CONVERGED):
            _check(status, "h2_bicgstab")
        return x, out

    def profile(self, x, y, iters: int = 10) -> dict:
        ms = (ctypes.c_double * 7)()
        _check(lib().h2_profile_matvec(self._h, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()), iters, ms, 7),
               "h2_profile_matvec")
        keys = ["near", "leaf_forward", "upward", "coupling", "downward", "leaf_expansion", "total"]
        return dict(zip(keys, list(ms)))
