"""Host-side checks of the C ABI (no GPU needed).

- the shared library loads and exports every function include/h2.h declares;
- h2_load rejects malformed trees and partitions before touching the device.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import cases
from paper_1703_01175_gb300 import build
from paper_1703_01175_gb300 import h2 as h2py

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_all()


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(h2[a-z0-9_]*)\s*\(", txt)))


def test_exports_every_declared_symbol():
    L = h2py.lib()
    names = _declared("h2.h")
    assert names, "no declarations found"
    for name in names:
        assert hasattr(L, name), name
    assert set(h2py.exported_symbols()) <= set(names)


def test_status_strings():
    L = h2py.lib()
    for s in range(8):
        assert L.h2_status_string(s)


def _load_status(arrs):
    try:
        h2py.H2Matrix(arrs)
    except h2py.H2Error as e:
        return e.status, str(e)
    return 0, ""


def _fresh():
    return cases.get("ragged").arrays()


def test_valid_data_reaches_the_device_step():
    # without a GPU a valid representation fails only at the CUDA step
    st, msg = _load_status(_fresh())
    assert st in (0, h2py.H2_ERR_CUDA), msg


@pytest.mark.parametrize("mutate,needle", [
    (lambda a: a.rank.__setitem__(a.nc - 1, 10_000), "rank"),
    (lambda a: a.size.__setitem__(3, a.size[3] + 3), "tree"),
    (lambda a: a.child.__setitem__(0, a.nc + 5), "child"),
    (lambda a: a.near_col.__setitem__(0, 0), "near"),
    (lambda a: a.Z_off.__setitem__(1, a.Z.size), "Z block"),
    (lambda a: a.S_off.__setitem__(0, -4), "S block"),
    (lambda a: a.adm_col.__setitem__(2, a.adm_col[3]), "tile"),
    (lambda a: a.Z.__setitem__(7, np.nan), "non-finite"),
    (lambda a: a.level_ptr.__setitem__(1, 2), "level"),
])
def test_h2_load_rejects(mutate, needle):
    a = _fresh()
    mutate(a)
    st, msg = _load_status(a)
    assert st == h2py.H2_ERR_ARG, msg
    assert needle in msg


def test_null_arguments():
    L = h2py.lib()
    h = ctypes.c_void_p()
    assert L.h2_load(None, None, None, ctypes.byref(h)) == h2py.H2_ERR_ARG
    assert h.value is None
    assert L.h2_matvec(None, None, None, 1, 1, 0, None) == h2py.H2_ERR_ARG
    L.h2_free(None)
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    assert L.h2_sym_stats(None, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == h2py.H2_ERR_ARG
    assert L.h2_sym_near(None, None, 1) == h2py.H2_ERR_ARG
    assert L.h2_sym_near_stats(None, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == h2py.H2_ERR_ARG


def test_load_file_rejects_foreign_and_corrupted_files(tmp_path):
    """h2_load_file checks the header and the content hash before any device
    work, so these rejections need no GPU."""
    L = h2py.lib()
    h = ctypes.c_void_p()
    missing = tmp_path / "missing.h2"
    assert L.h2_load_file(str(missing).encode(), None, ctypes.byref(h)) == h2py.H2_ERR_ARG and not h.value
    junk = tmp_path / "junk.h2"
    junk.write_bytes(b"not an operator file at all" * 10)
    assert L.h2_load_file(str(junk).encode(), None, ctypes.byref(h)) == h2py.H2_ERR_ARG and not h.value
    # a correct header with a truncated body
    head = b"H2PACKED" + np.uint32(1).tobytes() + np.array([8, 15, 4], np.int32).tobytes() \
        + np.array([10, 64, 3, 3], np.int64).tobytes()
    trunc = tmp_path / "trunc.h2"
    trunc.write_bytes(head + b"\0" * 40)
    assert L.h2_load_file(str(trunc).encode(), None, ctypes.byref(h)) == h2py.H2_ERR_ARG and not h.value
    assert b"truncated or corrupted" in L.h2_last_error()
    with pytest.raises(h2py.H2Error):
        h2py.H2Matrix.from_file(str(junk))


def test_constructor_library_exports_every_declared_symbol():
    """libh2con.so (the GPU constructor kernels) loads on a host without a GPU
    and exports every function include/h2con.h declares."""
    from paper_1703_01175_gb300 import construct_gpu
    L = construct_gpu.lib()
    names = _declared("h2con.h")
    assert "h2c_aca" in names and "h2c_gemm_grouped" in names
    for name in names:
        assert hasattr(L, name), name
