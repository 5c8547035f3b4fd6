"""The scratch-free product entry point (h2_matvec_noalloc), for callers that
must not call the CUDA allocator while running: its result must equal the
ordinary h2_matvec on the same operator and input, on consecutive calls (the
shared scratch array keeps the previous call's contents, so the second call
checks that it is cleared)."""
import ctypes

import numpy as np
import pytest

import cases
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_matvec():
    from paper_1703_01175_gb300 import build, h2
    build.build_all()
    L = h2.lib()
    L.h2_matvec_noalloc.restype = ctypes.c_int
    L.h2_matvec_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    A = h2.H2Matrix(cases.get("cube12").arrays())
    try:
        stream = torch.cuda.current_stream().cuda_stream
        for seed in (1, 2):
            x = torch.from_numpy(synth.random_complex(A.n, seed).astype(np.complex64)).cuda()
            y_ref = A.matvec(x)
            y = torch.full_like(x, complex(7.0, -3.0))
            st = L.h2_matvec_noalloc(A.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     ctypes.c_void_p(stream))
            assert st == 0, L.h2_last_error().decode()
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
            assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    finally:
        A.close()
