"""The paper's complexity claims on one geometry family, at full size.

Sec. II.B and Sec. V.B: for a 1-D geometry (a rod, or a line of cubes) the
rank needed at a prescribed accuracy stays constant as the electric size
grows, so storage and the product cost grow linearly in N (Eqs. 19-22). The
series here is the line of 4^3-voxel dielectric cubes (pitch 0.5, eps_r 2.54)
with 512, 1024, 2048 and 4096 cubes (N = 98,304 ... 786,432), built on the GPU:

- the largest cluster rank does not grow with N (within max(2, 10 %));
- stored bytes per unknown stay flat (largest / smallest <= 1.25);
- the FP32 product time grows at most linearly (per-unknown time of the
  largest case within 1.3 x that of the 1024-cube case);
- the smallest case's product matches sampled rows of the dense VIE within
  10 eps (the representation error does not depend on the series).
"""
import json
import math

import numpy as np
import pytest

import synth
from oracle import vie

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

COUNTS = (512, 1024, 2048, 4096)


def _measure(name):
    from paper_1703_01175_gb300 import construct_gpu, h2
    w = synth.workload(name)
    v = w.voxels
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps)
    perm = dh.perm
    A = h2.H2Matrix.from_device(dh)
    dh.free()
    del dh
    torch.cuda.empty_cache()
    try:
        st = A.stats()
        n = st["n"]
        entries = st["near_elems"] + st["coupling_elems"] + 2 * st["transfer_elems"] + 2 * st["leaf_elems"]
        A.autotune()
        x = torch.from_numpy(synth.random_complex(n, 3).astype(np.complex64)).cuda()
        y = torch.empty_like(x)
        for _ in range(3):
            A.matvec(x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            A.matvec(x, y)
        e1.record()
        torch.cuda.synchronize()
        out = {"n": n, "max_rank": st["max_rank"], "bytes_per_unknown": 8.0 * entries / n,
               "us": e0.elapsed_time(e1) / 20 * 1e3}
        if name == f"array{COUNTS[0]}":
            # sampled rows against the dense VIE (natural order)
            rows = np.sort(np.random.default_rng(4).choice(n, 32, replace=False))
            unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
            x_np = x.cpu().numpy().astype(np.complex128)
            x_nat = np.empty_like(x_np)
            x_nat[unk] = x_np
            exact = vie.z_rows(v.centres, v.dv, v.eps_r, 2 * math.pi, unk[rows]) @ x_nat
            out["row_err"] = float(np.linalg.norm(y.cpu().numpy()[rows] - exact) / np.linalg.norm(exact))
        assert A.device_status() == 0
        return out
    finally:
        A.close()
        torch.cuda.empty_cache()


def test_line_of_cubes_scales_linearly():
    from paper_1703_01175_gb300 import build
    build.build_all()
    res = {c: _measure(f"array{c}") for c in COUNTS}
    print("1-D scaling series:", json.dumps(res))
    r0 = res[COUNTS[0]]["max_rank"]
    for c in COUNTS:
        assert res[c]["max_rank"] <= r0 + max(2, 0.1 * r0), res
    bpu = [res[c]["bytes_per_unknown"] for c in COUNTS]
    assert max(bpu) <= 1.25 * min(bpu), res
    assert res[4096]["us"] / res[4096]["n"] <= 1.3 * res[1024]["us"] / res[1024]["n"], res
    assert res[COUNTS[0]]["row_err"] <= 10 * 1e-4, res
