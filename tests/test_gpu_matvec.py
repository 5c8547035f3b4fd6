"""Parity of the CUDA H^2 product with the FP64 oracle on the same H^2 data.

Bar: FP32 product within 1e-5 relative (2-norm) of the oracle's FP64 product,
and element by element within 1e-5 of the largest output entry; the FP64-
accumulated product (FP32-stored data) within 1e-6. Cases span several leaf
tiles, ragged (non power of two) trees, odd ranks, leaves of one voxel, a
single-leaf tree (no admissible blocks), slab and 1-D array geometries.
"""
import numpy as np
import pytest

import cases
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = ["cube8", "ragged", "cube12", "slab", "array", "single_leaf", "tiny_leaves", "odd"]


@pytest.fixture(scope="module")
def loaded():
    from paper_1703_01175_gb300 import build, h2
    build.build_all()
    out = {}
    yield out
    for m in out.values():
        m.close()


def _mat(loaded, name, symmetric=False, dtype=np.complex128, tc_pipeline=True):
    from paper_1703_01175_gb300 import h2
    key = (name, symmetric, dtype, tc_pipeline)
    if key not in loaded:
        loaded[key] = h2.H2Matrix(cases.get(name).arrays(dtype=dtype, symmetric=symmetric), tc_pipeline=tc_pipeline)
    return loaded[key]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", CASES)
def test_fp32_matches_oracle(loaded, name):
    c = cases.get(name)
    A = _mat(loaded, name)
    for seed in (1, 2):
        x = synth.random_complex(c.n, seed)
        y_or = c.oracle_matvec(x)
        xd = torch.from_numpy(x.astype(np.complex64)).cuda()
        y = A.matvec(xd).cpu().numpy().astype(np.complex128)
        assert _rel(y, y_or) <= 1e-5
        assert np.abs(y - y_or).max() <= 1e-5 * np.abs(y_or).max()


@pytest.mark.parametrize("name", ["cube8", "ragged", "cube12"])
def test_fp64acc_matches_oracle(loaded, name):
    c = cases.get(name)
    A = _mat(loaded, name)
    x = synth.random_complex(c.n, 3)
    y_or = c.oracle_matvec(x)
    y = A.matvec(torch.from_numpy(x).cuda(), prec="fp64acc").cpu().numpy()
    assert _rel(y, y_or) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64acc", "dfacc"])
@pytest.mark.parametrize("name", ["cube8", "cube12"])
def test_accumulation_exact_on_stored_data(loaded, name, prec):
    """FP64 and double-float accumulation reproduce the FP64 product of the
    FP32-stored data to 1e-12 (FP32 accumulation would be off by ~1e-7)."""
    c = cases.get(name)
    A = _mat(loaded, name)
    x = synth.random_complex(c.n, 5)
    y_ex = c.oracle_matvec_stored(x)
    y = A.matvec(torch.from_numpy(x).cuda(), prec=prec).cpu().numpy()
    assert _rel(y, y_ex) <= 1e-12


def test_c64_input_and_symmetric_form(loaded):
    c = cases.get("cube8")
    x = synth.random_complex(c.n, 4)
    # symmetric form W = U represents K-type data; compare with the oracle on the same data
    A = _mat(loaded, "cube8", symmetric=True, dtype=np.complex64)
    from oracle.h2build import H2
    from oracle import h2mv
    hs = H2(c.tree, c.part, c.hZ.rank, c.hZ.U, None, c.hZ.T, c.hZ.S, c.hZ.Z)
    y_or = h2mv.h2_matvec(hs, x)
    y = A.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert _rel(y, y_or) <= 1e-5


def test_multiple_rhs_and_host_entry(loaded):
    c = cases.get("ragged")
    A = _mat(loaded, "ragged")
    X = synth.random_complex(c.n, 5, cols=3)
    Y_or = c.oracle_matvec(X)
    Xd = torch.from_numpy(np.asfortranarray(X.astype(np.complex64))).cuda()
    Xd = Xd.t().contiguous().t()  # column-major (n, 3)
    Y = A.matvec(Xd).cpu().numpy()
    assert _rel(Y, Y_or) <= 1e-5
    Yh = A.matvec_host(X.astype(np.complex64))
    assert _rel(Yh, Y_or) <= 1e-5


def test_zero_vector_and_repeat_determinism(loaded):
    c = cases.get("cube12")
    A = _mat(loaded, "cube12")
    z = torch.zeros(c.n, dtype=torch.complex64, device="cuda")
    assert torch.count_nonzero(A.matvec(z)).item() == 0
    x = torch.from_numpy(synth.random_complex(c.n, 9).astype(np.complex64)).cuda()
    y1 = A.matvec(x).clone()
    y2 = A.matvec(x)
    assert torch.equal(y1, y2)  # row-owned reductions: bitwise reproducible


def _colmajor(X):
    return torch.from_numpy(np.asfortranarray(X.astype(np.complex64))).cuda().t().contiguous().t()


@pytest.mark.parametrize("name,R", [("cube12", 33), ("ragged", 2), ("slab", 40), ("cube12", 97), ("ragged", 200)])
def test_multi_rhs_fp32_matches_oracle(loaded, name, R):
    from oracle import h2mv
    c = cases.get(name)
    A = _mat(loaded, name)
    X = synth.random_complex(c.n, 11, cols=R)
    Y_or = h2mv.h2_dense(c.hZ) @ X
    Y = A.matvec(_colmajor(X)).cpu().numpy()
    assert _rel(Y, Y_or) <= 1e-5
    for j in (0, R - 1):
        assert np.linalg.norm(Y[:, j] - Y_or[:, j]) <= 1e-5 * np.linalg.norm(Y_or[:, j])


@pytest.mark.parametrize("pipeline", [True, False])
@pytest.mark.parametrize("name,R", [("cube12", 128), ("cube12", 5), ("ragged", 130), ("slab", 64),
                                    ("array", 17), ("tiny_leaves", 3), ("odd", 7)])
def test_splitbf16_tensor_cores_match_oracle(loaded, name, R, pipeline):
    """Split-bf16 tcgen05 path (deepest pipeline and two stages): within
    eps = 1e-4 of the oracle's FP64 product
    (the accuracy stated for the lower-precision form)."""
    from oracle import h2mv
    c = cases.get(name)
    A = _mat(loaded, name, tc_pipeline=pipeline)
    X = synth.random_complex(c.n, 12, cols=R)
    Y_or = h2mv.h2_dense(c.hZ) @ X
    for rep in range(2):
        Y = A.matvec(_colmajor(X), prec="splitbf16").cpu().numpy()
        assert A.device_status() == 0
        assert _rel(Y, Y_or) <= 1e-4
        colerr = np.linalg.norm(Y - Y_or, axis=0) / np.linalg.norm(Y_or, axis=0)
        assert colerr.max() <= 1e-4


def test_splitbf16_packed_and_wide_layouts_alternate(loaded):
    """At most 64 right-hand sides use the packed plane layout (real and
    imaginary parts in the two halves of one 128-lane tile), more use the
    128-wide one; alternating them on one handle (32, 128, 32, 100, 1) keeps
    every product within eps of the oracle, and the packed columns agree with
    the same columns of a wide product within eps."""
    from oracle import h2mv
    c = cases.get("cube12")
    A = _mat(loaded, "cube12")
    X = synth.random_complex(c.n, 15, cols=128)
    Y_or = h2mv.h2_dense(c.hZ) @ X
    wide = None
    for R in (32, 128, 32, 100, 1):
        Y = A.matvec(_colmajor(X[:, :R]), prec="splitbf16").cpu().numpy().reshape(c.n, R)
        assert A.device_status() == 0
        colerr = np.linalg.norm(Y - Y_or[:, :R], axis=0) / np.linalg.norm(Y_or[:, :R], axis=0)
        assert colerr.max() <= 1e-4, (R, float(colerr.max()))
        if R == 128:
            wide = Y
        elif wide is not None:
            assert _rel(Y, wide[:, :R]) <= 1e-4


def test_graph_replay_and_autotune(loaded):
    """The captured-graph product equals the directly launched one bitwise;
    after autotuning the launch shapes the product still matches the oracle."""
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube12")
    A = _mat(loaded, "cube12")
    B = h2.H2Matrix(c.arrays(), graphs=False)
    try:
        x = torch.from_numpy(synth.random_complex(c.n, 23).astype(np.complex64)).cuda()
        y1 = A.matvec(x).clone()
        y2 = A.matvec(x).clone()          # replay of the captured graph
        y3 = B.matvec(x)
        assert torch.equal(y1, y2) and torch.equal(y1, y3)
        rep = A.autotune()
        assert "near" in rep and rep["near"]["threads"] in (128, 192, 256, 384, 512, 768, 1024)
        y4 = A.matvec(x).cpu().numpy()
        y_or = c.oracle_matvec(x.cpu().numpy().astype(np.complex128))
        assert _rel(y4, y_or) <= 1e-5
    finally:
        B.close()


def test_split_graph_replay_and_tc_autotune(loaded, tmp_path):
    """Split-bf16 product captured into a CUDA graph on first use and replayed
    afterwards: bitwise equal to the directly launched product. Pipeline depths
    chosen by h2_autotune_tc change no arithmetic order (bitwise equal product,
    still within eps of the oracle), and a report cached for this GPU and
    operator shape is applied to another handle without timing."""
    from oracle import h2mv
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube12")
    A = _mat(loaded, "cube12")
    X = _colmajor(synth.random_complex(c.n, 14, cols=130))
    Y1, Y2, Y3 = torch.empty_like(X), torch.empty_like(X), torch.empty_like(X)
    A.configure(graphs=True)
    try:
        A.matvec(X, Y1, prec="splitbf16")      # captured
        A.matvec(X, Y2, prec="splitbf16")      # another output: another graph
        Y1.zero_()
        A.matvec(X, Y1, prec="splitbf16")      # replayed
        A.configure(graphs=False)
        A.matvec(X, Y3, prec="splitbf16")      # direct launches
        assert torch.equal(Y1, Y2) and torch.equal(Y1, Y3)
        cache = str(tmp_path / "tune.json")
        rep = A.autotune(nrhs_tc=130, cache=cache)
        tc = {k: v for k, v in rep.items() if k.startswith("tc_")}
        assert tc and all(2 <= v["ns"] <= 8 for v in tc.values())
        Y4 = torch.empty_like(X)
        A.matvec(X, Y4, prec="splitbf16")
        assert torch.equal(Y4, Y3)
        Y_or = h2mv.h2_dense(c.hZ) @ X.cpu().numpy().astype(np.complex128)
        assert _rel(Y4.cpu().numpy(), Y_or) <= 1e-4
        B = h2.H2Matrix(c.arrays())
        try:
            rb = B.autotune(nrhs_tc=130, cache=cache)
            assert rb.get("cached") is True
            assert {k: v["ns"] for k, v in rb.items() if k.startswith("tc_")} == {k: v["ns"] for k, v in tc.items()}
            assert torch.equal(B.matvec(X, prec="splitbf16"), Y3)
        finally:
            B.close()
    finally:
        A.configure(graphs=True)


def test_tensor_core_timeout_is_reported_and_context_survives(loaded):
    """Injected timeout: with a wait limit of 0 polls every first wait of the
    tensor-core kernels runs out; the kernels drain their copies, skip their
    output and flag the handle, h2_device_status reports H2_ERR_TIMEOUT, and
    the CUDA context stays usable (another handle's product is still right)."""
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube8")
    A = h2.H2Matrix(c.arrays(), wait_limit=0)
    try:
        X = synth.random_complex(c.n, 44, cols=4)
        A.matvec(_colmajor(X), prec="splitbf16")
        assert A.device_status() == 6   # H2_ERR_TIMEOUT
    finally:
        A.close()
    B = _mat(loaded, "cube8")
    x = synth.random_complex(c.n, 45)
    y = B.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert _rel(y, c.oracle_matvec(x)) <= 1e-5
    assert B.device_status() == 0


def test_workspace_allocation_failure_is_reported(loaded):
    """A batched solve whose Krylov basis cannot fit in device memory returns
    H2_ERR_ALLOC and leaves the handle usable."""
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube8")
    A = _mat(loaded, "cube8")
    R = 16384
    B = torch.zeros(c.n, R, dtype=torch.complex128, device="cuda").t().contiguous().t()
    B[0, :] = 1.0
    with pytest.raises(h2.H2Error) as e:
        # Krylov basis of 1025 x N x R complex128 entries: 413 GB, above the 288 GB of HBM
        A.gmres_batched(B, tol=1e-4, restart=1024, maxit=10, prec="fp32")
    assert e.value.status == 2   # H2_ERR_ALLOC
    x = synth.random_complex(c.n, 46)
    y = A.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert _rel(y, c.oracle_matvec(x)) <= 1e-5


def test_save_and_reload_reproduce_products(loaded, tmp_path):
    """An operator written by h2_save and read by h2_load_file gives bitwise
    the same FP32 and split-bf16 products; a flipped byte is rejected."""
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube12")
    A = h2.H2Matrix(c.arrays())   # fresh: the shared handles may carry autotuned CTA sizes
    path = tmp_path / "cube12.h2"
    A.save(str(path))
    B = h2.H2Matrix.from_file(str(path))
    try:
        assert B.stats() == A.stats()
        x = torch.from_numpy(synth.random_complex(c.n, 47).astype(np.complex64)).cuda()
        assert torch.equal(A.matvec(x), B.matvec(x))
        X = _colmajor(synth.random_complex(c.n, 48, cols=5))
        assert torch.equal(A.matvec(X, prec="splitbf16"), B.matvec(X, prec="splitbf16"))
    finally:
        B.close()
        A.close()
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0xFF
    bad = tmp_path / "flipped.h2"
    bad.write_bytes(bytes(raw))
    with pytest.raises(h2.H2Error) as e:
        h2.H2Matrix.from_file(str(bad))
    assert e.value.status == 1   # H2_ERR_ARG


@pytest.mark.parametrize("name", CASES)
def test_symmetric_couplings_match_oracle(loaded, name):
    """Couplings stored once per admissible pair (sym_couple): the product
    matches the oracle within 1e-5 and the full-storage product within 1e-6,
    replays bitwise (graph and direct launches), and stores exactly half of
    the coupling entries."""
    from paper_1703_01175_gb300 import h2
    c = cases.get(name)
    full = _mat(loaded, name)
    A = h2.H2Matrix(c.arrays(), sym_couple=True)
    B = h2.H2Matrix(c.arrays(), sym_couple=True, graphs=False)
    try:
        st = A.sym_stats()
        assert 2 * st["stored_elems"] == full.stats()["coupling_elems"]
        assert st["max_asym"] <= 1e-6
        for seed in (3, 4):
            x = synth.random_complex(c.n, seed)
            xt = torch.from_numpy(x.astype(np.complex64)).cuda()
            y1 = A.matvec(xt).clone()
            y2 = A.matvec(xt).clone()
            y3 = B.matvec(xt)
            assert torch.equal(y1, y2) and torch.equal(y1, y3)
            y = y1.cpu().numpy()
            assert _rel(y, c.oracle_matvec(x)) <= 1e-5
            assert _rel(y, full.matvec(xt).cpu().numpy()) <= 1e-6
    finally:
        A.close()
        B.close()


@pytest.mark.parametrize("name", ["cube8", "ragged", "slab", "odd"])
def test_symmetric_dual_kernel_launch_shapes(loaded, name):
    """Both launch shapes of the dual kernel (4 consumer warps, three CTAs per
    SM: 160 threads; 8 warps, two CTAs: 288 threads), for the couplings and
    the near field: each matches the oracle within 1e-5, the two agree within
    1e-6 (their slot sums group differently), each replays bitwise; the
    autotuner reports a choice for both."""
    import json
    from paper_1703_01175_gb300 import h2
    c = cases.get(name)
    x = synth.random_complex(c.n, 9)
    xt = torch.from_numpy(x.astype(np.complex64)).cuda()
    A = h2.H2Matrix(c.arrays(), sym_couple=True)
    try:
        ref = c.oracle_matvec(x)
        for near in (False, True):
            if near:
                A.sym_near(c.chi)
            ys = {}
            for threads in (160, 288):
                A.apply_tuning({"sym_couple": {"threads": threads}, "sym_near": {"threads": threads}})
                y1 = A.matvec(xt).clone()
                assert torch.equal(y1, A.matvec(xt))
                assert A.device_status() == 0
                ys[threads] = y1.cpu().numpy()
                assert _rel(ys[threads], ref) <= 1e-5
            assert _rel(ys[160], ys[288]) <= 1e-6
        rep = A.autotune()
        assert rep["sym_couple"]["threads"] in (160, 288) and rep["sym_near"]["threads"] in (160, 288)
        assert set(rep["sym_couple"]["tried"]) == {"160", "288"}
        with pytest.raises(h2.H2Error):
            A.apply_tuning({"sym_couple": {"threads": 192}})
        json.dumps(rep)
    finally:
        A.close()


def test_symmetric_couplings_reject_asymmetric_data(loaded):
    """A coupling block whose transpose partner differs is refused with
    H2_ERR_STATE on the first product; the handle's full-storage paths and
    other handles keep working."""
    import dataclasses
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube8")
    arrs = c.arrays()
    S = arrs.S.copy()
    j = int(np.argmax(np.diff(arrs.S_off)))            # a large block
    S[arrs.S_off[j]] += 0.5 * np.abs(S).max()
    bad = dataclasses.replace(arrs, S=S)
    A = h2.H2Matrix(bad, sym_couple=True)
    try:
        x = torch.from_numpy(synth.random_complex(c.n, 5).astype(np.complex64)).cuda()
        with pytest.raises(h2.H2Error) as e:
            A.matvec(x)
        assert e.value.status == 7   # H2_ERR_STATE
        X = torch.from_numpy(np.asfortranarray(synth.random_complex(c.n, 6, cols=3).astype(np.complex64)))
        A.matvec(X.cuda().t().contiguous().t(), prec="splitbf16")   # full storage still usable
        assert A.device_status() == 0
    finally:
        A.close()
    y = _mat(loaded, "cube8").matvec(x).cpu().numpy()
    assert _rel(y, c.oracle_matvec(x.cpu().numpy().astype(np.complex128))) <= 1e-5


def test_symmetric_kernel_timeout_is_reported(loaded):
    """wait_limit=0 makes the first bounded wait of the symmetric-storage
    kernel's bulk-copy pipeline run out: the kernel lets its copies land,
    skips its output and flags the handle (H2_ERR_TIMEOUT), for the couplings
    and for the near field; the context stays usable."""
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube8")
    x = synth.random_complex(c.n, 46)
    xt = torch.from_numpy(x.astype(np.complex64)).cuda()
    A = h2.H2Matrix(c.arrays(), sym_couple=True, wait_limit=0)
    try:
        A.matvec(xt)
        assert A.device_status() == 6   # H2_ERR_TIMEOUT
    finally:
        A.close()
    B = h2.H2Matrix(c.arrays(), sym_couple=True, wait_limit=0)
    try:
        B.sym_near(c.chi)
        B.matvec(xt)
        assert B.device_status() == 6
    finally:
        B.close()
    C = h2.H2Matrix(c.arrays(), sym_couple=True)
    try:
        y = C.matvec(xt).cpu().numpy()
        assert C.device_status() == 0
        assert _rel(y, c.oracle_matvec(x)) <= 1e-5
    finally:
        C.close()


def test_symmetric_couplings_after_reload(loaded, tmp_path):
    """An operator saved and reloaded with sym_couple builds the same
    couplings-once structure and gives the same product bitwise as a handle
    loaded from the arrays with the option."""
    from paper_1703_01175_gb300 import h2
    c = cases.get("ragged")
    A = h2.H2Matrix(c.arrays(), sym_couple=True)
    path = tmp_path / "ragged_sym.h2"
    try:
        A.save(str(path))
        B = h2.H2Matrix.from_file(str(path), sym_couple=True)
        try:
            x = torch.from_numpy(synth.random_complex(c.n, 41).astype(np.complex64)).cuda()
            assert torch.equal(A.matvec(x).clone(), B.matvec(x))
            assert B.sym_stats() == A.sym_stats()
        finally:
            B.close()
    finally:
        A.close()


@pytest.mark.parametrize("name", CASES)
def test_symmetric_near_field_matches_oracle(loaded, name):
    """Near field stored once per leaf pair (with the couplings once per
    pair): stores the diagonal blocks and one block of each pair, matches
    the oracle within 1e-5 and the full-storage product within 1e-6, replays
    bitwise, and h2_sym_near(NULL) returns to the couplings-only product."""
    from paper_1703_01175_gb300 import h2
    c = cases.get(name)
    full = _mat(loaded, name)
    arrs = c.arrays()
    A = h2.H2Matrix(arrs, sym_couple=True)
    try:
        x = synth.random_complex(c.n, 7)
        xt = torch.from_numpy(x.astype(np.complex64)).cuda()
        y_cpl = A.matvec(xt).clone()
        A.sym_near(c.chi)
        st = A.sym_near_stats()
        leaves = np.asarray(arrs.child).reshape(-1, 2)[:, 0] < 0
        diag = int(np.sum(np.asarray(arrs.size, dtype=np.int64)[leaves] ** 2))
        assert 2 * st["stored_elems"] == full.stats()["near_elems"] + diag
        assert st["max_asym"] <= 1e-5
        y1 = A.matvec(xt).clone()
        assert torch.equal(y1, A.matvec(xt))
        y = y1.cpu().numpy()
        assert _rel(y, c.oracle_matvec(x)) <= 1e-5
        assert _rel(y, full.matvec(xt).cpu().numpy()) <= 1e-6
        A.sym_near(None)
        assert torch.equal(A.matvec(xt), y_cpl)
    finally:
        A.close()


def test_symmetric_near_field_refuses_zero_chi(loaded):
    """A zero chi (void voxel) leaves the near field in full storage with
    H2_ERR_STATE; products keep working."""
    from paper_1703_01175_gb300 import h2
    c = cases.get("cube8")
    A = h2.H2Matrix(c.arrays())
    try:
        chi = c.chi.copy()
        chi[5] = 0.0
        with pytest.raises(h2.H2Error) as e:
            A.sym_near(chi)
        assert e.value.status == 7   # H2_ERR_STATE
        x = synth.random_complex(c.n, 8)
        y = A.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
        assert _rel(y, c.oracle_matvec(x)) <= 1e-5
    finally:
        A.close()
