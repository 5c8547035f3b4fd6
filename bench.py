"""Benchmark of the GB300 H^2 VIE product and solve.

Workload (default): the 32^3-voxel dielectric cube (side 2 wavelengths,
eps_r ~ U[2,6] per voxel, N = 98,304 unknowns, leaf 96, eta = 1, eps = 1e-4),
single right-hand side, FP32 product. One step = one H^2 matrix-vector product
(leaf forward, upward transfers, couplings, downward transfers, leaf
expansion, near field) with the H^2 data resident in HBM; the data is far
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (the product
does not shard across GPUs here) and rank 0 prints the max over ranks.
--impl reference times the FP64 CPU oracle on the same H^2 data on the host
cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cube32"
WORKLOAD_DESC = ("cube32: 32^3 voxel dielectric cube, side 2 lambda, eps_r ~ U[2,6] (seed 2), "
                 "N=98304, leaf 96 unknowns, eta=1, eps=1e-4, 1 RHS")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _peaks_bf16():
    """Dense bf16 tensor peak in GFLOP/s (burst: the product is timed alone)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]) * 1e3
    return 1.9e6


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# Selective reorthogonalisation threshold of the "new" solves: one projection
# keeps w' orthogonal to the basis to about u / eta (Daniel et al. 1976), 10 u
# here; the plain solve keeps the classical eta = 1/sqrt(2).
NEW_ETA = 0.1
NEW_ARNOLDI = "fp32"  # c64 basis, FP32 products with compensated sums, FP64 reductions


def build_workload(name: str):
    """H^2 arrays of the workload from the host constructor (setup, cached on
    disk between runs). Returns (workload, arrays, tree permutation, seconds)."""
    import synth
    from paper_1703_01175_gb300 import construct
    w = synth.workload(name)
    v = w.voxels
    t0 = time.time()
    arrs, perm = construct.build_vie_h2_cached(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps)
    return w, arrs, perm, time.time() - t0


def build_workload_gpu(name: str, device: int):
    """H^2 data of the workload built on the GPU (setup; the same algorithm as
    the host constructor). Returns (workload, host copy of the arrays, tree
    permutation, seconds, DeviceH2 for h2_load_device)."""
    import synth
    from paper_1703_01175_gb300 import construct_gpu
    w = synth.workload(name)
    v = w.voxels
    t0 = time.time()
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps, device=device)
    arrs = dh.to_host()
    return w, arrs, dh.perm, time.time() - t0, dh


def _traffic_from_profile(kernel_src: str, which: str):
    """Per-launch DRAM traffic of the near-field or coupling launch on the
    32^3 cube from the committed ncu summary, if it was taken on the current
    kernel source."""
    path = os.path.join(ROOT, "profiles", f"rowgemv_{which}_cube32.txt")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def oracle_matvec_fn(arrs, perm):
    """The oracle's FP64 H^2 product on the given H^2 data (host cores)."""
    from oracle import h2io, h2mv
    h = h2io.from_flat(arrs, perm)
    return lambda x: h2mv.h2_matvec(h, x)


def _blas_threads():
    try:
        from paper_1703_01175_gb300.construct import _BlasThreads
        return _BlasThreads.threads()
    except Exception:
        return os.cpu_count()


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest value over the ranks of the process group (the slowest
    replica's time per step); the value itself for one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    if rank != 0:
        return
    w, arrs, perm, tb = build_workload(args.workload)
    apply_h2 = oracle_matvec_fn(arrs, perm)
    import synth
    x = synth.random_complex(arrs.n, 1)
    for _ in range(args.warmup):
        apply_h2(x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        apply_h2(x)
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    cores = _blas_threads()
    line = {"impl": "reference", "metric": "h2_matvec_ms", "value": ms, "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64)",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": "one full FP64 H^2 product of the workload per step"},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1703_01175_gb300 import build, h2 as h2py
    import synth

    build.build_all()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w, arrs, perm, t_build, dh = build_workload_gpu(args.workload, local_rank)
    A = h2py.H2Matrix.from_device(dh, device=local_rank)
    dh.free()
    del dh
    n = arrs.n
    if args.only_mrhs:
        # profiling mode: the multi-RHS product alone (no autotuner trial
        # launches, no single-RHS product before it); the last --steps
        # products run inside the NVTX range "timed"
        R = max(1, args.mrhs)
        Xm = torch.from_numpy(np.asfortranarray(synth.random_complex(n, 31, cols=R).astype(np.complex64)))
        Xm = Xm.to(dev).t().contiguous().t()
        Ym = torch.empty_like(Xm)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for k in range(args.warmup + args.steps):
            if k == args.warmup:
                torch.cuda.nvtx.range_push("timed")
                e0.record()
            A.matvec(Xm, Ym, prec=args.mrhs_prec)
        e1.record()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        status = A.device_status()
        A.close()
        if rank == 0:
            print(json.dumps({"only_mrhs": True, "nrhs": R, "prec": args.mrhs_prec, "workload": args.workload,
                              "ms": e0.elapsed_time(e1) / max(1, args.steps), "status": status}), flush=True)
        return

    if args.only_gmres:
        # profiling mode: one cycle of the batched solve (no other legs)
        R = max(1, args.gmres_batch)
        Bm = synth.random_plane_waves(w.voxels, R, seed=5)[(3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)]
        Bt = torch.from_numpy(np.asfortranarray(Bm)).to(dev).t().contiguous().t()
        A.gmres_batched(Bt, tol=1e-12, restart=4, maxit=4, prec="splitbf16", arnoldi=args.arnoldi,
                        reorth_eta=NEW_ETA, check=False)  # workspace and tensor-core images
        torch.cuda.synchronize(dev)
        m = args.gmres_steps
        torch.cuda.nvtx.range_push("timed")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Xs, info = A.gmres_batched(Bt, tol=1e-12, restart=m, maxit=m, prec="splitbf16", arnoldi=args.arnoldi,
                                   reorth_eta=NEW_ETA, check=False)
        e1.record()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        A.close()
        if rank == 0:
            print(json.dumps({"only_gmres": True, "nrhs": R, "steps": m, "workload": args.workload,
                              "arnoldi": args.arnoldi, "ms_per_step": e0.elapsed_time(e1) / m}), flush=True)
        return

    tuning = A.autotune()
    st = A.stats()
    x_np = synth.random_complex(n, 1).astype(np.complex64)
    x = torch.from_numpy(x_np).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        A.matvec(x, y)
    torch.cuda.synchronize(dev)

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push("timed")  # profilers select the timed launches by this range
        ev0.record(stream)
        for _ in range(args.steps):
            A.matvec(x, y)
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)

    if args.only_matvec:
        A.close()
        if rank == 0:
            print(json.dumps({"metric": "h2_matvec_ms", "value": ms, "unit": "ms", "workload": args.workload,
                              "steps": args.steps, "only_matvec": True}), flush=True)
        return

    # per-stage times on the launching stream (sequential, isolated)
    prof = A.profile(x, y, iters=max(5, args.steps))
    hbm, peak_kind = _peaks()
    near_bytes = 8.0 * st["near_elems"] + 16.0 * n
    near_gbs = near_bytes / (prof["near"] * 1e-3) / 1e9
    couple_bytes = 8.0 * st["coupling_elems"]
    couple_gbs = couple_bytes / (prof["coupling"] * 1e-3) / 1e9 if prof["coupling"] > 0 else 0.0
    dominant = "couple" if prof["coupling"] > prof["near"] else "near"
    total_bytes = 8.0 * (st["near_elems"] + st["coupling_elems"] + 2 * st["transfer_elems"]
                         + 2 * st["leaf_elems"]) + 16.0 * n
    mv_gbs = total_bytes / (ms * 1e-3) / 1e9
    src = os.path.join(ROOT, "paper_1703_01175_gb300", "csrc", "h2_gemv.cu")
    traffic = _traffic_from_profile(src, "near")
    traffic_couple = _traffic_from_profile(src, "couple")

    # couplings stored once per admissible pair (S^{s,t} = (S^{t,s})^T): the same product on the same data,
    # reported beside the headline with its own byte count
    sym = None
    if args.sym:
        As = h2py.H2Matrix(arrs, device=local_rank, sym_couple=True)
        sym_tune = As.autotune().get("sym_couple")
        ss = As.sym_stats()
        ys = torch.empty_like(x)
        for _ in range(max(3, args.warmup)):
            As.matvec(x, ys)
        torch.cuda.synchronize(dev)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            As.matvec(x, ys)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        ms_sym = s0.elapsed_time(s1) / args.steps
        sprof = As.profile(x, ys, iters=max(5, args.steps))
        # stored couplings once, plus the scratch vector written and read once
        sym_couple_bytes = 8.0 * ss["stored_elems"] + 16.0 * ss["scratch_entries"]
        sym_bytes = total_bytes - 8.0 * st["coupling_elems"] + sym_couple_bytes
        sym_gbs = sym_bytes / (ms_sym * 1e-3) / 1e9
        sc_gbs = sym_couple_bytes / (sprof["coupling"] * 1e-3) / 1e9
        diff = float(torch.linalg.norm(ys - y) / torch.linalg.norm(y))
        sym = {"ms": ms_sym, "speedup_vs_full_storage": ms / ms_sym, "bytes_per_product": sym_bytes,
               "gbs": sym_gbs, "frac_hbm": sym_gbs / hbm, "stored_coupling_elems": ss["stored_elems"],
               "scratch_entries": ss["scratch_entries"], "max_asym": ss["max_asym"],
               "coupling_stage_ms": sprof["coupling"], "coupling_stage_gbs": sc_gbs,
               "coupling_stage_frac_hbm": sc_gbs / hbm, "rel_diff_vs_full_storage": diff,
               "dual_kernel_tuning": sym_tune}
        # and the near field once per leaf pair (needs chi, nowhere zero on this workload)
        chi = np.repeat(np.asarray(w.voxels.eps_r, dtype=np.complex128)[perm] - 1.0, 3)
        try:
            As.sym_near(chi)
            near_tune = As.autotune().get("sym_near")
            sn = As.sym_near_stats()
            for _ in range(max(3, args.warmup)):
                As.matvec(x, ys)
            torch.cuda.synchronize(dev)
            s0.record(stream)
            for _ in range(args.steps):
                As.matvec(x, ys)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            ms_sn = s0.elapsed_time(s1) / args.steps
            nprof = As.profile(x, ys, iters=max(5, args.steps))
            # stored blocks once, scratch written and read, x read, chi x written and read, y written
            near_sym_bytes = 8.0 * sn["stored_elems"] + 16.0 * sn["scratch_entries"] + 32.0 * n
            sn_bytes = sym_bytes - near_bytes + near_sym_bytes
            sn_gbs = sn_bytes / (ms_sn * 1e-3) / 1e9
            nn_gbs = near_sym_bytes / (nprof["near"] * 1e-3) / 1e9
            sym["with_near"] = {
                "ms": ms_sn, "speedup_vs_full_storage": ms / ms_sn, "bytes_per_product": sn_bytes, "gbs": sn_gbs,
                "frac_hbm": sn_gbs / hbm, "stored_near_elems": sn["stored_elems"], "max_asym": sn["max_asym"],
                "near_stage_ms": nprof["near"], "near_stage_gbs": nn_gbs, "near_stage_frac_hbm": nn_gbs / hbm,
                "rel_diff_vs_full_storage": float(torch.linalg.norm(ys - y) / torch.linalg.norm(y)),
                "dual_kernel_tuning": near_tune}
        except h2py.H2Error as e:
            sym["with_near"] = {"unavailable": str(e)}
        As.close()

    # GMRES to 1e-4: plain (FP32 products, FP64 Arnoldi) and with FP64-accumulated restart residuals
    b_np = synth.default_rhs(w)[3 * perm[:, None] + np.arange(3)[None, :]].reshape(-1)
    b = torch.from_numpy(b_np).to(dev)
    gm = {"tol": w.tol, "restart": 50, "rhs": "x-polarised plane wave, +z incidence"}
    for label, refine in (("plain", False), ("refined", True)):
        A.gmres(b, tol=w.tol, restart=50, maxit=2000, refine=refine)  # warm-up (workspace)
        torch.cuda.synchronize(dev)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        xs, info = A.gmres(b, tol=w.tol, restart=50, maxit=2000, refine=refine)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        gm[label] = {"ms": g0.elapsed_time(g1), "iterations": info[0]["iterations"],
                     "rel_res": info[0]["rel_res"], "status": info[0]["status"],
                     "reorth_steps": info[0]["reorth_steps"]}

    # the paper's solver: BiCGStab, FP32 products, true residual checked with the FP64-accumulated product
    A.bicgstab(b, tol=w.tol, maxit=10, refine=True)  # warm-up (workspace)
    torch.cuda.synchronize(dev)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    xs, info = A.bicgstab(b, tol=w.tol, maxit=3000, refine=True)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    gm["bicgstab"] = {"ms": g0.elapsed_time(g1), "iterations": info[0]["iterations"],
                      "products": 2 * info[0]["iterations"], "restarts": info[0]["restarts"],
                      "rel_res": info[0]["rel_res"], "status": info[0]["status"]}

    # multi-RHS products: R right-hand sides at once (split-bf16 tensor cores vs FP32 CUDA cores)
    mr = None
    if args.mrhs > 0:
        R = args.mrhs
        Xm = torch.from_numpy(np.asfortranarray(synth.random_complex(n, 31, cols=R).astype(np.complex64)))
        Xm = Xm.to(dev).t().contiguous().t()
        Ym = torch.empty_like(Xm)
        mr = {"nrhs": R}
        entries = st["near_elems"] + st["coupling_elems"] + 2 * st["transfer_elems"] + 2 * st["leaf_elems"]
        tc_entries = st["near_elems"] + st["coupling_elems"]
        tc_tuning = A.autotune(nrhs_tc=R, fp32=False)
        for label, prec in (("splitbf16", "splitbf16"), ("fp32", "fp32")):
            for _ in range(3):
                A.matvec(Xm, Ym, prec=prec)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                A.matvec(Xm, Ym, prec=prec)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t_ms = e0.elapsed_time(e1) / args.steps
            mr[label] = {"ms": t_ms, "us_per_rhs": 1e3 * t_ms / R,
                         "algorithmic_tflops": 8.0 * R * entries / (t_ms * 1e-3) / 1e12}
        # executed on the tensor cores: 3 split products per real MAC (padding not counted)
        mr["splitbf16"]["tensor_tflops_executed"] = 3.0 * mr["splitbf16"]["algorithmic_tflops"]
        mr["splitbf16"]["tensor_frac_of_bf16_peak"] = mr["splitbf16"]["tensor_tflops_executed"] * 1e3 / _peaks_bf16()
        # streamed: hi and lo bf16 of Re and Im of every stored entry (8 B), X read and Y written once
        split_bytes = 8.0 * entries + 16.0 * R * n
        mr["splitbf16"]["bytes"] = split_bytes
        mr["splitbf16"]["gbs"] = split_bytes / (mr["splitbf16"]["ms"] * 1e-3) / 1e9
        mr["splitbf16"]["frac_hbm"] = mr["splitbf16"]["gbs"] / _peaks()[0]
        mr["splitbf16"]["pipeline_depths"] = {k: v["ns"] for k, v in tc_tuning.items()}
        # the same product launched directly, without the captured graph
        A.configure(graphs=False)
        for _ in range(3):
            A.matvec(Xm, Ym, prec="splitbf16")
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            A.matvec(Xm, Ym, prec="splitbf16")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        A.configure(graphs=True)
        mr["splitbf16"]["ms_without_graph"] = e0.elapsed_time(e1) / args.steps
        mr["status"] = A.device_status()
        mr["speedup_vs_single_rhs_fp32"] = (ms * R) / mr["splitbf16"]["ms"]
        mr["tc_entries"] = tc_entries

    # "new" solve: R right-hand sides in lockstep, split-bf16 tensor-core products, Arnoldi on a c64 basis and
    # double-float-accumulated restart residuals; compared per right-hand side with plain single-RHS GMRES
    # (FP32 products, FP64 Arnoldi, FP64-accumulated restart residuals)
    if args.gmres_batch > 0:
        R = args.gmres_batch
        Bm = synth.random_plane_waves(w.voxels, R, seed=5)[(3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)]
        Bt = torch.from_numpy(np.asfortranarray(Bm)).to(dev).t().contiguous().t()
        m_new = args.gmres_restart
        b0 = Bt[:, 0].contiguous()
        for label, arn, eta in (("plain_m%d" % m_new, "fp64", 0.0), ("plain_m%d_df" % m_new, "df", NEW_ETA)):
            torch.cuda.synchronize(dev)
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            xs, info = A.gmres(b0, tol=w.tol, restart=m_new, maxit=4000, refine=True, arnoldi=arn, reorth_eta=eta)
            g1.record(stream)
            torch.cuda.synchronize(dev)
            gm[label] = {"ms": g0.elapsed_time(g1), "iterations": info[0]["iterations"],
                         "rel_res": info[0]["rel_res"], "status": info[0]["status"],
                         "reorth_steps": info[0]["reorth_steps"],
                         "arnoldi": "FP64" if arn == "fp64" else "double-float on the FP32 pipes",
                         "reorth_eta": eta if eta > 0 else 2 ** -0.5,
                         "refinement_product": "FP64ACC" if arn == "fp64" else "DFACC"}
        torch.cuda.synchronize(dev)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        Xs, info = A.gmres_batched(Bt, tol=w.tol, restart=m_new, maxit=4000, refine=True, prec="splitbf16",
                                   arnoldi=NEW_ARNOLDI, reorth_eta=NEW_ETA)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        t_new = g0.elapsed_time(g1)
        gm["new_batched"] = {"nrhs": R, "restart": m_new, "ms_total": t_new, "ms_per_rhs": t_new / R,
                             "converged": sum(1 for i in info if i["status"] == 0),
                             "max_rel_res": max(i["rel_res"] for i in info),
                             "mean_iterations": float(np.mean([i["iterations"] for i in info])),
                             "mean_reorth_steps": float(np.mean([i["reorth_steps"] for i in info])),
                             "reorth_eta": NEW_ETA,
                             "products": "split-bf16 tensor cores; Gram-Schmidt on a c64 basis (FP32 products, "
                                         "compensated per-thread sums, FP64 reductions) with selective "
                                         "reorthogonalisation; double-float-accumulated restart residuals",
                             "arnoldi": NEW_ARNOLDI}
        # plain batched: the same right-hand sides in lockstep, FP32 CUDA-core products, FP64 Arnoldi at the
        # default eta, FP64-accumulated restart residuals -- isolates what mixed precision buys
    if args.gmres_batch > 0 and args.plain_batched:
        torch.cuda.synchronize(dev)
        g0.record(stream)
        Xp, info_p = A.gmres_batched(Bt, tol=w.tol, restart=m_new, maxit=4000, refine=True, prec="fp32",
                                     arnoldi="fp64", reorth_eta=0.0)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        t_pb = g0.elapsed_time(g1)
        gm["plain_batched"] = {"nrhs": R, "restart": m_new, "ms_total": t_pb, "ms_per_rhs": t_pb / R,
                               "converged": sum(1 for i in info_p if i["status"] == 0),
                               "max_rel_res": max(i["rel_res"] for i in info_p),
                               "mean_iterations": float(np.mean([i["iterations"] for i in info_p])),
                               "mean_reorth_steps": float(np.mean([i["reorth_steps"] for i in info_p])),
                               "reorth_eta": 2 ** -0.5, "arnoldi": "fp64",
                               "products": "FP32 CUDA-core multi-RHS GEMMs; FP64 Gram-Schmidt; "
                                           "FP64-accumulated restart residuals"}
        del Xp
        gm["new_vs_plain_batched_per_rhs"] = gm["plain_batched"]["ms_per_rhs"] / gm["new_batched"]["ms_per_rhs"]
    if args.gmres_batch > 0:
        gm["new_vs_plain_per_rhs"] = gm["plain_m%d" % m_new]["ms"] / gm["new_batched"]["ms_per_rhs"]
        gm["new_vs_plain_df_per_rhs"] = gm["plain_m%d_df" % m_new]["ms"] / gm["new_batched"]["ms_per_rhs"]

    # learned preconditioner (config 4): the network trained by train_precond on pairs from the method's own
    # solves of the 48^3 smooth-permittivity cube, as the right preconditioner of batched flexible GMRES(m)
    # (split-bf16 products, c64-basis Arnoldi) against plain batched GMRES(m) on 32 held-out plane waves
    wpath = os.path.join(ROOT, "paper_1703_01175_gb300", "weights", "vie_cube48.npz")
    if args.learned and os.path.exists(wpath):
        gm["learned"] = learned_leg(wpath, local_rank, dev, stream)

    # end to end through the host-pointer entry point: x copied in from pinned host memory, the product,
    # y copied back to pinned host memory, every step (host wall clock around the synchronous calls)
    xh = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    yh = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    xh.copy_(torch.from_numpy(x_np))
    xh_np, yh_np = xh.numpy(), yh.numpy()
    for _ in range(3):
        A.matvec_host(xh_np, out=yh_np)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        A.matvec_host(xh_np, out=yh_np)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        apply_h2 = oracle_matvec_fn(arrs, perm)
        xc = x_np.astype(np.complex128)
        apply_h2(xc)
        t0 = time.perf_counter()
        reps = 0
        while reps < 1 or (time.perf_counter() - t0 < 10.0 and reps < 3):
            apply_h2(xc)
            reps += 1
        cpu_ms = (time.perf_counter() - t0) * 1e3 / reps
        cpu = {"value": cpu_ms, "unit": "ms", "cores": _blas_threads(), "kind": "oracle",
               "sample": f"{reps} full FP64 H^2 product(s) of the workload on the host (numpy)"}
        # one core, comparable to the paper's single-core setting
        from paper_1703_01175_gb300.construct import _BlasThreads
        with _BlasThreads(1):
            t0 = time.perf_counter()
            apply_h2(xc)
            cpu["single_core"] = {"value": (time.perf_counter() - t0) * 1e3, "unit": "ms", "cores": 1,
                                  "sample": "one full FP64 H^2 product of the workload, BLAS on one thread"}

    A.close()
    torch.cuda.empty_cache()
    geos = None
    if args.geometries:
        geos = {}
        for gname in ("slab256", "cube64v", "array4096"):
            try:
                geos[gname] = geometry_leg(gname, 5, 3, local_rank)
            except Exception as e:  # a failed leg is reported, the headline stands
                geos[gname] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()
    if rank != 0:
        return
    launches = st["kernels_per_matvec"]
    line = {
        "metric": "h2_matvec_ms", "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 (fp32)", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC if args.workload == WORKLOAD else args.workload, "l2": "H^2 data per step larger than L2 (no flush needed)",
                   "parallelism": f"replicas x{world}", "h2_build_s": round(t_build, 1), "h2_built_on": "GPU (construct_gpu)",
                   "h2_bytes_per_step": total_bytes, "near_blocks": st["near_blocks"],
                   "adm_blocks": st["adm_blocks"], "max_rank": st["max_rank"]},
        "matvec_gbs": mv_gbs, "matvec_frac_hbm": mv_gbs / hbm,
        "stages_ms": prof,
        "autotune": {k: v["threads"] for k, v in tuning.items()},
        "gmres": gm,
        "mrhs": mr,
        "roofline": ({"bound": "hbm", "kernel": "rowgemv (coupling launch, all levels)", "achieved": couple_gbs,
                      "peak": hbm, "unit": "GB/s", "frac": couple_gbs / hbm, "traffic": traffic_couple,
                      "algorithmic_bytes_per_launch": couple_bytes, "peak_source": peak_kind}
                     if dominant == "couple" else
                     {"bound": "hbm", "kernel": "rowgemv (near-field launch)", "achieved": near_gbs,
                      "peak": hbm, "unit": "GB/s", "frac": near_gbs / hbm, "traffic": traffic,
                      "algorithmic_bytes_per_launch": near_bytes, "peak_source": peak_kind}),
        "symmetric_couplings": sym,
        "geometries": geos,
        "stage_roofline": {"near": {"gbs": near_gbs, "frac": near_gbs / hbm, "bytes": near_bytes},
                           "couple": {"gbs": couple_gbs, "frac": couple_gbs / hbm, "bytes": couple_bytes}},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def run_geometry(args, local_rank):
    line = geometry_leg(args.geometry, args.steps, args.warmup, local_rank)
    print(json.dumps(line), flush=True)


GEOMETRY_NRHS = {"slab256": 128, "cube64v": 256, "array4096": 256, "cube48": 32}


def geometry_leg(geometry, steps, warmup, local_rank):
    """One of the paper's scaling geometries at full size (BASELINE configs 3
    and 5): H^2 data built on the GPU (construct_gpu, timed separately), loaded
    through h2_load_device; the FP32 single-RHS product and the split-bf16
    product of the workload's right-hand sides, each with its algorithmic bytes
    against the HBM peak; ranks and admissible blocks per level; bytes per
    unknown."""
    import torch
    import synth
    from paper_1703_01175_gb300 import build, construct_gpu, h2 as h2py
    build.build_all()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.workload(geometry)
    v = w.voxels
    t0 = time.time()
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps,
                                        device=local_rank)
    torch.cuda.synchronize(dev)
    t_build = time.time() - t0
    build_info = dh.info
    rank, lp = dh.rank.astype(np.int64), dh.level_ptr
    adm_rows = np.diff(dh.adm_ptr.astype(np.int64))
    levels = []
    for l in range(len(lp) - 1):
        r = rank[lp[l]:lp[l + 1]]
        a = adm_rows[lp[l]:lp[l + 1]]
        if r.max() == 0 and a.sum() == 0:
            continue
        levels.append({"level": l, "clusters": int(len(r)), "n_t": int(dh.size[lp[l]]), "max_rank": int(r.max()),
                       "mean_rank": round(float(r.mean()), 1), "adm_blocks": int(a.sum()),
                       "C_sp": round(float(a.sum()) / max(1, int((a > 0).sum())), 1)})
    t1 = time.time()
    A = h2py.H2Matrix.from_device(dh, device=local_rank)
    t_load = time.time() - t1
    dh.free()
    del dh
    torch.cuda.empty_cache()
    st = A.stats()
    n = st["n"]
    entries = st["near_elems"] + st["coupling_elems"] + 2 * st["transfer_elems"] + 2 * st["leaf_elems"]
    hbm, peak_kind = _peaks()
    x = torch.from_numpy(synth.random_complex(n, 1).astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    A.autotune()
    for _ in range(max(3, warmup)):
        A.matvec(x, y)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        e0.record()
        for _ in range(steps):
            A.matvec(x, y)
        e1.record()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    bytes_fp32 = 8.0 * entries + 16.0 * n
    R = GEOMETRY_NRHS[geometry]
    Xm = torch.from_numpy(np.asfortranarray(synth.random_complex(n, 31, cols=R).astype(np.complex64)))
    Xm = Xm.to(dev).t().contiguous().t()
    Ym = torch.empty_like(Xm)
    tc = A.autotune(nrhs_tc=R, fp32=False)
    for _ in range(3):
        A.matvec(Xm, Ym, prec="splitbf16")
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(steps):
        A.matvec(Xm, Ym, prec="splitbf16")
    e1.record()
    torch.cuda.synchronize(dev)
    ms_split = e0.elapsed_time(e1) / steps
    status = A.device_status()
    A.close()
    del Xm, Ym, x, y
    torch.cuda.empty_cache()
    bytes_split = 8.0 * entries + 2 * 8.0 * R * n   # hi and lo bf16 of Re and Im per stored entry; X read, Y written
    tensor_tflops = 24.0 * R * entries / (ms_split * 1e-3) / 1e12   # executed: 3 split products x 4 real MACs x 2
    line = {"geometry": geometry, "n": n, "nrhs": R, "h2_build_s": round(t_build, 1),
            "h2_build_stages_s": {k: round(v, 2) for k, v in build_info["seconds"].items()},
            "load_s": round(t_load, 2),
            "fp32": {"ms": ms, "gbs": bytes_fp32 / (ms * 1e-3) / 1e9, "frac_hbm": bytes_fp32 / (ms * 1e-3) / 1e9 / hbm,
                     "bytes": bytes_fp32},
            "splitbf16": {"ms": ms_split, "us_per_rhs": 1e3 * ms_split / R, "gbs": bytes_split / (ms_split * 1e-3) / 1e9,
                          "frac_hbm": bytes_split / (ms_split * 1e-3) / 1e9 / hbm, "tensor_tflops_executed": tensor_tflops,
                          "tensor_frac_of_bf16_peak": tensor_tflops * 1e3 / _peaks_bf16(), "status": status,
                          "pipeline_depths": {k: v["ns"] for k, v in tc.items()}},
            "bytes_per_unknown": bytes_fp32 / n, "stored_entries": entries, "max_rank": st["max_rank"],
            "near_blocks": st["near_blocks"], "adm_blocks": st["adm_blocks"], "levels": levels,
            "peak_gbs": hbm, "peak_source": peak_kind, "clocks": clk.summary()}
    return line


def geometry_solve_leg(geometry, local_rank, nrhs, restart, maxit, plain_rhs=1):
    """Solves on one of the paper's scaling geometries at full size: the
    batched mixed-precision GMRES(m) (split-bf16 tensor-core products, c64-basis
    Arnoldi with selective reorthogonalisation, double-float-accumulated restart
    residuals) on `nrhs` random plane waves, run in batches whose Krylov basis
    fits the free device memory, against plain single-RHS GMRES(m) (FP32
    products, FP64 Arnoldi, FP64-accumulated restart residuals) on the first
    `plain_rhs` of them; per right-hand side, with CUDA events."""
    import torch
    import synth
    from paper_1703_01175_gb300 import build, construct_gpu, h2 as h2py
    build.build_all()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = synth.workload(geometry)
    v = w.voxels
    t0 = time.time()
    dh = construct_gpu.build_vie_h2_gpu(v.centres, v.dv, v.eps_r, n_min=w.n_min, eta=w.eta, eps=w.eps,
                                        device=local_rank)
    torch.cuda.synchronize(dev)
    t_build = time.time() - t0
    perm = dh.perm
    A = h2py.H2Matrix.from_device(dh, device=local_rank)
    dh.free()
    del dh
    torch.cuda.empty_cache()
    n = A.n
    A.autotune()
    A.autotune(nrhs_tc=min(nrhs, 128), fp32=False)
    unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    Bm = synth.random_plane_waves(v, nrhs, seed=5)[unk]
    # batch size: the c64 Krylov basis (m + 1 columns), the c128 right-hand sides and solutions and the
    # per-RHS work vectors within 80 % of the free memory, at most 128 right-hand sides per batch
    free, _ = torch.cuda.mem_get_info(dev)
    per_rhs = (restart + 1) * n * 8 + 2 * n * 16 + 8 * n * 16
    batch = int(max(1, min(128, nrhs, (0.8 * free) // per_rhs)))
    out = {"geometry": geometry, "n": n, "h2_build_s": round(t_build, 1), "tol": w.tol, "restart": restart,
           "maxit": maxit, "nrhs": nrhs, "batch": batch, "rhs": "random plane waves (seed 5)"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # untimed call of the same shape: Krylov workspace, tensor-core planes and graphs
    Bw = torch.from_numpy(np.asfortranarray(Bm[:, :batch])).to(dev).t().contiguous().t()
    A.gmres_batched(Bw, tol=1e-12, restart=restart, maxit=2, refine=True, prec="splitbf16", arnoldi=NEW_ARNOLDI,
                    reorth_eta=NEW_ETA, check=False)
    del Bw
    infos, t_new = [], 0.0
    for c0 in range(0, nrhs, batch):
        Bt = torch.from_numpy(np.asfortranarray(Bm[:, c0:c0 + batch])).to(dev).t().contiguous().t()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        Xs, info = A.gmres_batched(Bt, tol=w.tol, restart=restart, maxit=maxit, refine=True, prec="splitbf16",
                                   arnoldi=NEW_ARNOLDI, reorth_eta=NEW_ETA)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t_new += e0.elapsed_time(e1)
        infos += info
        del Xs, Bt
        torch.cuda.empty_cache()
    out["new_batched"] = {"ms_total": t_new, "ms_per_rhs": t_new / nrhs,
                          "converged": sum(1 for i in infos if i["status"] == 0),
                          "max_rel_res": max(i["rel_res"] for i in infos),
                          "mean_iterations": float(np.mean([i["iterations"] for i in infos])),
                          "max_iterations": int(max(i["iterations"] for i in infos)),
                          "arnoldi": NEW_ARNOLDI, "reorth_eta": NEW_ETA}
    print(json.dumps({"geometry_solve_partial": out}), file=sys.stderr, flush=True)
    plain = []
    for j in range(plain_rhs):
        b0 = torch.from_numpy(np.ascontiguousarray(Bm[:, j])).to(dev)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        xs, info = A.gmres(b0, tol=w.tol, restart=restart, maxit=maxit, refine=True, arnoldi="fp64")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        plain.append({"ms": e0.elapsed_time(e1), "iterations": info[0]["iterations"],
                      "rel_res": info[0]["rel_res"], "status": info[0]["status"],
                      "new_iterations_same_rhs": infos[j]["iterations"]})
        del xs, b0
    out["plain"] = plain
    both = all(p["status"] == 0 for p in plain) and out["new_batched"]["converged"] == nrhs
    out["both_converged"] = both
    if both:
        out["new_vs_plain_per_rhs"] = float(np.mean([p["ms"] for p in plain])) / out["new_batched"]["ms_per_rhs"]
    out["status"] = A.device_status()
    A.close()
    return out


def learned_leg(wpath, local_rank, dev, stream, nrhs=32, restart=50, maxit=3000):
    """Batched FGMRES with the trained network against plain batched GMRES on
    held-out plane waves (seed 6) of the 48^3 smooth-permittivity cube; the
    time ratio is quoted only when both arms converged on every right-hand
    side."""
    import torch
    import synth
    from paper_1703_01175_gb300 import precond as P, h2 as h2py
    z = np.load(wpath)
    rec = json.loads(str(z["record"])) if "record" in z.files else {}
    layers = [tuple(int(v) for v in x) for x in z["layers"]]
    Wl = [z[f"W{i}"] for i in range(len(layers))]
    Bl = [z[f"b{i}"] for i in range(len(layers))]
    wname = rec.get("train_workload", "cube48")
    w, arrs, perm, t_build, dh = build_workload_gpu(wname, local_rank)
    del arrs
    Aw = h2py.H2Matrix.from_device(dh, device=local_rank)
    dh.free()
    del dh
    out = {"weights": os.path.relpath(wpath, ROOT), "workload": wname, "n": Aw.n, "nrhs": nrhs, "restart": restart,
           "n_params": int(sum(x.size for x in Wl) + sum(x.size for x in Bl)),
           "training": {k: rec.get(k) for k in ("pairs", "solve_pairs", "probe_pairs", "loss", "epochs")}}
    try:
        gmw = P.GridMap(w.voxels.shape, perm, w.voxels.eps_r)
        P.load_into(Aw, layers, Wl, Bl, gmw)
        unk = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
        B = synth.random_plane_waves(w.voxels, nrhs, seed=6)[unk]
        Bt = torch.from_numpy(np.asfortranarray(B)).to(dev).t().contiguous().t()
        for label, pc in (("plain", False), ("fgmres_learned", True)):
            Aw.gmres_batched(Bt, tol=1e-12, restart=4, maxit=4, refine=True, prec="splitbf16", arnoldi="fp32",
                             reorth_eta=NEW_ETA, precond=pc, check=False)   # workspace, images
            torch.cuda.synchronize(dev)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            X, info = Aw.gmres_batched(Bt, tol=w.tol, restart=restart, maxit=maxit, refine=True, prec="splitbf16",
                                       arnoldi="fp32", reorth_eta=NEW_ETA, precond=pc, check=False)
            g1.record(stream)
            torch.cuda.synchronize(dev)
            out[label] = {"ms_total": g0.elapsed_time(g1), "ms_per_rhs": g0.elapsed_time(g1) / nrhs,
                          "converged": sum(1 for i in info if i["status"] == 0),
                          "mean_iterations": float(np.mean([i["iterations"] for i in info])),
                          "max_rel_res": max(i["rel_res"] for i in info),
                          "mean_precond_cycles": float(np.mean([i["precond_cycles"] for i in info]))}
            del X
        both = out["plain"]["converged"] == nrhs and out["fgmres_learned"]["converged"] == nrhs
        out["both_converged"] = both
        out["time_ratio_plain_over_learned"] = (out["plain"]["ms_total"] / out["fgmres_learned"]["ms_total"]
                                                if both else None)
        # the plain FP32 GMRES(m) of the method on one of the same right-hand sides (single RHS, FP32
        # products, FP64 Arnoldi, FP64-accumulated restart residuals): the comparator of the full
        # mixed-precision, batched, learned-preconditioned solve
        b0 = Bt[:, 0].contiguous()
        torch.cuda.synchronize(dev)
        g0.record(stream)
        xs, info = Aw.gmres(b0, tol=w.tol, restart=restart, maxit=maxit, refine=True, arnoldi="fp64", check=False)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        out["plain_fp32_single"] = {"ms": g0.elapsed_time(g1), "iterations": info[0]["iterations"],
                                    "rel_res": info[0]["rel_res"], "status": info[0]["status"]}
        if out["plain_fp32_single"]["status"] == 0 and out["fgmres_learned"]["converged"] == nrhs:
            out["learned_batched_vs_plain_fp32_per_rhs"] = (out["plain_fp32_single"]["ms"] /
                                                           out["fgmres_learned"]["ms_per_rhs"])
        del xs
    finally:
        Aw.close()
        torch.cuda.empty_cache()
    return out


def nn_timing(steps=20, dims=(48, 48, 48)):
    """CUDA-event times of the learned preconditioner's tensor-core
    convolutions on the 48^3 grid (32 -> 32 channels, the hidden layers of the
    network): forward for batches of 1 and 32 grids, weight gradient for a
    training batch of 8; with the executed tensor flops against the bf16
    peak (the forward counts 2 x 27 x 32 x 32 flops per voxel, the weight
    gradient the same twice for its hi and lo dz products)."""
    import torch
    from paper_1703_01175_gb300 import build, precond as P
    build.build_all()
    V = dims[0] * dims[1] * dims[2]
    out = {"grid": list(dims), "cin": 32, "cout": 32}
    g = torch.Generator(device="cuda").manual_seed(3)
    w = (torch.randn(32 * 27 * 32, device="cuda", generator=g) * 0.05).to(torch.bfloat16)
    bias = torch.zeros(32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for B in (1, 32):
        x = torch.randn(B * V * 32, device="cuda", generator=g).to(torch.bfloat16)
        y = torch.empty_like(x)
        for _ in range(3):
            P._call("h2nn_conv3d_fwd", P._p(x), P._p(w), P._p(bias), P._p(y), None, B, *dims, 32, 32, 1, st)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            P._call("h2nn_conv3d_fwd", P._p(x), P._p(w), P._p(bias), P._p(y), None, B, *dims, 32, 32, 1, st)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        fl = 2.0 * 27 * 32 * 32 * V * B
        out[f"fwd_B{B}"] = {"ms": ms, "tflops": fl / (ms * 1e-3) / 1e12,
                            "frac_bf16_peak": fl / (ms * 1e-3) / 1e9 / _peaks_bf16()}
        del x, y
    B = 8
    x = torch.randn(B * V * 32, device="cuda", generator=g).to(torch.bfloat16)
    dz = torch.randn(B * V * 32, device="cuda", generator=g)
    dw = torch.empty(32 * 27 * 32, device="cuda")
    db = torch.empty(32, device="cuda")
    for _ in range(3):
        P._call("h2nn_conv3d_bwd_weight", P._p(dz), P._p(x), P._p(dw), P._p(db), B, *dims, 32, 32, 0, st)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        P._call("h2nn_conv3d_bwd_weight", P._p(dz), P._p(x), P._p(dw), P._p(db), B, *dims, 32, 32, 0, st)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    fl = 2.0 * 2.0 * 27 * 32 * 32 * V * B
    out["bwd_weight_B8"] = {"ms": ms, "tflops": fl / (ms * 1e-3) / 1e12,
                            "frac_bf16_peak": fl / (ms * 1e-3) / 1e9 / _peaks_bf16()}
    out["status"] = P._nnlib().h2nn_device_status()
    print(json.dumps({"nn_timing": out}), flush=True)


def fp_rates():
    """FP64 and FP32 (tensor cores off) GEMM throughput of cuda:0 with cuBLAS:
    the ceilings of the FP64 Gram-Schmidt passes and of their double-float
    replacement on the FP32 pipes."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    for name, dt, n in (("fp64", torch.float64, 8192), ("fp32", torch.float32, 8192)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        for _ in range(3):
            torch.matmul(a, b)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3 if dt == torch.float64 else 10
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"n": n, "ms": ms, "tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12}
    print(json.dumps({"gemm_rates": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned-preconditioner leg")
    ap.add_argument("--gmres-batch", type=int, default=128, help="right-hand sides of the batched solve (0: skip)")
    ap.add_argument("--gmres-restart", type=int, default=400, help="restart of the batched / plain comparison")
    ap.add_argument("--mrhs", type=int, default=128, help="right-hand sides of the multi-RHS leg (0: skip)")
    ap.add_argument("--no-sym", dest="sym", action="store_false",
                    help="skip the product with couplings stored once per admissible pair")
    ap.add_argument("--nn", action="store_true",
                    help="time the learned preconditioner's convolutions on the 48^3 grid and exit")
    ap.add_argument("--fp-rates", action="store_true",
                    help="print the FP64 and FP32 (non-tensor) GEMM rates of the GPU and exit")
    ap.add_argument("--mrhs-prec", default="splitbf16", choices=["splitbf16", "fp32"],
                    help="product of the --only-mrhs profiling mode")
    ap.add_argument("--workload", default=WORKLOAD, help="synthetic workload name (profiling uses smaller ones)")
    ap.add_argument("--only-mrhs", action="store_true",
                    help="run split-bf16 multi-RHS products only (profiling)")
    ap.add_argument("--only-gmres", action="store_true",
                    help="run one cycle of --gmres-steps steps of the batched double-float solve only (profiling)")
    ap.add_argument("--gmres-steps", type=int, default=60, help="Arnoldi steps of the --only-gmres cycle")
    ap.add_argument("--arnoldi", default="fp32", choices=["fp64", "df", "fp32"],
                    help="Arnoldi arithmetic of the --only-gmres cycle")
    ap.add_argument("--geometry", default=None, choices=["slab256", "cube64v", "array4096", "cube48"],
                    help="time one full-size scaling geometry built on the GPU and exit")
    ap.add_argument("--geometry-solve", default=None, choices=["slab256", "cube64v", "array4096"],
                    help="time only the batched mixed-precision solve against plain GMRES on this geometry")
    ap.add_argument("--solve-rhs", type=int, default=0, help="right-hand sides of --geometry-solve (0: the geometry's)")
    ap.add_argument("--solve-restart", type=int, default=150, help="GMRES restart of --geometry-solve")
    ap.add_argument("--solve-maxit", type=int, default=3000, help="iteration cap of --geometry-solve")
    ap.add_argument("--solve-plain-rhs", type=int, default=1, help="plain single-RHS solves of --geometry-solve")
    ap.add_argument("--no-geometries", dest="geometries", action="store_false",
                    help="skip the full-size slab, 64^3 cube and cube-array legs (GPU construction, about 3 minutes)")
    ap.add_argument("--no-plain-batched", dest="plain_batched", action="store_false",
                    help="skip the batched plain GMRES arm (FP64 Arnoldi, about two minutes)")
    ap.add_argument("--only-matvec", action="store_true",
                    help="time the products only (no GMRES, host-pointer or CPU legs): a fixed launch sequence")
    args = ap.parse_args()
    if args.fp_rates:
        fp_rates()
        return
    if args.nn:
        nn_timing(args.steps)
        return
    if args.geometry:
        run_geometry(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.geometry_solve:
        line = geometry_solve_leg(args.geometry_solve, int(os.environ.get("LOCAL_RANK", "0")),
                                  args.solve_rhs or GEOMETRY_NRHS[args.geometry_solve], args.solve_restart,
                                  args.solve_maxit, args.solve_plain_rhs)
        print(json.dumps({"geometry_solve": line}), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
