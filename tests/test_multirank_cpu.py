"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

The product does not shard: `bench.py --gpus N` runs N independent replicas,
times each one and reports the slowest (the maximum over ranks); rank 0 alone
prints the JSON line. These tests run that host logic on two CPU processes:
the maximum over ranks, and the reference arm launched the way the driver
launches it (torch.distributed.run, rendezvous on 127.0.0.1), which must print
exactly one line, from rank 0, with n_gpus = 2.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(1.5 + rank, world)
        one = bench.max_over_ranks(7.0, 1)   # one rank: the value itself, no collective
        with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
            json.dump({"max": got, "one": one}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.loads((tmp_path / f"rank{r}.json").read_text())
        assert d == {"max": 2.5, "one": 7.0}


def test_reference_arm_two_ranks_prints_one_line():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cube8",
           "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["higher_is_better"] is False
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
