"""The bench's multi-rank host logic on CPU: world_size-2 gloo ranks.

Under torchrun every rank solves its own replica (weak scaling; no data-path
collective).  The job's time is the maximum over ranks, and the whole-job rate
counts every rank's unknowns within that time.  This runs the same helpers
bench.py uses, with the gloo backend on CPU, plus the reference arm's rule
that only rank 0 times the oracle and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import cmg_problems
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")  # rank r "took" 1.5 + r seconds
    rate = bench.job_rate(world, 1000, t)
    # replicas: rank r draws the seeded problem with seed r
    prob = cmg_problems.make_problem("poisson3d_fourier", 3, seed=rank)
    dist.barrier()
    q.put((rank, t, rate, prob.tables.tobytes()))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, tab0), (r1, t1, v1, tab1) = out
    assert t0 == t1 == 2.5          # the slower rank's time, on both ranks
    assert v0 == v1 == 2 * 1000 / 2.5
    assert tab0 != tab1             # independent replicas


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line(tmp_path):
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "poisson2d_257", "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "DoF/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["cycle"].startswith("V(0,1) red-black")
