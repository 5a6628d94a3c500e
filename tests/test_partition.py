"""Slab partition of the hierarchy over ranks (paper_2511_19036_gb300.partition).

* The plan covers every plane of every level exactly once, aligns each coarse
  level with the finer one (coarse plane c with fine plane 2c + 1), and
  agglomerates on rank 0 the coarse levels where a rank would own too few
  planes, and every level below them.
* The planes the plan says P_l reads and R_l reaches equal the nonzero pattern
  of the first-principles prolongation matrix (tests/fem_dense.py).
* A distributed red-black compact FMG on 2 and 3 gloo ranks, driven by the
  plan and the Exchanger (tests/slab_engine.py), gives every section of u~
  bit for bit equal to the single-rank oracle, for a 2-D L = 7 and a 3-D L = 5
  problem.
"""
import os
import socket
import sys

import numpy as np
import pytest

from fem_dense import prolongation
from paper_2511_19036_gb300.partition import SlabPlan, planes_of

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dim,L,world", [(3, 5, 2), (3, 5, 3), (2, 7, 3), (3, 11, 8), (2, 4, 4), (3, 3, 1)])
def test_plan_covers_aligns_and_agglomerates(dim, L, world):
    plan = SlabPlan(dim, L, world)
    was_dist = True
    for l in range(L, 0, -1):
        n = planes_of(l)
        owners = [plan.owner(l, z) for z in range(n)]
        assert sorted(sum((list(plan.owned(l, r)) for r in range(world)), [])) == list(range(n))
        if plan.distributed[l]:
            assert was_dist and world > 1 and l > 1
            assert min(len(plan.owned(l, r)) for r in range(world)) >= plan.min_planes
            if l < L:
                for c in range(n):  # coarse plane c with the fine plane 2c + 1
                    assert owners[c] == plan.owner(l + 1, 2 * c + 1)
        else:
            assert all(o == 0 for o in owners)
        was_dist = plan.distributed[l]
    assert not plan.distributed[1]


@pytest.mark.parametrize("dim,l", [(3, 3), (3, 4), (2, 5)])
def test_operator_reach_matches_the_prolongation_matrix(dim, l):
    P = prolongation(dim, l)
    n, nc = planes_of(l), planes_of(l - 1)
    per = n ** (dim - 1)
    per_c = nc ** (dim - 1)
    reads = {z: sorted({int(col) // per_c for row in range(z * per, (z + 1) * per) for col in np.flatnonzero(P[row])})
             for z in range(n)}
    for world in (2, 3):
        plan = SlabPlan(dim, l, world, min_planes=1)
        for r in range(world):
            own = plan.owned(l, r)
            want_R = sorted({c for z in own for c in reads[z]})
            assert plan.restrict_target(l, r) == want_R
            fine = list(own) + plan.stencil_halo(l, r)
            want_P = sorted({c for z in fine for c in reads[z]} - set(plan.owned(l - 1, r)))
            assert plan.prolong_source(l, r) == want_P


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = {"2d": ("poisson2d_manufactured", 7, 4, 4, 1.0), "3d": ("poisson3d_manufactured", 5, 5, 4, 0.75)}


def _worker(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import cmg_problems as P
        import oracle
        from slab_engine import SlabFMG
        from paper_2511_19036_gb300.partition import Exchanger, SlabPlan, TorchTransport
        name, L, b1, b2, omega = CASES[case]
        prob = P.make_problem(name, L)
        plan = SlabPlan(prob.dim, L, world)
        ex = Exchanger(plan, TorchTransport())
        eng = SlabFMG(prob, plan, ex, b1, b2, 3, omega)
        eng.fmg()
        secs = [eng.gather(l) for l in range(1, L + 1)]
        if rank == 0:
            o = oracle.Oracle.for_problem(prob, b1=b1, b2=b2, N=3, nu1=0, nu2=1, omega=omega, smoother=1)
            o.fmg()
            assert o.status == 0 and o.inexact == 0
            diff = []
            for l in range(1, L + 1):
                ref = o.get_section(oracle.U, l, words=False)[2].reshape(secs[l - 1].shape)
                diff.append(int(np.sum(ref != secs[l - 1])))
            dist_levels = [l for l in range(1, L + 1) if plan.distributed[l]]
            q.put(("ok", diff, dist_levels))
        dist.barrier()
    except Exception as e:  # report to the parent instead of hanging the other rank
        q.put(("error", repr(e), []))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("2d", 2), ("2d", 3), ("3d", 2), ("3d", 3)])
def test_partitioned_fmg_equals_single_rank_oracle(case, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    status, diff, dist_levels = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
    assert status == "ok", diff
    assert all(p.exitcode == 0 for p in procs)
    assert diff == [0] * len(diff), diff
    assert len(dist_levels) >= 3  # the finest levels really were split
