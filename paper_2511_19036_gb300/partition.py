"""Slab partition of the compact hierarchy over ranks, and its exchanges (host logic).

The compact cycle is data-parallel over the nodes of each level; what couples
ranks is the reach of its three operators: the 7-/5-point stencil A_l (one node
in each direction), the prolongation P_l (a fine node reads the coarse nodes of
its Kuhn edge) and the restriction R_l = P_l^T.  A BFP block is 32 consecutive
x-values of one row (Sec. 6.1.3 storage), so a partition that never splits a
block cuts each level into slabs of whole planes: z-planes in 3-D, rows (y) in
2-D.  This module holds that partition:

* ``SlabPlan``: which planes of every level each rank owns.  The finest level is
  cut into balanced contiguous slabs; every coarser level follows the finer one
  (coarse plane c goes to the owner of fine plane 2c + 1, the plane it
  coincides with), so that the planes P_l and R_l connect stay on one rank or
  its neighbour.  A level where some rank would own fewer than ``min_planes``
  planes is agglomerated on rank 0, and so is every coarser level (the coarse
  solve on level 1 always is).
* the planes each step reads from other ranks (``stencil_halo``,
  ``prolong_source``) and the coarse planes a rank's restriction contributes to
  (``restrict_target``), all derived from the operators' reach.
* ``Exchanger``: those transfers over a ``Transport``: planes copied from their
  owners, partial sums added into owned planes, and all-reduces of the section
  metadata (the largest and smallest block exponents that the kernels derive
  their fixed-point grids from).  No request messages: every rank derives from
  the plan what every other rank needs from it.

Arrays handed to the Exchanger are full-level arrays with the planes as the
first axis; a rank reads and writes only the planes the plan gives it.  The
exchanges are the ones a multi-GPU run of the CUDA kernels makes between
launches (one halo plane per neighbour per sweep for the stencil, the coarse
planes under a slab for P_l, partial coarse planes for R_l); with one GPU per
box they are exercised on CPU ranks (gloo) in the tests.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def planes_of(level: int) -> int:
    """Planes of level l (2^l - 1 interior nodes per axis)."""
    return (1 << level) - 1


def _parents(z: int) -> Tuple[int, ...]:
    """Coarse planes (0-based) that P_l reads for fine plane z (0-based): an
    even 1-based node number K = z + 1 coincides with coarse node K/2, an odd
    one lies between (K - 1)/2 and (K + 1)/2 (Kuhn edge interpolation)."""
    K = z + 1
    if K % 2 == 0:
        return (K // 2 - 1,)
    return ((K - 1) // 2 - 1, (K + 1) // 2 - 1)


class SlabPlan:
    """Ownership of the planes of levels 1..L_max by ranks 0..world-1."""

    def __init__(self, dim: int, L_max: int, world: int, min_planes: int = 2):
        if dim not in (2, 3) or L_max < 1 or world < 1 or min_planes < 1:
            raise ValueError("bad partition parameters")
        self.dim, self.L_max, self.world, self.min_planes = dim, L_max, world, min_planes
        self.bounds: Dict[int, List[int]] = {}
        self.distributed: Dict[int, bool] = {}
        n = planes_of(L_max)
        base, extra = divmod(n, world)
        b = [0]
        for r in range(world):
            b.append(b[-1] + base + (1 if r < extra else 0))
        dist = world > 1 and min(b[r + 1] - b[r] for r in range(world)) >= min_planes
        for level in range(L_max, 0, -1):
            n = planes_of(level)
            if level < L_max:
                fine = self.bounds[level + 1]
                b = [0] + [min(n, fine[r] // 2) for r in range(1, world)] + [n]
                dist = dist and level > 1 and min(b[r + 1] - b[r] for r in range(world)) >= min_planes
            if not dist:
                b = [0] + [n] * world
            self.bounds[level] = b
            self.distributed[level] = dist

    # ---------------------------------------------------------------- ownership
    def owned(self, level: int, rank: int) -> range:
        b = self.bounds[level]
        return range(b[rank], b[rank + 1])

    def owner(self, level: int, plane: int) -> int:
        b = self.bounds[level]
        for r in range(self.world):
            if b[r] <= plane < b[r + 1]:
                return r
        raise IndexError("plane %d outside level %d" % (plane, level))

    def active(self, level: int, rank: int) -> bool:
        return len(self.owned(level, rank)) > 0

    # ---------------------------------------------------------------- reach of the operators
    def stencil_halo(self, level: int, rank: int) -> List[int]:
        """Planes of `level` that the stencil on rank's slab reads but rank does not own."""
        own = self.owned(level, rank)
        if not own:
            return []
        n = planes_of(level)
        return [z for z in (own.start - 1, own.stop) if 0 <= z < n and z not in own]

    def prolong_source(self, level: int, rank: int, halo: bool = True) -> List[int]:
        """Planes of level - 1 that P_level reads for rank's fine planes (plus the
        stencil halo planes when halo is set), that rank does not own."""
        own = self.owned(level, rank)
        if not own or level < 2:
            return []
        fine = list(own) + (self.stencil_halo(level, rank) if halo else [])
        own_c = self.owned(level - 1, rank)
        nc = planes_of(level - 1)
        need = sorted({c for z in fine for c in _parents(z) if 0 <= c < nc})
        return [c for c in need if c not in own_c]

    def restrict_target(self, level: int, rank: int) -> List[int]:
        """Planes of level - 1 that R_level receives from rank's fine planes (owned
        or not); the ones rank does not own hold partial sums for their owners."""
        own = self.owned(level, rank)
        if not own or level < 2:
            return []
        nc = planes_of(level - 1)
        return sorted({c for z in own for c in _parents(z) if 0 <= c < nc})


# -------------------------------------------------------------------- transport
class Transport:
    """Point-to-point plane transfers and all-reduces between ranks."""

    rank: int
    world: int

    def exchange(self, sends: Dict[int, np.ndarray], recvs: Dict[int, Tuple[tuple, np.dtype]]
                 ) -> Dict[int, np.ndarray]:
        """Sends sends[q] to rank q and receives an array of shape/dtype recvs[q]
        from rank q, for every listed q, without deadlock."""
        raise NotImplementedError

    def allreduce(self, x: np.ndarray, op: str) -> np.ndarray:
        raise NotImplementedError


class TorchTransport(Transport):
    """Transport over torch.distributed (gloo on CPU, NCCL on GPUs)."""

    def __init__(self, group=None, device: str = "cpu"):
        import torch.distributed as dist
        self._dist = dist
        self.group = group
        self.device = device
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, sends, recvs):
        import torch
        dist = self._dist
        reqs, out = [], {}
        for q, (shape, dtype) in sorted(recvs.items()):
            buf = torch.empty(shape, dtype=_torch_dtype(dtype), device=self.device)
            out[q] = buf
            reqs.append(dist.irecv(buf, src=q, group=self.group))
        for q, arr in sorted(sends.items()):
            t = torch.from_numpy(np.ascontiguousarray(arr)).to(self.device)
            reqs.append(dist.isend(t, dst=q, group=self.group))
        for r in reqs:
            r.wait()
        return {q: b.cpu().numpy() for q, b in out.items()}

    def allreduce(self, x, op):
        import torch
        dist = self._dist
        t = torch.from_numpy(np.ascontiguousarray(x)).to(self.device)
        red = {"sum": dist.ReduceOp.SUM, "max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN}[op]
        dist.all_reduce(t, op=red, group=self.group)
        return t.cpu().numpy()


def _torch_dtype(dtype):
    import torch
    return {np.dtype(np.float64): torch.float64, np.dtype(np.int64): torch.int64,
            np.dtype(np.int32): torch.int32, np.dtype(np.uint8): torch.uint8,
            np.dtype(np.int8): torch.int8}[np.dtype(dtype)]


class LocalTransport(Transport):
    """A world of one rank (no peers)."""

    def __init__(self):
        self.rank, self.world = 0, 1

    def exchange(self, sends, recvs):
        if sends or recvs:
            raise ValueError("a single rank has no peers")
        return {}

    def allreduce(self, x, op):
        return np.asarray(x)


# -------------------------------------------------------------------- exchanges
class Exchanger:
    """The plan's transfers for one rank over a Transport."""

    def __init__(self, plan: SlabPlan, transport: Transport):
        if transport.world != plan.world:
            raise ValueError("transport and plan disagree on the number of ranks")
        self.plan, self.t = plan, transport
        self.rank = transport.rank

    def fetch(self, arr: np.ndarray, level: int, needs: Sequence[Sequence[int]]) -> None:
        """Copies into arr the planes needs[self.rank] from their owners (arr is the
        full level array of `level`); needs[q] lists the planes rank q reads
        (every rank passes the same lists, derived from the plan)."""
        me, plan = self.rank, self.plan
        own = plan.owned(level, me)
        sends = {}
        for q in range(plan.world):
            if q == me:
                continue
            mine = [z for z in needs[q] if z in own]
            if mine:
                sends[q] = arr[mine]
        recv_planes: Dict[int, List[int]] = {}
        for z in needs[me]:
            if z in own:
                continue
            recv_planes.setdefault(plan.owner(level, z), []).append(z)
        recvs = {q: ((len(zs),) + arr.shape[1:], arr.dtype) for q, zs in recv_planes.items()}
        got = self.t.exchange(sends, recvs)
        for q, zs in recv_planes.items():
            arr[zs] = got[q]

    def halo(self, arr: np.ndarray, level: int) -> None:
        """The stencil's halo planes of `level` from the neighbours."""
        self.fetch(arr, level, [self.plan.stencil_halo(level, q) for q in range(self.plan.world)])

    def prolong_source(self, arr_coarse: np.ndarray, level: int) -> None:
        """The planes of level - 1 that P_level reads on this rank (arr_coarse is
        the array of level - 1)."""
        self.fetch(arr_coarse, level - 1, [self.plan.prolong_source(level, q) for q in range(self.plan.world)])

    def reduce_to_owners(self, arr_coarse: np.ndarray, level: int) -> None:
        """Adds the partial sums this rank's restriction left in planes of level - 1
        it does not own into their owners' planes, and clears them here."""
        plan, me = self.plan, self.rank
        own = plan.owned(level - 1, me)
        sends, recv_from = {}, {}
        for q in range(plan.world):
            if q == me:
                continue
            out = [c for c in plan.restrict_target(level, me) if plan.owner(level - 1, c) == q]
            if out:
                sends[q] = arr_coarse[out]
            inc = [c for c in plan.restrict_target(level, q) if c in own]
            if inc:
                recv_from[q] = inc
        recvs = {q: ((len(cs),) + arr_coarse.shape[1:], arr_coarse.dtype) for q, cs in recv_from.items()}
        got = self.t.exchange(sends, recvs)
        for q, cs in recv_from.items():
            arr_coarse[cs] += got[q]
        for q, arr in sends.items():
            out = [c for c in plan.restrict_target(level, me) if plan.owner(level - 1, c) == q]
            arr_coarse[out] = 0

    def allreduce_exponents(self, emax: int, emin: int) -> Tuple[int, int]:
        """Section metadata over the ranks: the largest and the smallest block
        exponent of the nonzero blocks (-128 / 127 stand for "none")."""
        mx = self.t.allreduce(np.array([emax], dtype=np.int64), "max")
        mn = self.t.allreduce(np.array([emin], dtype=np.int64), "min")
        return int(mx[0]), int(mn[0])

    def allreduce_sum(self, x: float) -> float:
        return float(self.t.allreduce(np.array([x], dtype=np.float64), "sum")[0])
