"""Batched solves across ranks: instances are split, nothing of a solve is exchanged.

Instances of the batched form are independent problems.  So with one process
per GPU every rank builds and solves only its own instances, in one batched
graph launch, and no collective touches the data path.  The single exchange
is a final gather of the per-right-hand-side iteration counts and statuses to
rank 0.

Every rank computes the same assignment from the instance sizes alone
(greedy longest-processing-time: largest work first, each to the least
loaded rank, ties to the lowest index), so no message is needed to agree on
it.  The work of an instance is taken as dofs x right-hand sides: one
iteration costs O(n) per right-hand side, and the iteration counts of the
CSLP + deflation method grow only mildly with k.
"""
from __future__ import annotations

from typing import Sequence


def instance_work(n_dof: int, nrhs: int) -> int:
    """Work estimate of one instance: dofs x right-hand sides."""
    return int(n_dof) * int(nrhs)


def assign_instances(work: Sequence[int], world: int) -> list[list[int]]:
    """Instance indices per rank (each list ascending).

    Deterministic: every rank that calls it with the same `work` gets the
    same split.  Empty ranks are allowed (more ranks than instances)."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-int(work[i]), i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(work[i])
    return [sorted(p) for p in parts]


def my_instances(work: Sequence[int], rank: int, world: int) -> list[int]:
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    return assign_instances(work, world)[rank]


def gather_counts(local: dict, rank: int, world: int, dist=None, group=None):
    """Gather {instance: (iterations, statuses)} of every rank to rank 0.

    Returns the merged dict on rank 0 (keys ascending) and None elsewhere.
    Without a process group (`dist` None) it returns this rank's own counts.
    Host objects only: the solutions stay on each rank's GPU."""
    if dist is None or world == 1:
        return dict(sorted(local.items()))
    out = [None] * world if rank == 0 else None
    dist.gather_object(local, out, dst=0, group=group)
    if rank != 0:
        return None
    merged: dict = {}
    for part in out:
        for k, v in part.items():
            if k in merged:
                raise RuntimeError(f"instance {k} solved on two ranks")
            merged[k] = v
    return dict(sorted(merged.items()))


def solve_batched_sharded(problems, rank: int, world: int, dist=None, group=None, tol=1e-7, maxit=100, **ctx_kw):
    """Solve this rank's share of `problems` (a list of (Problem, nrhs)) in
    one batched launch and gather the iteration counts to rank 0.

    Returns (local solutions {instance: tensor (nrhs, n)}, gathered counts on
    rank 0 or None elsewhere).  Needs the CUDA library on every rank that has
    instances."""
    from .solver import from_problem, solve_batched
    import torch

    work = [instance_work((pr.n_el + pr.p - 2) ** pr.dim, nr) for pr, nr in problems]
    mine = my_instances(work, rank, world)
    sols: dict = {}
    local: dict = {}
    if mine:
        ctxs, rhs = [], []
        for i in mine:
            pr, nr = problems[i]
            c = from_problem(pr, **ctx_kw)
            ctxs.append(c)
            rhs.append(torch.stack([c.point_source(*s) for s in pr.sources[:nr]]))
        xs, its, sts, _ = solve_batched(ctxs, rhs, tol=tol, maxit=maxit)
        for j, i in enumerate(mine):
            sols[i] = xs[j]
            local[i] = ([int(v) for v in its[j]], [int(v) for v in sts[j]])
    return sols, gather_counts(local, rank, world, dist, group)
