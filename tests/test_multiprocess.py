"""Host-side N > 1 path of the benchmark on CPU: two `gloo` ranks.

The solve shards as independent replicas (one instance per rank, no
exchange inside a solve), so the only multi-rank logic is the launch
environment, the max-over-ranks step time with its barrier, the job-level
time per solve, and rank-0-only output.  These run without a GPU.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench._dist()
        step_ms, per_solve = bench.job_time(times[rank], ws, dist, device="cpu")
        q.put((rank, env, step_ms, per_solve))
    finally:
        dist.destroy_process_group()


def _run_ranks(times):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ws = len(times)
    procs = [ctx.Process(target=_worker, args=(r, ws, port, times, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_job_time_two_gloo_ranks():
    """Every rank sees the slowest rank's step time; the job retires two solves per step."""
    res = _run_ranks([3.0, 7.5])
    for rank, (ws, r, local), step_ms, per_solve in res:
        assert (ws, r, local) == (2, rank, rank)
        assert step_ms == 7.5
        assert per_solve == 7.5 / 2


def test_job_time_single_rank_is_identity():
    import bench
    assert bench.job_time(4.25, 1) == (4.25, 4.25)
    assert bench.job_time(4.25, 1, dist=None, device="cpu") == (4.25, 4.25)


def test_reference_arm_nonzero_rank_exits_without_work():
    """Under torchrun only rank 0 times the oracle and prints; the others exit 0 silently."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, env=env, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


@pytest.mark.parametrize("ws", [2])
def test_reference_arm_under_torchrun_prints_one_line(ws, tmp_path):
    """The reference arm launched as the N > 1 job is: one JSON line from rank 0 alone."""
    import json
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={ws}",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", str(ws),
           "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600, cwd=str(tmp_path))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["n_gpus"] == ws
    assert rec["higher_is_better"] is False
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["value"] == rec["cpu_baseline"]["value"] > 0


# ------------------------------------------------------------------ batched instances split by rank
def _cfg4_work():
    import workloads as W
    from paper_2010_10232_gb300.sharding import instance_work
    inst = W.config4(64)
    return [instance_work((pr.n_el + pr.p - 2) ** pr.dim, nr) for pr, nr in inst]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_instance_split_covers_and_balances(world):
    from paper_2010_10232_gb300.sharding import assign_instances, my_instances
    work = _cfg4_work()
    parts = assign_instances(work, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(work)))                       # every instance exactly once
    assert parts == assign_instances(list(work), world)         # same split on every rank
    assert all(my_instances(work, r, world) == parts[r] for r in range(world))
    loads = [sum(work[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(work)                 # list-scheduling bound


def test_instance_split_more_ranks_than_instances():
    from paper_2010_10232_gb300.sharding import assign_instances
    parts = assign_instances([5, 3], 4)
    assert parts == [[0], [1], [], []]
    with pytest.raises(ValueError):
        assign_instances([1], 0)


def _gather_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_2010_10232_gb300.sharding import my_instances, gather_counts
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        work = _cfg4_work()
        mine = my_instances(work, rank, ws)
        # stand-in results of this rank's batched launch: iterations i + 10, status 0 per right-hand side
        local = {i: ([i + 10] * 2, [0, 0]) for i in mine}
        q.put((rank, mine, gather_counts(local, rank, ws, dist)))
    finally:
        dist.destroy_process_group()


def test_gather_counts_two_gloo_ranks():
    """Each rank keeps its own instances; rank 0 alone receives every count, once."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, mine0, g0), (_, mine1, g1) = out
    assert g1 is None
    assert not set(mine0) & set(mine1) and len(mine0) + len(mine1) == 64
    assert list(g0) == list(range(64))
    assert all(g0[i] == ([i + 10] * 2, [0, 0]) for i in range(64))


def test_host_cpu_record():
    import bench
    info = bench.host_cpu()
    assert info["nproc"] == os.cpu_count() and info["machine"]
