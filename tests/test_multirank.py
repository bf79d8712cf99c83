"""The N > 1 launch path of bench.py on the CPU (gloo, world size 2; the GPUs of this run are
one per call): every rank advances its own instance and its share of the 64-instance batch, so
the only collective is the timing reduction, which takes the maximum over ranks; the batch
split is computed alike on every rank without communication; under torchrun the reference arm
runs on rank 0 alone, which prints one JSON line, while the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, REPO)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.rank_env()
        got = bench.max_over_ranks(1.25 + rank, "cpu")       # rank 1 is the slower one
        q.put((r, w, loc, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, w, loc) for r, w, loc, _ in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(got == 2.25 for *_, got in res)


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, REPO)
    import torch
    import torch.distributed as dist
    from paper_2202_07989_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [p["n"] ** 2 for p in W.batched_params(64)]
        mine = W.shard(sizes, world, rank)
        # every rank's share, gathered: the ranks agree on the split without exchanging data
        mask = torch.zeros(64, dtype=torch.int64)
        mask[mine] = 1
        masks = [torch.zeros(64, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(masks, mask)
        q.put((rank, mine, [m.tolist() for m in masks]))
    finally:
        dist.destroy_process_group()


def test_batch_split_across_gloo_ranks():
    """Two gloo ranks split the 64-instance batch as the benchmark does at N > 1: the shares
    are disjoint, cover every instance, and each rank's share is the one the other ranks
    compute for it (the split needs no communication)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [set(mine) for _, mine, _ in res]
    assert shares[0].isdisjoint(shares[1]) and shares[0] | shares[1] == set(range(64))
    for rank, mine, masks in res:
        for r, m in enumerate(masks):
            assert {i for i in range(64) if m[i]} == shares[r]


def test_max_over_ranks_without_a_group_is_the_value():
    sys.path.insert(0, REPO)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5


def test_reference_arm_under_torchrun():
    """python -m torch.distributed.run --nproc-per-node 2 bench.py --impl reference: one JSON
    line from rank 0 with the launch's n_gpus, exit status 0 on both ranks."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=REPO, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
