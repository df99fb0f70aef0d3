"""Multi-rank host logic on CPU: two gloo ranks on 127.0.0.1 (the GPU runs use
the same code over NCCL, one rank per GPU)."""
import os
import socket
import subprocess
import sys

import pytest

from paper_2010_01628_gb300 import inputs
from paper_2010_01628_gb300.ranks import Ranks, partition_domains

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        r = Ranks(device="cpu")
        r.barrier()
        mx = r.max_over_ranks(1.5 + rank)
        sm = r.sum_over_ranks(rank + 1)
        cells = [n ** 3 for n, _ in inputs.hartmann_batch(64, seed=2)]
        mine = partition_domains(cells, world)[rank]
        shares = [None] * world
        dist.all_gather_object(shares, mine)
        q.put((rank, r.world, mx, sm, shares))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_sweep_and_reduce_timings():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cells = [n ** 3 for n, _ in inputs.hartmann_batch(64, seed=2)]
    for rank, world, mx, sm, shares in got:
        assert world == 2
        assert mx == 2.5 and sm == 3.0
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(64))  # every domain on exactly one rank
        loads = [sum(cells[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(cells)
    assert got[0][4] == got[1][4]  # both ranks computed the same partition


def test_partition_is_balanced_and_deterministic():
    cells = [n ** 3 for n, _ in inputs.hartmann_batch(64, seed=2)]
    for world in (1, 2, 3, 4, 8):
        shares = partition_domains(cells, world)
        assert shares == partition_domains(cells, world)
        assert sorted(i for s in shares for i in s) == list(range(64))
        loads = [sum(cells[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(cells)
    assert partition_domains(cells, 1) == [list(range(64))]
    with pytest.raises(ValueError):
        partition_domains(cells, 0)


def test_single_rank_reductions_are_identity(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    r = Ranks()
    assert not r.distributed and r.max_over_ranks(3.25) == 3.25 and r.sum_over_ranks(2) == 2.0
    r.barrier()


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the oracle arm is timed once: ranks other than 0 exit 0
    at once, printing nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
