"""The N > 1 path of bench.py on CPU: two gloo ranks, as torchrun launches them (RANK, WORLD_SIZE,
LOCAL_RANK, MASTER_ADDR=127.0.0.1).  Fields are sharded across ranks with no collective on the
data path (weak scaling): the shards are disjoint, the time is the maximum over ranks, the value
counts the fields of every rank, and the reference arm runs on rank 0 only."""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, B, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    from paper_0807_4494_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cpu = torch.device("cpu")
    r, w, _ = bench.dist_env()
    L, s = 12, 1
    flm = inputs.coeffs(L, s, B, seed=bench.rank_seed(r, B))
    shards = [None] * w
    dist.all_gather_object(shards, (r, flm))
    t = bench.max_over_ranks(10.0 * (r + 1), w, cpu)
    bench.barrier(w, cpu)
    value = bench.throughput(w, B, 5, t)
    # the reference arm prints on rank 0 only and the other ranks return without work
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        ns = type("A", (), {"L": 8, "s": 0, "batch": B, "steps": 1, "warmup": 0})()
        bench.run_reference(ns)
    q.put((r, shards, t, value, out.getvalue()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_fields_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, B, world = _free_port(), 3, 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, B, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, shards, t, value, printed = q.get(timeout=240)
        res[r] = (shards, t, value, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = dict(res[0][0])
    # disjoint shards: rank 1's fields are the seeds after rank 0's
    assert not np.array_equal(shards[0], shards[1])
    from paper_0807_4494_gb300 import inputs
    both = inputs.coeffs(12, 1, 2 * B, seed=0)
    assert np.array_equal(np.concatenate([shards[0], shards[1]]), both)
    for r in range(world):
        assert res[r][1] == 20.0                                  # max over ranks
        assert res[r][2] == pytest.approx(world * B * 5 / 0.020)  # all ranks' fields / slowest time
    assert '"impl": "reference"' in res[0][3]
    assert res[1][3] == ""
