"""The multi-rank path of the replica batch on CPU: two gloo ranks shard the
64 replicas (balanced by atoms, every replica exactly once, no
communication needed to agree), gather per-replica results in replica order
and take the slowest rank's time.  No GPU: the same host code runs under
NCCL in bench.py."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from synth import replica_sizes


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1402_7216_gb300.shard import gather_replica_values, max_over_ranks, shard_replicas
        counts = replica_sizes(64)
        shards = shard_replicas(counts, world)
        mine = shards[rank]
        vals = [0.5 * counts[i] + i for i in mine]            # a per-replica result
        full = gather_replica_values(vals, mine, len(counts))
        t = max_over_ranks(10.0 + 3.0 * rank)
        out.put((rank, shards, mine, full.tolist(), t))
    finally:
        dist.destroy_process_group()


def test_shard_replicas_balanced_and_complete():
    from paper_1402_7216_gb300.shard import shard_replicas
    counts = replica_sizes(64)
    for world in (1, 2, 3, 8):
        sh = shard_replicas(counts, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(64))
        loads = [sum(counts[i] for i in s) for s in sh]
        assert max(loads) <= sum(counts) / world + max(counts)   # greedy bound
        assert max(loads) / (sum(loads) / world) < 1.1
    assert shard_replicas(counts, 2) == shard_replicas(list(counts), 2)   # deterministic


def test_two_gloo_ranks_shard_gather_and_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    counts = replica_sizes(64)
    want = [0.5 * counts[i] + i for i in range(64)]
    (_, sh0, m0, f0, t0), (_, sh1, m1, f1, t1) = res
    assert sh0 == sh1                                        # both ranks agree without talking
    assert sorted(m0 + m1) == list(range(64)) and not set(m0) & set(m1)
    assert f0 == pytest.approx(want) and f1 == pytest.approx(want)
    assert t0 == t1 == 13.0                                  # the slower rank's time


def test_single_process_helpers_without_a_process_group():
    from paper_1402_7216_gb300.shard import gather_replica_values, max_over_ranks
    assert max_over_ranks(3.5) == 3.5
    out = gather_replica_values([10.0, 30.0], [1, 3], 4)
    assert out[1].item() == 10.0 and out[3].item() == 30.0
    assert out[0].isnan().item() and out[2].isnan().item()
    with pytest.raises(ValueError):
        gather_replica_values([1.0], [0, 1], 4)
