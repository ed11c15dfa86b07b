"""Host-side sharding of independent systems (replicas) over the ranks of a
torch.distributed job: one process per GPU, each evaluating its own share of
the replicas with no collective on the data path.  Only the bookkeeping
crosses ranks (the slowest rank's time, the results gathered on rank 0), so
the same code runs under NCCL on GPUs and under gloo on CPU."""
import torch
import torch.distributed as dist


def shard_replicas(counts, world):
    """Assigns replica indices to `world` ranks, balancing the atoms: the
    largest replica goes to the least-loaded rank first (ties to the lower
    rank).  Deterministic, so every rank computes the same assignment
    without communicating.  Returns one sorted index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(counts)), key=lambda i: (-int(counts[i]), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(counts[i])
    return [sorted(s) for s in out]


def max_over_ranks(value, device=None):
    """The largest `value` over all ranks (the job's time is the slowest
    rank's); the value itself without a process group."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_replica_values(local_values, indices, n_rep, device=None):
    """Per-replica values computed by each rank for its `indices`, gathered
    into one tensor [n_rep] in replica order on every rank."""
    local_values = torch.as_tensor(local_values, dtype=torch.float64, device=device).reshape(-1)
    if len(indices) != local_values.numel():
        raise ValueError("one value per local replica")
    out = torch.full((n_rep,), float("nan"), dtype=torch.float64, device=device)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        out[torch.as_tensor(indices, dtype=torch.long, device=device)] = local_values
        return out
    # pad every rank's share to the longest so that one all_gather suffices
    world = dist.get_world_size()
    width = n_rep
    idx = torch.full((width,), -1, dtype=torch.long, device=device)
    val = torch.zeros(width, dtype=torch.float64, device=device)
    idx[:len(indices)] = torch.as_tensor(indices, dtype=torch.long, device=device)
    val[:len(indices)] = local_values
    all_idx = [torch.empty_like(idx) for _ in range(world)]
    all_val = [torch.empty_like(val) for _ in range(world)]
    dist.all_gather(all_idx, idx)
    dist.all_gather(all_val, val)
    for i, v in zip(all_idx, all_val):
        m = i >= 0
        out[i[m]] = v[m]
    return out
