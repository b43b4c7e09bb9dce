"""Independent replicas across GPUs: channels are independent solves, so
N ranks run N channels with no data-path collective.  Only the timing is
combined: a barrier before and after the timed region and the maximum of
the per-rank times (the job is as slow as its slowest rank)."""
import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend, device=None):
    """Initialise torch.distributed for world_size > 1; returns the module or None."""
    ws, _, _ = env()
    if ws <= 1:
        return None
    import torch.distributed as dist
    if device is not None:
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)
    return dist


def replica_seed(base, rank):
    """Seed of rank's input field: every rank runs its own channel."""
    return base + rank


def max_over_ranks(value, dist, device="cpu"):
    """Maximum of a per-rank scalar over all ranks (the value itself alone)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, seconds_local, dist, device="cpu"):
    """Whole-job rate: all ranks' units over the slowest rank's time."""
    ws = dist.get_world_size() if dist is not None else 1
    slowest = max_over_ranks(seconds_local, dist, device)
    return ws * units_per_rank / slowest, slowest
