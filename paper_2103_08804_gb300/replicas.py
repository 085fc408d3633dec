"""Multi-GPU plan: replicas and sequence sharding, no data-path collective.

The projection steps of one sequence run on one GPU; several GPUs either run
independent replicas (bench.py: one sequence per rank, its own seed) or
split the sequences of a momentum scan (shard_specs).  Nothing is exchanged
on the data path; the only collectives are the timing and bookkeeping
reductions below (max of the step times, sums of the work done), which run
over NCCL on GPUs and over gloo in the CPU tests.
"""

import os

import torch


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend=None):
    """Join the process group when world_size > 1 (NCCL with CUDA, else
    gloo); returns (world_size, rank, local_rank)."""
    ws, rank, local = env()
    if ws > 1:
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return ws, rank, local


def _device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    """The largest x over ranks (whole-job time = the slowest rank's)."""
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, x):
    """The sum of x over ranks (work done by the whole job)."""
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_seed(base, rank):
    """Seed of rank's replica: distinct random streams per rank."""
    return base + 17 * rank


def shard_specs(specs, rank, ws):
    """Round-robin share of the sequences for this rank (disjoint, covering)."""
    return list(specs[rank::ws])
