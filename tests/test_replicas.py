"""The multi-rank path on CPU ranks (gloo, world size 2): replicas and the
sequence sharding of the momentum scan exchange nothing on the data path;
the timing and bookkeeping reductions (max of step times, sum of work) and
the shard assignment are checked here."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    from paper_2103_08804_gb300 import batch, replicas
    w, r, _ = replicas.init(backend="gloo")
    assert (w, r) == (ws, rank)
    specs = batch.momentum_scan_specs(L=4, alpha=1, chains=(8, 12), walkers=4, n_moments=2,
                                      n_iter=1)
    mine = replicas.shard_specs(specs, r, w)
    names = [None] * w
    dist.all_gather_object(names, [s.name for s in mine])
    t_max = replicas.max_over_ranks(w, 1.5 + r)
    n_all = replicas.sum_over_ranks(w, len(mine))
    seeds = [None] * w
    dist.all_gather_object(seeds, replicas.replica_seed(1000, r))
    replicas.barrier(w)
    if r == 0:
        out.put({"names": names, "all": [s.name for s in specs], "t_max": t_max,
                 "n_all": n_all, "seeds": seeds})
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_and_reduce():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(ws, _free_port(), q), nprocs=ws, start_method="spawn")
    res = q.get()
    shards = res["names"]
    flat = [n for sh in shards for n in sh]
    assert sorted(flat) == sorted(res["all"]) and len(set(flat)) == len(flat)  # disjoint, covering
    assert all(len(sh) > 0 for sh in shards)
    assert res["t_max"] == 2.5                        # the slowest rank's time
    assert res["n_all"] == len(res["all"])            # work summed over ranks
    assert len(set(res["seeds"])) == ws               # independent replica streams


def test_single_rank_is_the_identity():
    from paper_2103_08804_gb300 import replicas
    assert replicas.max_over_ranks(1, 3.0) == 3.0
    assert replicas.sum_over_ranks(1, 4.0) == 4.0
    assert replicas.shard_specs([1, 2, 3], 0, 1) == [1, 2, 3]
