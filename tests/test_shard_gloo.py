"""The multi-GPU path on CPU: two gloo ranks anneal their replica shards with
the oracle and reduce the best energy; the union equals one unsharded run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2608_25376_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, mode, replicas, out):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P = oracle.Problem(4, 4)
    first, count = shard.replica_range(rank, world, replicas, mode)
    res = oracle.anneal_structured(P, list(range(first, first + count)), 300, seed=4, n_threads=1)
    best = shard.reduce_best(int(res.best.min()) if count else np.iinfo(np.int64).max)
    out[rank] = (first, count, res.energies.tolist(), best)
    dist.destroy_process_group()


@pytest.mark.parametrize("mode,replicas", [("weak", 5), ("strong", 9)])
def test_two_rank_shards_equal_one_run(orc, mode, replicas):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, mode, replicas, out)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=180)
        assert p.exitcode == 0
    total = replicas * world if mode == "weak" else replicas
    full = orc.anneal_structured(orc.Problem(4, 4), total, 300, seed=4)
    got = []
    for r in range(world):
        first, count, E, best = out[r]
        got += E
        assert best == int(full.best.min())
    assert got == full.energies.tolist()


def test_replica_ranges():
    assert shard.replica_range(1, 4, 10, "weak") == (10, 10)
    ranges = [shard.replica_range(r, 4, 10, "strong") for r in range(4)]
    assert ranges == [(0, 3), (3, 3), (6, 2), (8, 2)]
    with pytest.raises(ValueError):
        shard.replica_range(4, 4, 10)
