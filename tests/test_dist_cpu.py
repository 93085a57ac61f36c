"""The N > 1 host logic on CPU: two gloo ranks (no GPU).

Replicas of the single-LP path report units of all ranks over the slowest
rank's time; a batch of LPs shards by problem (each problem on exactly one
rank, loads balanced by nonzeros) with no data-path collective.
"""
import os
import socket

import numpy as np
import pytest

from paper_2105_12715_gb300 import dist as pdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, weights, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = pdist.shard_by_weight(weights, world, rank)
        # replica timing: rank r processed 100 (r + 1) units in 2 + r seconds
        rate, slowest = pdist.job_throughput(100.0 * (rank + 1), 2.0 + rank)
        load = pdist.reduce_scalar(float(np.sum(np.asarray(weights)[mine])), "max")
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([rate, slowest, load] + mine, dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard(tmp_path):
    import torch.multiprocessing as mp

    rng = np.random.default_rng(3)
    weights = (np.exp(rng.uniform(np.log(750), np.log(300_000), 37))).round().tolist()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, weights, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    # units of all ranks / slowest rank's time, the same on every rank
    assert r0[0] == pytest.approx(300.0 / 3.0) and r1[0] == r0[0]
    assert r0[1] == r1[1] == 3.0
    # every problem on exactly one rank
    shards = [r0[3:].astype(int).tolist(), r1[3:].astype(int).tolist()]
    assert sorted(shards[0] + shards[1]) == list(range(len(weights)))
    # LPT bound: the heavier shard exceeds the mean load by at most the largest item
    total = float(np.sum(weights))
    assert r0[2] == r1[2] <= total / 2 + max(weights)


def test_shard_by_weight_single_process_cases():
    w = [5, 1, 1, 1, 1, 1]
    assert pdist.shard_by_weight(w, 1, 0) == list(range(6))
    a, b = pdist.shard_by_weight(w, 2, 0), pdist.shard_by_weight(w, 2, 1)
    assert a == [0] and b == [1, 2, 3, 4, 5]  # 5 vs 5
    assert pdist.shard_by_weight([], 3, 2) == []
    with pytest.raises(ValueError):
        pdist.shard_by_weight(w, 2, 2)
    assert pdist.reduce_scalar(4.0, "max") == 4.0  # not initialized: identity
