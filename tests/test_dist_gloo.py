"""The multi-rank path on CPU: two gloo ranks merge per-level accumulators of
disjoint sample shards and take the maximum time over ranks, as a replicated
or sharded run on several GPUs does (no GPU needed)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

from oracle import mlmc as o_mlmc   # noqa: E402

WORLD = 2
LEVELS = 3


def _shard(rank, level):
    """Rank `rank`'s level-`level` differences Y (deterministic, sizes differ per rank)."""
    g = np.random.default_rng(1000 * rank + level)
    return g.standard_normal(50 + 37 * rank + 11 * level) * 10.0 ** (-level - 2) + 0.03 / (level + 1)


def _local_acc(M, Y):
    """This rank's accumulator of Y, built by merging single-sample accumulators."""
    acc = M.capi.mlmc_acc()
    for y in Y:
        one = M.capi.mlmc_acc()
        one.n, one.mean, one.m2, one.sum, one.sumsq = 1, float(y), 0.0, float(y), float(y) * float(y)
        M.mlmc_acc_merge(acc, one)
    return acc


def _worker(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import paper_2503_05533_gb300 as M
        from paper_2503_05533_gb300 import replicas
        accs = [_local_acc(M, _shard(rank, l)) for l in range(LEVELS)]
        merged = replicas.merge_over_ranks(dist, accs)
        t = replicas.max_over_ranks(dist, 1.5 + rank)
        np.save(os.path.join(out_dir, "rank%d.npy" % rank),
                np.array([[a.n, a.mean, a.m2] for a in merged] + [[t, 0.0, 0.0]]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_merge_accumulators_and_time(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, start_method="spawn", join=True)
    res = [np.load(os.path.join(str(tmp_path), "rank%d.npy" % r)) for r in range(WORLD)]
    # every rank holds the same bits
    assert np.array_equal(res[0], res[1])
    for level in range(LEVELS):
        Y = np.concatenate([_shard(r, level) for r in range(WORLD)])
        m, v = o_mlmc.mean_var(Y)
        n, mean, m2 = res[0][level]
        assert n == len(Y)
        assert abs(mean - m) <= 1e-15 * abs(m) + 1e-18
        assert abs(m2 / n - v) <= 1e-12 * v
    assert res[0][LEVELS][0] == 2.5    # max over ranks of 1.5 + rank
