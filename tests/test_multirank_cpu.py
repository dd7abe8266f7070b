"""Multi-rank paths on CPU with the gloo backend (world size 2).

* The sharded index: rows partitioned by id range, each rank answers the same
  queries against its shard, the answers are all-gathered and merged.  Here
  the per-shard search is the oracle and the merge a plain key sort (the CUDA
  kernels need a GPU); what is under test is the partition, the gather order
  and the id offsets -- the merged answer must equal the oracle over all rows.
* The bench's N > 1 plumbing: barrier and the max over ranks of the timed
  region."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _key_merge(ids, lcp, bases):
    """Plain reference merge: the k smallest (255 - lcp, global id) keys."""
    P, Q, k = ids.shape
    out_i = np.full((Q, k), -1, np.int32)
    out_l = np.zeros((Q, k), np.uint8)
    for q in range(Q):
        keys = sorted((255 - int(lcp[s, q, j]), int(bases[s]) + int(ids[s, q, j]))
                      for s in range(P) for j in range(k) if ids[s, q, j] >= 0)[:k]
        for j, (a, g) in enumerate(keys):
            out_i[q, j], out_l[q, j] = g, 255 - a
    return torch.from_numpy(out_i), torch.from_numpy(out_l)


def _sharded_worker(rank, world, port, outdir):
    _init(rank, world, port)
    try:
        from paper_2602_04936_b300.shard import ShardedIndex, shard_bounds
        S, Qs, _ = W.make_dataset("tree16_u8", N=700, Q=64)
        bases, counts = shard_bounds(len(S), world)
        local = torch.from_numpy(S[bases[rank]:bases[rank] + counts[rank]])

        def search(index, queries, k):
            ids, lc = oracle.topk_batch(index, queries.numpy(), k)
            return torch.from_numpy(ids), torch.from_numpy(lc)

        def merge(ids, lcp, b):
            return _key_merge(ids.numpy(), lcp.numpy(), b)

        sh = ShardedIndex(local, len(S), search=search, merge=merge, build=lambda rows: rows.numpy())
        ids, lc = sh.topk(torch.from_numpy(Qs), 10)
        np.save(os.path.join(outdir, "ids%d.npy" % rank), ids.numpy())
        np.save(os.path.join(outdir, "lcp%d.npy" % rank), lc.numpy())
    finally:
        dist.destroy_process_group()


def test_shard_bounds():
    from paper_2602_04936_b300.shard import shard_bounds
    for N, w in [(10, 3), (7, 7), (5, 8), (1_000_000, 4), (0, 2)]:
        b, c = shard_bounds(N, w)
        assert sum(c) == N and b[0] == 0 and all(b[i] + c[i] == b[i + 1] for i in range(w - 1))
        assert max(c) - min(c) <= 1


def test_sharded_topk_two_ranks_equals_oracle(tmp_path):
    world = 2
    mp.spawn(_sharded_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    S, Qs, _ = W.make_dataset("tree16_u8", N=700, Q=64)
    want_i, want_l = oracle.topk_batch(S, Qs, 10)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / ("ids%d.npy" % r)), want_i)
        assert np.array_equal(np.load(tmp_path / ("lcp%d.npy" % r)), want_l)


def _bench_worker(rank, world, port, outdir):
    _init(rank, world, port)
    try:
        import bench
        bench.barrier(world)
        m = bench.max_over_ranks(1.5 + rank, world)
        with open(os.path.join(outdir, "max%d.txt" % rank), "w") as f:
            f.write(repr(m))
    finally:
        dist.destroy_process_group()


def test_bench_max_over_ranks_two_ranks(tmp_path):
    world = 2
    mp.spawn(_bench_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        assert float(open(tmp_path / ("max%d.txt" % r)).read()) == 2.5
