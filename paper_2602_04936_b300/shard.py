"""Sharded index over the ranks of a process group (one GPU per rank).

The rows are partitioned by original-id range: rank r holds rows
[bases[r], bases[r] + counts[r]) and builds its own index over them.  A batch
of queries is answered by every rank against its shard; the P answers (local
ids) are all-gathered and merged by ``lcp_shard_merge`` into the global top k,
which is byte-identical to the answer of one index over all rows (the shard
answers are ordered by (LCP desc, id asc) and global ids are unique).

The one exchange is the all-gather of Q x k x 5 bytes per shard.  The search
and merge callables default to this package's CUDA entry points; tests of the
process-group plumbing on CPU (gloo) pass their own.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_bounds(N: int, world: int):
    """Contiguous id ranges, as equal as possible: (bases, counts)."""
    q, r = divmod(N, world)
    counts = [q + (1 if i < r else 0) for i in range(world)]
    bases = [sum(counts[:i]) for i in range(world)]
    return bases, counts


class ShardedIndex:
    def __init__(self, local_rows: torch.Tensor, N: int, max_k: int = 128, group=None,
                 search=None, merge=None, build=None):
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.bases, self.counts = shard_bounds(N, self.world)
        if local_rows.shape[0] != self.counts[self.rank]:
            raise ValueError("rank %d holds %d rows, its shard has %d"
                             % (self.rank, local_rows.shape[0], self.counts[self.rank]))
        if search is None or merge is None or build is None:
            from . import lcp_index_build, lcp_shard_merge, lcp_topk_batch
            build = build or (lambda rows: lcp_index_build(rows, max_k=max_k))
            search = search or lcp_topk_batch
            merge = merge or lcp_shard_merge
        self._search, self._merge = search, merge
        self.index = build(local_rows)

    def topk(self, queries: torch.Tensor, k: int):
        """Global top k of the same queries on every rank: ([Q, k] ids, [Q, k] lcp)."""
        ids, lcp = self._search(self.index, queries, k)
        if self.world == 1:
            return self._merge(ids.unsqueeze(0), lcp.unsqueeze(0), self.bases)
        Q, k = ids.shape
        # gathered shard-major: rows [r*Q, (r+1)*Q) come from rank r
        all_ids = torch.empty((self.world * Q, k), dtype=ids.dtype, device=ids.device)
        all_lcp = torch.empty((self.world * Q, k), dtype=lcp.dtype, device=lcp.device)
        dist.all_gather_into_tensor(all_ids, ids.contiguous(), group=self.group)
        dist.all_gather_into_tensor(all_lcp, lcp.contiguous(), group=self.group)
        return self._merge(all_ids.view(self.world, Q, k), all_lcp.view(self.world, Q, k), self.bases)
