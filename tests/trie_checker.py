"""Pointer trie following the paper's algorithms literally (test checker).

* ``build``            -- Algorithm 1 (BuildLCPIndex) + Algorithm 2
                          (ComputeSubtreeSizes), Sec. 5.2.
* ``descend``          -- the descent of Algorithm 3 (Query), Sec. 5.3.
* ``collect_bfs``      -- Algorithm 4 (CollectTopK): BFS from a node, posting
                          lists first, children in sorted symbol order.
* ``query_bfs``        -- Algorithm 3 + Algorithm 4 as printed: descend, then
                          CollectTopK from the deepest node reached.
* ``tal_by_trie``      -- the TAL bucket (items under q's depth-d node) ranked
                          by the Definition's order, from trie levels.
* ``topk_by_trie``     -- Definition "Top-k LCP Retrieval" (Sec. 2.1) evaluated
                          through the trie instead of by comparing sequences:
                          the items of T_{v_j} minus T_{v_{j+1}} along q's path
                          have LCP exactly j (descent lemma, App. A), and each
                          level is emitted in ascending item index.

This is a second, independent route to the oracle's answers; it never calls
the oracle.
"""
from __future__ import annotations

from collections import deque


class Node:
    __slots__ = ("children", "post", "size")

    def __init__(self):
        self.children = {}
        self.post = []
        self.size = 0


def build(S):
    """Algorithm 1: insert every sequence along its path; post(leaf) gets i."""
    root = Node()
    for i, s in enumerate(S):
        v = root
        for c in s:
            c = int(c)
            if c not in v.children:
                v.children[c] = Node()
            v = v.children[c]
        v.post.append(i)
    compute_subtree_sizes(root)
    return root


def compute_subtree_sizes(v):
    """Algorithm 2, iteratively (post-order) to avoid deep recursion."""
    order, stack = [], [v]
    while stack:
        u = stack.pop()
        order.append(u)
        stack.extend(u.children.values())
    for u in reversed(order):
        u.size = len(u.post) + sum(c.size for c in u.children.values())


def descend(root, q):
    """Algorithm 3 descent: returns the path [v_0=root, v_1, ..., v_d]."""
    path = [root]
    v = root
    for c in q:
        c = int(c)
        if c not in v.children:
            break
        v = v.children[c]
        path.append(v)
    return path


def items_in(v):
    out, stack = [], [v]
    while stack:
        u = stack.pop()
        out.extend(u.post)
        stack.extend(u.children.values())
    return out


def collect_bfs(v, k):
    """Algorithm 4 literally: BFS, posting lists, sorted children, stop at k."""
    result = []
    queue = deque([v])
    while len(result) < k and queue:
        u = queue.popleft()
        for i in u.post:
            result.append(i)
            if len(result) == k:
                return result
        for c in sorted(u.children):
            queue.append(u.children[c])
    return result


def topk_by_trie(root, q, k, N):
    """Top-k by the definition, computed from trie membership only."""
    path = descend(root, q)
    d = len(path) - 1
    out_ids, out_lcp = [], []
    inner = set()
    for j in range(d, -1, -1):
        level = sorted(set(items_in(path[j])) - inner)
        for i in level:
            if len(out_ids) < k:
                out_ids.append(i)
                out_lcp.append(j)
        inner |= set(level)
    while len(out_ids) < k:
        out_ids.append(-1)
        out_lcp.append(0)
    return out_ids, out_lcp


def query_bfs(root, q, k):
    """Algorithms 3 + 4: the first k items of T_v in BFS order, v the deepest
    node on q's path; every item of T_v has LCP = depth(v).  Padded."""
    path = descend(root, q)
    d = len(path) - 1
    ids = collect_bfs(path[-1], k)
    lcp = [d] * len(ids)
    return ids + [-1] * (k - len(ids)), lcp + [0] * (k - len(ids))


def tal_by_trie(root, q, k, d):
    """The TAL bucket is T_{v_d} (empty when q's path is shorter than d); its
    items at trie level j >= d along the path have LCP exactly j."""
    path = descend(root, q)
    D = len(path) - 1
    out_ids, out_lcp = [], []
    inner = set()
    for j in range(D, d - 1, -1):
        level = sorted(set(items_in(path[j])) - inner)
        for i in level:
            if len(out_ids) < k:
                out_ids.append(i)
                out_lcp.append(j)
        inner |= set(level)
    return out_ids + [-1] * (k - len(out_ids)), out_lcp + [0] * (k - len(out_lcp))

