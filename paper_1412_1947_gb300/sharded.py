"""The method's data path sharded over ranks (one process per GPU): the exchanges that make
a sharded run give exactly the one-GPU result.

Points are sharded by index range: rank r holds the rows [lo_r, hi_r) of the data, and the
ranges ascend with r.  What each rank computes on its own rows -- its column bounds, its
share of the landmark L, its landmark distances, Lloyd on the subclusters it owns, its
part of the SSE -- comes from a `RankOps` object (on GPUs: the library's kernels on the
rank's own device).  This module holds only the coordination, as torch.distributed
collectives (NCCL between GPUs, gloo between CPU processes):

* scaling (Algorithm 1 step 1): all-reduce(min) and all-reduce(max) of the per-rank
  column bounds;
* every peel round (Algorithm 1 steps 2-5, Eq. 1 distances):
    - all-reduce(min) of the per-rank minima gives L exactly (min is order-free);
    - the N-th smallest key K is found by a radix select over the keys' 64-bit patterns
      (non-negative float64 values order like their bit patterns): per pass, every rank
      counts its keys under the current prefix into 2^11 digit bins, and one
      all-reduce(sum) gives the global histogram, from which every rank picks the same
      digit; six passes fix all 64 bits;
    - the keys equal to K are taken in ascending index: an all-gather of the per-rank
      counts of K, and rank r takes what is left of the quota after the ranks before it
      (which hold the lower indices);
  so the selection is the same set of N points as one GPU's, tie-break included;
* Lloyd (Algorithm 1 steps 3-4): subcluster s belongs to rank s mod W; its members, in
  ascending index, are the ranks' pieces in rank order; the pooled local centers are
  all-gathered in subcluster order, and the final Lloyd on them runs on every rank
  (deterministic, so every rank gets the same centers);
* the SSE (Algorithm 1 step 5): per-rank float64 partials, all-gathered and added in rank
  order, so that every rank and every run gets the same value (equal to the one-GPU sum up
  to the rounding of the association).

The transfers of subcluster members (gather_object to each owner) and of pooled centers
(all_gather_object) pickle host arrays, which fits the sizes this module is tested at; a
multi-GPU run would move rows with point-to-point copies into each owner's own memory.
Not measured on hardware.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# (shift, width) of the six radix passes over a 64-bit key, most significant first
PASSES = [(53, 11), (42, 11), (31, 11), (20, 11), (9, 11), (0, 9)]


class RankOps:
    """What one rank computes on its own rows (index range [lo, hi) of the data)."""

    lo: int
    hi: int
    d: int

    def column_bounds(self) -> tuple[np.ndarray, np.ndarray]:
        """Per-attribute min and max of this rank's raw rows (float64, d each)."""
        raise NotImplementedError

    def scale(self, mn: np.ndarray, mx: np.ndarray) -> None:
        """Min-max scale this rank's rows with the global bounds."""
        raise NotImplementedError

    def remaining(self) -> np.ndarray:
        """Global indices of this rank's rows not yet peeled, ascending (int64)."""
        raise NotImplementedError

    def landmark_min(self) -> np.ndarray:
        """Per-attribute min over this rank's remaining rows (+inf where none remain)."""
        raise NotImplementedError

    def keys(self, L: np.ndarray) -> np.ndarray:
        """The landmark keys of remaining(), as the uint64 bit patterns of the float64
        squared distances to L, in the order of remaining()."""
        raise NotImplementedError

    def take(self, positions: np.ndarray) -> None:
        """Remove the rows at these positions of remaining()."""
        raise NotImplementedError

    def rows(self, global_idx: np.ndarray) -> np.ndarray:
        """This rank's scaled rows at these global indices (float32, len x d)."""
        raise NotImplementedError

    def lloyd(self, seg_rows: np.ndarray, segment: int) -> np.ndarray:
        """Local Lloyd of one subcluster: its k_eff centers (float64)."""
        raise NotImplementedError

    def final_lloyd(self, pooled: np.ndarray) -> np.ndarray:
        """Lloyd on the pooled local centers (float32 rows): the final centers."""
        raise NotImplementedError

    def sse_partial(self, centers: np.ndarray) -> float:
        """Sum over this rank's rows, in index order, of the squared distance to the
        nearest final center (float64)."""
        raise NotImplementedError


def _allreduce(arr: np.ndarray, op, group=None) -> np.ndarray:
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(arr))
    dist.all_reduce(t, op=op, group=group)
    return t.numpy()


def _allgather_int(v: int, group=None) -> np.ndarray:
    import torch
    import torch.distributed as dist
    w = dist.get_world_size(group)
    out = [torch.zeros(1, dtype=torch.int64) for _ in range(w)]
    dist.all_gather(out, torch.tensor([v], dtype=torch.int64), group=group)
    return np.array([int(o.item()) for o in out], np.int64)


def global_bounds(ops: RankOps, group=None) -> tuple[np.ndarray, np.ndarray]:
    """Column min and max over all ranks' rows (exact)."""
    import torch.distributed as dist
    mn, mx = ops.column_bounds()
    return (_allreduce(np.asarray(mn, np.float64), dist.ReduceOp.MIN, group),
            _allreduce(np.asarray(mx, np.float64), dist.ReduceOp.MAX, group))


def landmark(ops: RankOps, group=None) -> np.ndarray:
    """L: the per-attribute minimum over every rank's remaining rows."""
    import torch.distributed as dist
    return _allreduce(np.asarray(ops.landmark_min(), np.float64), dist.ReduceOp.MIN, group)


def select_key(keys: np.ndarray, n_take: int, group=None) -> tuple[int, int]:
    """Radix select over all ranks' keys: (K, q) with K the n_take-th smallest key
    overall (1-based) and q the number of keys equal to K among the n_take smallest."""
    import torch.distributed as dist
    keys = np.asarray(keys, np.uint64)
    prefix, mask, need = 0, 0, int(n_take)
    for shift, width in PASSES:
        under = (keys & np.uint64(mask)) == np.uint64(prefix)
        digit = ((keys[under] >> np.uint64(shift)) & np.uint64((1 << width) - 1)).astype(np.int64)
        h = np.bincount(digit, minlength=1 << width).astype(np.int64)
        h = _allreduce(h, dist.ReduceOp.SUM, group)
        c = np.cumsum(h)
        b = int(np.searchsorted(c, need))          # first bin whose running count reaches need
        need -= int(c[b] - h[b])
        prefix |= b << shift
        mask |= ((1 << width) - 1) << shift
    return prefix, need


def split_quota(n_equal: int, q: int, group=None) -> int:
    """This rank's share of the q keys equal to K: what is left of q after the ranks
    before it (lower indices) have taken theirs."""
    import torch.distributed as dist
    counts = _allgather_int(n_equal, group)
    before = int(counts[:dist.get_rank(group)].sum())
    return max(0, min(n_equal, q - before))


def peel_round(ops: RankOps, N: int, group=None) -> np.ndarray:
    """One round of the peel: the global indices this rank contributes to the subcluster
    (ascending), removed from its remaining rows."""
    import torch.distributed as dist
    rem = ops.remaining()
    total = int(_allreduce(np.array([len(rem)], np.int64), dist.ReduceOp.SUM, group)[0])
    if total <= N:                                   # the last subcluster takes the rest
        ops.take(np.arange(len(rem)))
        return rem
    L = landmark(ops, group)
    keys = np.asarray(ops.keys(L), np.uint64)
    K, q = select_key(keys, N, group)
    eq = np.flatnonzero(keys == np.uint64(K))
    share = split_quota(len(eq), q, group)
    pos = np.sort(np.concatenate([np.flatnonzero(keys < np.uint64(K)), eq[:share]]))
    ops.take(pos)
    return rem[pos]


@dataclass
class ShardedResult:
    perm: np.ndarray          # n global indices in subcluster order (every rank)
    seg_off: np.ndarray       # S + 1
    local_centers: np.ndarray  # P x d float64, subcluster order
    final_centers: np.ndarray
    sse: float


def run(ops: RankOps, n: int, N: int, group=None) -> ShardedResult:
    """Scale, peel, local Lloyd on owned subclusters, pooled final Lloyd and SSE; every
    rank returns the same result."""
    import torch.distributed as dist
    w, r = dist.get_world_size(group), dist.get_rank(group)
    mn, mx = global_bounds(ops, group)
    ops.scale(mn, mx)
    # the peel: the rounds' pieces of this rank, then the subclusters' members merged
    pieces = []
    while int(_allreduce(np.array([len(ops.remaining())], np.int64), dist.ReduceOp.SUM, group)[0]) > 0:
        pieces.append(peel_round(ops, N, group))
    S = len(pieces)
    gathered = [None] * w
    dist.all_gather_object(gathered, pieces, group=group)
    segs = [np.concatenate([gathered[q][s] for q in range(w)]) for s in range(S)]
    seg_off = np.zeros(S + 1, np.int64)
    seg_off[1:] = np.cumsum([len(x) for x in segs])
    perm = np.concatenate(segs)
    assert len(perm) == n and np.array_equal(np.sort(perm), np.arange(n))
    # Lloyd: subcluster s on rank s mod w, its rows gathered from every rank in rank order
    got = None
    for q in range(w):
        recv = [None] * w if q == r else None
        dist.gather_object({s: ops.rows(pieces[s]) for s in range(S) if s % w == q}, recv, dst=q, group=group)
        if q == r:
            got = recv
    local = {s: ops.lloyd(np.concatenate([got[q][s] for q in range(w)]), s) for s in range(S) if s % w == r}
    allc = [None] * w
    dist.all_gather_object(allc, local, group=group)
    by_seg = {}
    for part in allc:
        by_seg.update(part)
    local_centers = np.concatenate([by_seg[s] for s in range(S)])
    final = ops.final_lloyd(local_centers.astype(np.float32))
    # SSE: per-rank partials added in rank order
    parts = [None] * w
    dist.all_gather_object(parts, float(ops.sse_partial(final)), group=group)
    sse = 0.0
    for p in parts:
        sse = sse + p
    return ShardedResult(perm, seg_off, local_centers, final, sse)
