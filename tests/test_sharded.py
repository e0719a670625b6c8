"""The sharded form of the method (index-range shards, one process per rank) against the
one-rank oracle: world_size 2 and 3 gloo ranks on CPU, tie-heavy inputs.

Each rank's own arithmetic (keys, Lloyd of the subclusters it owns, its SSE part) is the
oracle's, restated per shard here; what is under test is the exchange logic of
paper_1412_1947_gb300.sharded -- the all-reduce of L, the histogram all-reduce of the
radix select, the rank-ordered split of the boundary quota, the gathering of subcluster
members and pooled centers, and the rank-ordered SSE sum (Algorithm 1 steps 1-5).  The
merged partition and the centers must equal the oracle's bit for bit; the SSE equals it up
to the association of the sum and is the same on every rank."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1412_1947_gb300 import sharded


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleRank(sharded.RankOps):
    """A rank's rows [lo, hi) of the data, computed with the oracle's arithmetic."""

    def __init__(self, raw, lo, hi, local_k, final_k, iters, seed):
        self.raw, self.lo, self.hi, self.d = raw, lo, hi, raw.shape[1]
        self.local_k, self.final_k, self.iters, self.seed = local_k, final_k, iters, seed
        self.x = None
        self.rem = np.arange(lo, hi, dtype=np.int64)

    def column_bounds(self):
        part = self.raw[self.lo:self.hi].astype(np.float64)
        return part.min(axis=0), part.max(axis=0)

    def scale(self, mn, mx):
        # scaling a row needs only the global bounds: the oracle's scaling of all rows,
        # this rank's slice (and the bounds the exchange found must be the oracle's)
        full, omn, omx = oracle.scale(self.raw)
        np.testing.assert_array_equal(mn, omn)
        np.testing.assert_array_equal(mx, omx)
        self.x = full[self.lo:self.hi]

    def remaining(self):
        return self.rem

    def landmark_min(self):
        if len(self.rem) == 0:
            return np.full(self.d, np.inf)
        return self.x[self.rem - self.lo].astype(np.float64).min(axis=0)

    def keys(self, L):
        # float64, ascending attributes, no FMA: sum_j ((double)x_j - L_j)^2
        v = self.x[self.rem - self.lo].astype(np.float64)
        acc = np.zeros(len(v))
        for j in range(self.d):
            t = v[:, j] - L[j]
            acc = acc + t * t
        return acc.view(np.uint64)

    def take(self, positions):
        self.rem = np.delete(self.rem, positions)

    def rows(self, global_idx):
        return self.x[np.asarray(global_idx, np.int64) - self.lo]

    def lloyd(self, seg_rows, segment):
        return oracle.lloyd_seeded(seg_rows, self.local_k, self.iters, self.seed, stage=0, segment=segment)[0]

    def final_lloyd(self, pooled):
        return oracle.lloyd_seeded(pooled, self.final_k, self.iters, self.seed, stage=1, segment=0)[0]

    def sse_partial(self, centers):
        _, best, _ = oracle.assign(self.x, centers)
        s = 0.0
        for v in best:
            s = s + float(v)
        return s


def _rank_main(rank, world, port, bounds, case, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        raw, N, lk, fk, T, seed = case
        ops = OracleRank(raw, bounds[rank], bounds[rank + 1], lk, fk, T, seed)
        got = sharded.run(ops, len(raw), N)
        ref = oracle.two_level(raw, N, lk, fk, T, seed=seed)
        np.testing.assert_array_equal(got.perm, ref.perm)
        np.testing.assert_array_equal(got.seg_off, ref.seg_off)
        np.testing.assert_array_equal(got.local_centers, ref.local_centers)
        np.testing.assert_array_equal(got.final_centers, ref.final_centers)
        assert abs(got.sse - ref.sse) <= 1e-12 * ref.sse, (got.sse, ref.sse)
        sses = [None] * world
        dist.all_gather_object(sses, got.sse)
        assert len(set(sses)) == 1
        dist.destroy_process_group()
        q.put((rank, "ok"))
    except BaseException as e:            # reported to the parent, which fails the test
        q.put((rank, repr(e)))


def _run_ranks(case, bounds):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = len(bounds) - 1
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, bounds, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert all(v == "ok" for v in out.values()), out


def _tie_heavy(n, d, levels, seed):
    # attributes on a few levels: many points share a landmark distance, and the boundary
    # key of a round is held by points of several ranks
    rng = np.random.default_rng(seed)
    return rng.integers(0, levels, size=(n, d)).astype(np.float32)


def test_sharded_peel_selects_the_same_points_on_two_ranks():
    raw = _tie_heavy(2000, 3, 3, seed=5)
    _run_ranks((raw, 230, 6, 4, 5, 17), [0, 900, 2000])


def test_sharded_run_on_three_uneven_ranks():
    raw = _tie_heavy(1500, 4, 4, seed=6)
    raw[::7] = raw[3]                      # exact duplicates spread over every rank
    _run_ranks((raw, 200, 5, 6, 4, 23), [0, 1000, 1100, 1500])


def test_radix_passes_cover_the_key():
    # the six digit fields tile bits 0..63 with no gap and no overlap
    bits = np.zeros(64, int)
    for shift, width in sharded.PASSES:
        bits[shift:shift + width] += 1
    assert (bits == 1).all()
