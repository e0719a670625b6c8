"""The headline workload at full size (2^20 points, d=16, 256 subclusters of 4096, 64 local
centers, 25 iterations, final k=64), run the way bench.py times it (pipeline recorded
into a CUDA graph, device-resident input), against the oracle on the same seeded input."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import synth
from tests.parity import TIE_TOL, compare, run_gpu
import oracle

pytestmark = pytest.mark.gpu


def test_medium_workload_full_size():
    w = synth.MEDIUM
    raw = w.points()
    seed = 12345
    g = run_gpu(raw, w.N, w.local_k, w.final_k, w.iters, seed, graph=True, runs=2, device_points=True)
    o = oracle.two_level(raw, w.N, w.local_k, w.final_k, w.iters, seed, select_peel=True,
                         force_local=g.trace_local, force_final=g.trace_final, tie_tol=TIE_TOL)
    stats = compare(g, o)
    print("full-size parity:", stats)


def test_peel_partition_with_slices_beyond_the_key_cache():
    # 2^21 points: every CTA's slice exceeds the 4096 keys kept in shared memory, so the
    # round's keys go through the global per-slice array instead
    import oracle
    from paper_1412_1947_gb300 import binding as B
    raw = synth.mixture(1 << 21, 4, 16, outlier_frac=0.01, seed=8800)
    with B.Job(raw) as j:
        j.steps(1 << 17, 4, 4, 1, 3)
        perm, off = j.partition()
        x = j.scaled()
    operm, ooff, _ = oracle.peel(x, 1 << 17, select=True)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)


def test_peel_partition_with_dense_float32_keys():
    # 2^22 points in 64 attributes, subclusters of 2^20: near the cut-off several points
    # share each float32 key, so the float32 tight set outgrows shared memory and every
    # round settles its band in float64 across the grid (the wide-band selection)
    from paper_1412_1947_gb300 import binding as B
    raw = synth.mixture(1 << 22, 64, 64, seed=8801)
    with B.Job(raw) as j:
        j.steps(1 << 20, 2, 2, 1, 3)
        perm, off = j.partition()
        x = j.scaled()
    operm, ooff, _ = oracle.peel(x, 1 << 20, select=True)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)


def test_uneven_batch_full_size_sampled():
    # the 2048-instance uneven batch as the bench runs it (graph-recorded, one launch per
    # iteration over every instance), 3 iterations with label traces; a seeded sample of
    # instances, the smallest and the largest among them, against the oracle
    from tests.parity import compare_batch, run_gpu_batch
    parts, ks = synth.uneven_batch()
    g = run_gpu_batch(parts, ks, 3, seed=777)
    sizes = np.array([len(p) for p in parts])
    rng = np.random.default_rng(5)
    pick = set(rng.choice(len(parts), 10, replace=False).tolist()) | {int(sizes.argmin()), int(sizes.argmax())}
    stats = compare_batch(g, parts, ks, 3, seed=777, only=sorted(pick))
    print("uneven batch, sampled instances:", stats)


def _delta64(rows, L):
    # the peel's distance exactly as defined: float64, attributes summed in ascending order,
    # one rounding per operation
    acc = np.zeros(len(rows), np.float64)
    for j in range(rows.shape[1]):
        t = rows[:, j].astype(np.float64) - L[j]
        acc = acc + t * t
    return acc


def test_large_workload_full_size_properties():
    # 2^24 points in 64 attributes, subclusters of 65536, 256 local centers, final k = 1024,
    # 25 iterations, run as bench.py runs it; too large for the oracle end to end, so
    # properties that fix the result: a complete partition into equal subclusters, the
    # selection property of sampled rounds with exact float64 distances, and the final
    # labels of a sample equal to the float64 nearest center (near ties excepted)
    from paper_1412_1947_gb300 import binding as B
    w = synth.LARGE
    raw = w.points()
    with B.Job(raw) as j:
        j.option(B.PSCL_OPT_GRAPH)
        j.run(w.N, w.local_k, w.final_k, w.iters, 11)
        perm, off = j.partition()
        x = j.scaled()
        fc, lab, sse = j.result()
    del raw
    n, N = w.n, w.N
    assert np.array_equal(off, np.arange(0, n + 1, N))
    assert np.array_equal(np.sort(perm), np.arange(n))
    for r in (1, 100, 254):
        seg = perm[r * N:(r + 1) * N]
        later = perm[(r + 1) * N:]
        L = np.minimum(x[seg].min(0), np.min([x[later[i:i + (1 << 20)]].min(0)
                                              for i in range(0, len(later), 1 << 20)], axis=0)).astype(np.float64)
        ds = _delta64(x[seg], L)
        worst = max(zip(ds.tolist(), seg.tolist()))
        for i in range(0, len(later), 1 << 20):
            chunk = later[i:i + (1 << 20)]
            dl = _delta64(x[chunk], L)
            k = int(np.argmin(dl))
            best = min(zip(dl[dl == dl[k]].tolist(), chunk[dl == dl[k]].tolist()))
            assert worst < best, (r, worst, best)
    rng = np.random.default_rng(3)
    pick = rng.choice(n, 50000, replace=False)
    xs = x[pick].astype(np.float64)
    c = fc.astype(np.float64)
    dist = (xs ** 2).sum(1)[:, None] - 2.0 * xs @ c.T + (c ** 2).sum(1)[None, :]
    two = np.argpartition(dist, 1, axis=1)[:, :2]
    rows = np.arange(len(pick))[:, None]
    two = np.take_along_axis(two, np.argsort(dist[rows, two], axis=1, kind="stable"), axis=1)
    b1 = dist[rows[:, 0], two[:, 0]]
    b2 = dist[rows[:, 0], two[:, 1]]
    bad = lab[pick] != two[:, 0]
    assert np.all(b2[bad] - b1[bad] <= 1e-5 * np.maximum(1.0, b1[bad]) + 1e-9), int(bad.sum())
    assert np.isfinite(sse) and sse > 0
