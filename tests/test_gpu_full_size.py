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
