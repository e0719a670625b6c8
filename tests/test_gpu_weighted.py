"""Count-weighted pooled Lloyd on the GPU against the oracle: every local center weighs
its cluster's size in the Lloyd on the pooled local centers (the abstract: the second
level clusters the subclusters' means)."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.golden_io import arr, load
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,d,blobs,N,lk,fk,T", [
    (4096, 4, 3, 256, 16, 3, 20),            # the small workload's shape
    (30000, 16, 64, 4096, 64, 64, 6),        # the headline shape, scaled down
    (20000, 32, 20, 1500, 40, 30, 5),        # ragged last subcluster
    (9000, 64, 12, 1000, 100, 64, 4),
    (5000, 7, 9, 333, 5, 12, 8),             # generic d, few local centers
])
def test_weighted_pooling_matches_oracle(n, d, blobs, N, lk, fk, T):
    raw = synth.mixture(n, d, blobs, outlier_frac=0.01, seed=7000 + n + d)
    g = run_gpu(raw, N, lk, fk, T, seed=21, pool_weighted=True)
    o = run_oracle(raw, N, lk, fk, T, seed=21, gpu=g, pool_weighted=True)
    r = compare(g, o)
    u = run_gpu(raw, N, lk, fk, T, seed=21)
    np.testing.assert_array_equal(u.local_centers, g.local_centers)      # first level unchanged
    assert np.abs(u.final_centers - g.final_centers).max() > 0             # the weights act
    print(f"n={n} d={d}: weighted SSE {g.sse:.6g} vs unweighted {u.sse:.6g}; {r}")


def test_weighted_pooling_on_the_worked_example():
    # the 10-point example with first-k init: the pooled weights are the local cluster
    # sizes (2, 2, 1, 3, 1, 1)
    gd = load("hand_2d.txt")
    N, lk, fk, T = (int(v) for v in gd["params"][0])
    raw = arr(gd["raw"], np.float32)
    g = run_gpu(raw, N, lk, fk, T, seed=0, first_k=True, pool_weighted=True)
    o = run_oracle(raw, N, lk, fk, T, seed=0, gpu=g, first_k=True, pool_weighted=True)
    compare(g, o)
    np.testing.assert_array_equal(g.counts, [2, 2, 1, 3, 1, 1])


@pytest.mark.parametrize("name,prec", [("bf16x3", B.PSCL_PREC_BF16X3), ("tf32", B.PSCL_PREC_TF32)])
def test_weighted_pooling_with_tensor_core_local_level(name, prec):
    # the local level on the tensor cores (labels equal float32's), the weighted pooled
    # Lloyd in float32 with global sums
    raw = synth.mixture(30000, 16, 40, seed=7101)
    ref = run_gpu(raw, 2000, 32, 24, 5, seed=4, trace=False, pool_weighted=True)
    got = run_gpu(raw, 2000, 32, 24, 5, seed=4, trace=False, pool_weighted=True, prec=prec)
    np.testing.assert_array_equal(got.local_centers, ref.local_centers)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    assert got.sse == ref.sse


def test_weighted_pooling_graph_replay_and_unequal_groups():
    raw = synth.mixture(12000, 8, 16, outlier_frac=0.02, seed=7201)
    a = run_gpu(raw, 900, 20, 16, 5, seed=8, trace=False, pool_weighted=True)
    b = run_gpu(raw, 900, 20, 16, 5, seed=8, trace=False, pool_weighted=True, graph=True, runs=2)
    np.testing.assert_array_equal(a.final_centers, b.final_centers)
    assert a.sse == b.sse
    g = run_gpu(raw, 0, 12, 16, 5, seed=8, unequal_m=40, pool_weighted=True)
    o = run_oracle(raw, 0, 12, 16, 5, seed=8, gpu=g, unequal_m=40, pool_weighted=True)
    compare(g, o)


def test_weighted_pooling_at_quarter_headline_size():
    w = synth.scaled_down(synth.MEDIUM, 1 << 18)
    raw = w.points()
    g = run_gpu(raw, w.N, w.local_k, w.final_k, w.iters, seed=w.seed, pool_weighted=True)
    o = run_oracle(raw, w.N, w.local_k, w.final_k, w.iters, seed=w.seed, gpu=g, pool_weighted=True)
    compare(g, o)
