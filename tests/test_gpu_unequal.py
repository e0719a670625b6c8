"""Unequal-sized subclustering (Algorithm 2) on the GPU against the oracle: landmarks on
the segment from L to H, the grouping (bit-exact), then the same Lloyd stages."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,d,blobs,out,m,lk,fk,T", [
    (4096, 4, 3, 0.0, 16, 16, 3, 20),          # the small workload's shape
    (20000, 16, 30, 0.05, 64, 12, 20, 6),      # outliers: the case Algorithm 2 is for
    (9000, 5, 8, 0.01, 40, 9, 10, 5),          # generic d
    (30000, 32, 50, 0.0, 300, 8, 40, 4),       # many landmarks, some without points
    (12000, 64, 20, 0.02, 32, 20, 16, 3),
])
def test_unequal_matches_oracle(n, d, blobs, out, m, lk, fk, T):
    raw = synth.mixture(n, d, blobs, outlier_frac=out, seed=5000 + n + m)
    g = run_gpu(raw, 0, lk, fk, T, seed=13, unequal_m=m)
    o = run_oracle(raw, 0, lk, fk, T, seed=13, gpu=g, unequal_m=m)
    r = compare(g, o)
    print(f"n={n} d={d} m={m}: {len(g.seg_off) - 1} subclusters, sizes {np.diff(g.seg_off).min()}..{np.diff(g.seg_off).max()}, {r}")


def test_unequal_ties_between_landmarks():
    # a 1-D grid whose points sit exactly between two landmarks: the lower one wins
    x = np.repeat(np.arange(0, 33, dtype=np.float32) / 32, 5)[:, None]
    x = np.ascontiguousarray(np.concatenate([x, np.zeros_like(x)], axis=1))
    g = run_gpu(x, 0, 2, 2, 3, seed=1, unequal_m=8)
    o = run_oracle(x, 0, 2, 2, 3, seed=1, gpu=g, unequal_m=8)
    compare(g, o)


def test_unequal_then_equal_on_the_same_job():
    raw = synth.mixture(8000, 8, 10, seed=6001)
    with B.Job(raw) as j:
        j.option(B.PSCL_OPT_TRACE_LABELS)
        j.steps_unequal(32, 8, 10, 4, 3)
        pu, ou = j.partition()
        j.steps(1000, 8, 10, 4, 3)
        pe, oe = j.partition()
    ref = run_gpu(raw, 1000, 8, 10, 4, seed=3, trace=False)
    np.testing.assert_array_equal(pe, ref.perm)
    o = run_oracle(raw, 0, 8, 10, 4, seed=3, unequal_m=32)
    np.testing.assert_array_equal(pu, o.perm)
    np.testing.assert_array_equal(ou, o.seg_off)
