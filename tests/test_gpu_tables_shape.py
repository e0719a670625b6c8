"""The shape of the paper's timing runs (Tables 2 and 3): 2-D points, exactly 500 per
blob, k = n / 500; one-level Lloyd on all points (a batch of one instance) and the
two-level method at compression c = N / local_k, both against the oracle."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import synth
from tests.parity import compare, compare_batch, run_gpu, run_gpu_batch, run_oracle

pytestmark = pytest.mark.gpu

N_SUB = 1000


@pytest.mark.parametrize("c", [5, 10, 15, 20])
def test_two_level_at_compression_matches_oracle(c):
    raw = synth.blob_points(40, 500, 2, seed=synth.BASE_SEED + 91)
    k, lk, T = 40, -(-N_SUB // c), 10
    g = run_gpu(raw, N_SUB, lk, k, T, seed=3)
    o = run_oracle(raw, N_SUB, lk, k, T, seed=3, gpu=g)
    r = compare(g, o)
    assert len(g.local_centers) == 20 * lk
    print(f"compression {c}: SSE {g.sse:.6g}; {r}")


def test_one_level_on_all_points_matches_oracle():
    raw = synth.blob_points(40, 500, 2, seed=synth.BASE_SEED + 91)
    g = run_gpu_batch([raw], [40], 10, seed=3)
    compare_batch(g, [raw], [40], 10, seed=3)

