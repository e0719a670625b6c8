"""The tensor-core assignment (TF32 / BF16 operands, float32 accumulation, near ties
re-scored in float32) against the float32 direct path and the oracle."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

PRECS = [("tf32", B.PSCL_PREC_TF32), ("bf16", B.PSCL_PREC_BF16), ("tf32x3", B.PSCL_PREC_TF32X3),
         ("bf16x3", B.PSCL_PREC_BF16X3)]


@pytest.mark.parametrize("name,prec", PRECS)
@pytest.mark.parametrize("n,d,N,lk,fk,T", [
    (8192, 16, 1024, 16, 8, 4),        # k = 16: the smallest MMA N
    (30000, 16, 4096, 64, 32, 6),      # the headline shape, smaller
    (12000, 32, 2000, 100, 50, 4),     # N = 112 with 12 padded columns
    (9000, 64, 3000, 100, 64, 3),      # wide points, N = 112
    (5000, 4, 2500, 256, 16, 3),       # k = 256: the widest MMA N
    (7777, 8, 700, 33, 20, 5),         # ragged units and sets
])
def test_tensor_core_labels_equal_float32(name, prec, n, d, N, lk, fk, T):
    raw = synth.mixture(n, d, 10, outlier_frac=0.01, seed=2000 + n + d)
    ref = run_gpu(raw, N, lk, fk, T, seed=3, trace=False)
    got = run_gpu(raw, N, lk, fk, T, seed=3, trace=False, prec=prec)
    np.testing.assert_array_equal(got.perm, ref.perm)
    np.testing.assert_array_equal(got.local_centers, ref.local_centers)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    np.testing.assert_array_equal(got.labels, ref.labels)
    assert got.sse == ref.sse
    # the tensor cores did the work: every assignment went through them, and part of the
    # rows were decided by the contraction alone (the rest are near ties within the
    # worst-case operand-rounding bound, re-scored in float32)
    assert ref.rechecked == 0 and ref.assigned == 0
    P = got.local_centers.shape[0]
    assert got.assigned == (n + P) * T
    assert got.rechecked < 0.99 * max(got.assigned, 1), (got.rechecked, got.assigned)
    print(f"{name} n={n} d={d} k={lk}: re-scored {got.rechecked} of {got.assigned} rows")


def test_tensor_core_falls_back_above_256_centers():
    # more than 256 centers per set exceed one MMA: those sets take the float32 kernel
    # (same labels), the final set of 64 centers the tensor cores
    raw = synth.mixture(9000, 32, 10, seed=2099)
    ref = run_gpu(raw, 3000, 300, 64, 3, seed=3, trace=False)
    got = run_gpu(raw, 3000, 300, 64, 3, seed=3, trace=False, prec=B.PSCL_PREC_TF32)
    np.testing.assert_array_equal(got.labels, ref.labels)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    assert got.assigned == got.local_centers.shape[0] * 3


@pytest.mark.parametrize("name,prec", [("tf32", B.PSCL_PREC_TF32), ("bf16", B.PSCL_PREC_BF16),
                                       ("bf16x3", B.PSCL_PREC_BF16X3)])
def test_tensor_core_with_sums_in_global_memory(name, prec):
    # 256 centers of 64 attributes: operands fit shared memory, the exact sums do not and
    # go straight to the global sums; labels and centers still equal the float32 path
    raw = synth.mixture(20000, 64, 40, seed=2100)
    ref = run_gpu(raw, 5000, 256, 64, 3, seed=3, trace=False)
    got = run_gpu(raw, 5000, 256, 64, 3, seed=3, trace=False, prec=prec)
    np.testing.assert_array_equal(got.labels, ref.labels)
    np.testing.assert_array_equal(got.local_centers, ref.local_centers)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    assert got.assigned == (20000 + got.local_centers.shape[0]) * 3


@pytest.mark.parametrize("name,prec", PRECS)
def test_tensor_core_oracle_parity(name, prec):
    w = synth.SMALL
    raw = w.points()
    g = run_gpu(raw, w.N, w.local_k, w.final_k, w.iters, seed=11, prec=prec)
    o = run_oracle(raw, w.N, w.local_k, w.final_k, w.iters, seed=11, gpu=g)
    compare(g, o)
