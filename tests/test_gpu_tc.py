"""The tensor-core assignment (TF32 / BF16 operands, float32 accumulation, near ties
re-scored in float32) against the float32 direct path and the oracle.

The assignment step of Lloyd's iteration (Section 3.2, Eq. 1) served by tcgen05: the
labels, centers and SSE must equal the float32 direct path's bit for bit, since every row
whose tensor-core value is not a clear winner is re-scored with the float32 arithmetic."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

def served(d, k, prec):
    """Whether a set of k centers of d attributes runs on the tensor cores: d in {16, 32,
    64, 128}, k <= 256, and the two operand stages, two point stages and operand B within
    one CTA's shared memory (which leaves out d = 64 in TF32x3 above 16 centers and d = 128
    except BF16 with 16 centers)."""
    if prec == B.PSCL_PREC_TC:
        return served(d, k, B.PSCL_PREC_TF32X3) or served(d, k, B.PSCL_PREC_BF16X3)
    if d not in (16, 32, 64, 128) or k > 256:
        return False
    if d == 64 and prec == B.PSCL_PREC_TF32X3:
        return k <= 16
    if d == 128:
        return prec == B.PSCL_PREC_BF16 and k <= 16
    return True


PRECS = [("tf32", B.PSCL_PREC_TF32), ("bf16", B.PSCL_PREC_BF16), ("tf32x3", B.PSCL_PREC_TF32X3),
         ("bf16x3", B.PSCL_PREC_BF16X3), ("tc", B.PSCL_PREC_TC)]


@pytest.mark.parametrize("name,prec", PRECS)
@pytest.mark.parametrize("n,d,N,lk,fk,T", [
    (8192, 16, 1024, 16, 8, 4),        # k = 16: the smallest MMA N
    (30000, 16, 4096, 64, 32, 6),      # the headline shape, smaller
    (12000, 32, 2000, 100, 50, 4),     # N = 112 with 12 padded columns
    (9000, 64, 3000, 100, 64, 3),      # wide points, N = 112
    (5000, 16, 2500, 256, 16, 3),      # k = 256: the widest MMA N
    (7777, 32, 700, 33, 20, 5),        # ragged units and sets
    (6000, 128, 2000, 16, 16, 3),      # d = 128: four TMA boxes per row
    (3001, 128, 1500, 12, 10, 3),      # d = 128, ragged tiles and sets
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
    assert got.assigned == (n * served(d, lk, prec) + P * served(d, fk, prec)) * T
    assert got.rechecked < 0.99 * max(got.assigned, 1), (got.rechecked, got.assigned)
    print(f"{name} n={n} d={d} k={lk}: re-scored {got.rechecked} of {got.assigned} rows")


@pytest.mark.parametrize("d", [4, 8, 12])
def test_tensor_core_falls_back_for_other_widths(d):
    # d outside {16, 32, 64, 128} takes the float32 kernel: same labels, nothing assigned
    # by the tensor cores
    raw = synth.mixture(6000, d, 10, seed=2090 + d)
    ref = run_gpu(raw, 1500, 40, 16, 3, seed=3, trace=False)
    got = run_gpu(raw, 1500, 40, 16, 3, seed=3, trace=False, prec=B.PSCL_PREC_BF16X3)
    np.testing.assert_array_equal(got.labels, ref.labels)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    assert got.assigned == 0


def test_tensor_core_falls_back_above_256_centers():
    # more than 256 centers per set exceed one MMA: those sets take the float32 kernel
    # (same labels), the final set of 64 centers the tensor cores
    raw = synth.mixture(9000, 32, 10, seed=2099)
    ref = run_gpu(raw, 3000, 300, 64, 3, seed=3, trace=False)
    got = run_gpu(raw, 3000, 300, 64, 3, seed=3, trace=False, prec=B.PSCL_PREC_TF32)
    np.testing.assert_array_equal(got.labels, ref.labels)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    assert got.assigned == got.local_centers.shape[0] * 3
    assert not served(32, 300, B.PSCL_PREC_TF32) and served(32, 64, B.PSCL_PREC_TF32)


@pytest.mark.parametrize("name,prec", [("tf32", B.PSCL_PREC_TF32), ("bf16", B.PSCL_PREC_BF16),
                                       ("bf16x3", B.PSCL_PREC_BF16X3), ("tc", B.PSCL_PREC_TC)])
def test_tensor_core_256_centers_of_64_attributes(name, prec):
    # the precision workload's set shape: 256 centers of 64 attributes, the largest operand
    # B and the largest shared sums; labels and centers still equal the float32 path
    raw = synth.mixture(20000, 64, 40, seed=2100)
    ref = run_gpu(raw, 5000, 256, 64, 3, seed=3, trace=False)
    got = run_gpu(raw, 5000, 256, 64, 3, seed=3, trace=False, prec=prec)
    np.testing.assert_array_equal(got.labels, ref.labels)
    np.testing.assert_array_equal(got.local_centers, ref.local_centers)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    assert got.assigned == (20000 + got.local_centers.shape[0]) * 3


@pytest.mark.parametrize("name,prec", PRECS)
@pytest.mark.parametrize("n,d,N,lk,fk,T", [
    (8192, 16, 1024, 16, 8, 4),
    (4000, 32, 1000, 40, 20, 3),       # ragged tiles and sets
])
def test_tensor_core_oracle_parity(name, prec, n, d, N, lk, fk, T):
    raw = synth.mixture(n, d, 8, outlier_frac=0.01, seed=2200 + d)
    g = run_gpu(raw, N, lk, fk, T, seed=11, prec=prec)
    o = run_oracle(raw, N, lk, fk, T, seed=11, gpu=g)
    compare(g, o)
    assert g.assigned > 0


@pytest.mark.parametrize("name,prec", [("tc", B.PSCL_PREC_TC), ("bf16", B.PSCL_PREC_BF16)])
@pytest.mark.parametrize("n,d,N,lk,fk", [
    (40000, 64, 2000, 64, 1000),       # four chunks of centers, the last of 232
    (30000, 16, 1500, 40, 512),        # two full chunks
    (20000, 32, 1000, 20, 300),        # one full chunk and 44 more
    (9000, 32, 1000, 16, 100),         # one chunk
])
def test_final_stage_in_center_chunks(name, prec, n, d, N, lk, fk):
    # the SSE pass on the tensor cores, the centers in chunks of up to 256: labels and the
    # SSE equal the float32 pass bit for bit (near ties and rows another chunk comes close
    # to re-scored in float32; the SSE summed in the float32 pass's order)
    # (past 256 centers the pooled set's Lloyd iterations take the same chunked search, its
    # sums then in global memory: the label trace and the centers equal the float32 run's)
    raw = synth.mixture(n, d, 50, outlier_frac=0.01, seed=2300 + fk)
    ref = run_gpu(raw, N, lk, fk, 3, seed=5)
    got = run_gpu(raw, N, lk, fk, 3, seed=5, prec=prec)
    np.testing.assert_array_equal(got.trace_final, ref.trace_final)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    np.testing.assert_array_equal(got.labels, ref.labels)
    assert got.sse == ref.sse
