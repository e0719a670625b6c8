"""Error of every precision mode against the FP64 oracle on the precision workload's shape
(d = 64, 1024 blobs, subclusters of N with 256 local centers, final k = 1024, 25
iterations), at n = 2^18 (16 subclusters of 16384) so that the oracle finishes.

The tensor-core modes re-score every near tie in float32, so their labels, and hence
centers and SSE, equal the float32 path's bit for bit; the error against the oracle is
the float32 path's.  The table printed here is the precision report."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

W = synth.scaled_down(synth.LARGE, 1 << 18, N=16384)
MODES = [("fp32", B.PSCL_PREC_FP32), ("tf32", B.PSCL_PREC_TF32), ("bf16", B.PSCL_PREC_BF16),
         ("tf32x3", B.PSCL_PREC_TF32X3), ("bf16x3", B.PSCL_PREC_BF16X3)]


def test_error_vs_oracle_per_mode():
    raw = W.points()
    runs = {name: run_gpu(raw, W.N, W.local_k, W.final_k, W.iters, seed=21, prec=prec) for name, prec in MODES}
    ref = runs["fp32"]
    o = run_oracle(raw, W.N, W.local_k, W.final_k, W.iters, seed=21, gpu=ref)
    print(f"\nprecision report, n={W.n} d={W.d} N={W.N} local_k={W.local_k} final_k={W.final_k} iters={W.iters}")
    print("mode    local_err  final_err  sse_rel   rechecked/assigned  replayed_ties  label_ties")
    for name, g in runs.items():
        np.testing.assert_array_equal(g.labels, ref.labels)
        np.testing.assert_array_equal(g.final_centers, ref.final_centers)
        r = compare(g, o)
        print(f"{name:7s} {r['local_center_err']:.2e}  {r['final_center_err']:.2e}  {r['sse_rel']:.2e}  "
              f"{g.rechecked:>9d}/{g.assigned:<9d}  {r['replayed_ties']:>13d}  {r['label_ties']:>10d}")
