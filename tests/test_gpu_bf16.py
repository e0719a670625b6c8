"""Jobs stored in bfloat16: the points are bfloat16, the scaled values are rounded once to
bfloat16 (then everything runs as for float32 storage); against the oracle with the same
storage rule, on the host and device input paths, and through the job server."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import TIE_TOL, compare, run_gpu

import oracle

pytestmark = pytest.mark.gpu


def to_bf16(x):
    """float32 -> (bfloat16 bit patterns, their float32 values), round to nearest even."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
    return r, (r.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("n,d,N,lk,fk,T", [(4096, 4, 256, 16, 3, 20), (30000, 16, 2000, 20, 16, 5),
                                            (9000, 32, 1000, 12, 10, 4)])
def test_bf16_storage_matches_oracle(n, d, N, lk, fk, T):
    bits, vals = to_bf16(synth.mixture(n, d, 12, outlier_frac=0.01, seed=7000 + n))
    g = run_gpu(bits, N, lk, fk, T, seed=5)
    o = oracle.two_level(vals, N, lk, fk, T, 5, bf16=True, force_local=g.trace_local, force_final=g.trace_final,
                         tie_tol=TIE_TOL)
    compare(g, o)
    # the scaled values are bfloat16 values
    assert np.all((g.scaled.view(np.uint32) & 0xFFFF) == 0)


def test_bf16_device_input_and_graph_replay():
    import torch
    bits, vals = to_bf16(synth.mixture(20000, 16, 10, seed=7100))
    ref = run_gpu(bits, 2000, 16, 8, 5, seed=2, trace=False)
    dev = torch.from_numpy(vals).cuda().to(torch.bfloat16)
    got = run_gpu(dev, 2000, 16, 8, 5, seed=2, trace=False, graph=True, runs=2)
    np.testing.assert_array_equal(got.perm, ref.perm)
    np.testing.assert_array_equal(got.final_centers, ref.final_centers)
    assert got.sse == ref.sse


def test_bf16_footprint_and_serving():
    import torch
    bits, vals = to_bf16(synth.mixture(12000, 8, 6, seed=7200))
    ctx = B.pscl_ctx_create(0)
    j = B.Job(bits, ctx=ctx)
    j.run(200, 8, 8, 3, 1)
    c_alone, _, sse_alone = j.result(labels=False)
    assert B.pscl_ctx_bytes_in_use(ctx) == B.pscl_job_footprint(ctx, 12000, 8, 200, 8, 8, 3, on_device=False,
                                                                dtype=B.PSCL_BF16)
    j.close()
    B.pscl_ctx_destroy(ctx)
    dev = torch.from_numpy(vals).cuda().to(torch.bfloat16)
    with B.Server(slots=2) as s:
        t = s.submit(dev, 200, 8, 8, 3, 1)
        s.wait(t)
        c, _, sse, _ = s.fetch(t)
    np.testing.assert_array_equal(c, c_alone)
    assert sse == sse_alone
