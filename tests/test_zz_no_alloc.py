"""pscl_assign_sse_noalloc: the nearest-center + SSE step for callers that cannot allocate.

Some callers may not allocate device memory at all (their framework's allocator owns the
device, or allocation is forbidden once they are running).  This entry point runs the
SSE step's kernel with its scratch in a fixed array inside the library; the caller passes
the points, the centers and the output buffers.  Here its results are checked against
those of the normal path (pscl_cluster + pscl_get_result) on the same job, on two calls
in a row (the second one reuses the scratch the first one left behind).

This file is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import SSE_TOL

pytestmark = pytest.mark.gpu


def test_noalloc_matches_the_cluster_step_twice():
    import torch
    raw = synth.mixture(60000, 16, 20, outlier_frac=0.01, seed=4242)
    with B.Job(raw) as job:
        job.steps(4096, 32, 16, 6, seed=8)
        scaled = job.scaled()
        centers, labels, sse = job.result()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pts = torch.from_numpy(scaled).to(dev)
    cen = torch.from_numpy(centers).to(dev)
    stream = torch.cuda.Stream(dev)
    for call in range(2):
        out_lab = torch.full((len(scaled),), -1, dtype=torch.int32, device=dev)
        out_sse = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            B.pscl_assign_sse_noalloc(pts, cen, out_lab, out_sse, stream=stream.cuda_stream)
        stream.synchronize()
        np.testing.assert_array_equal(out_lab.cpu().numpy(), labels)
        got = float(out_sse.cpu().item())
        assert abs(got - sse) <= SSE_TOL * abs(sse), (call, got, sse)


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    dev = torch.device("cuda", 0)
    lib = B.lib()
    pts = torch.zeros((8, 4), dtype=torch.float32, device=dev)
    cen = torch.zeros((2, 4), dtype=torch.float32, device=dev)
    lab = torch.zeros(8, dtype=torch.int32, device=dev)
    sse = torch.zeros(1, dtype=torch.float64, device=dev)
    p = [t.data_ptr() for t in (pts, cen, lab, sse)]
    assert lib.pscl_assign_sse_noalloc(p[0], 0, 4, p[1], 2, p[2], p[3], None) == B.PSCL_EINVAL
    assert lib.pscl_assign_sse_noalloc(p[0], 8, 1025, p[1], 2, p[2], p[3], None) == B.PSCL_EINVAL
    assert lib.pscl_assign_sse_noalloc(p[0], 8, 4, p[1], 4097, p[2], p[3], None) == B.PSCL_EINVAL
    assert lib.pscl_assign_sse_noalloc(None, 8, 4, p[1], 2, p[2], p[3], None) == B.PSCL_EINVAL
    assert b"noalloc" in lib.pscl_last_error()
